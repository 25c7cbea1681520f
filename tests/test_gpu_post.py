"""Ambient occlusion and bloom (the post pass after the camera launch) on the GPU against the oracle's
step 17, and the pass's contract:

- parity: rgb8 within 1 LSB and the graded colour (rgb_graded, the colour quantisation reads)
  within 2e-4 of the oracle's fp64 step 17 followed by its fp32 grading, on the benchmark-like
  batch (spot lights, emission, grading), with shadows, and on ragged image sizes with the largest
  blur radius; the other channels as in every parity test;
- intensities of zero give the bits of the same batch without post-processing;
- fused and plain launches agree bit for bit, and so do renders that leave depth, normal and
  rgb_linear to the workspace;
- the entry points that cannot run the pass reject it.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_11633_b300 import lib as L
from paper_1906_11633_b300 import scenegen as sg
from paper_1906_11633_b300.render import Renderer, config, to_numpy
from tests.parity import compare

FINAL_TOL = 2e-4


@pytest.fixture(scope="module")
def oracle():
    from oracle import oracle as orc
    orc.build()
    return orc


@pytest.fixture(scope="module")
def renderer():
    return Renderer(sg.hand_meshes())


def _render(r, b, **kw):
    g = to_numpy(r.render(r.upload(b), rgb_linear=True, rgb_graded=True, **kw))
    torch.cuda.synchronize()
    assert r.status() == 0
    return g


def _check(g, o, label):
    st = compare(g, o, label)
    assert st["flips"] == 0
    e = np.abs(g["rgb_graded"].astype(np.float64) - o["rgb_final"])
    assert e.max() <= FINAL_TOL * max(1.0, float(np.abs(o["rgb_final"]).max())), (label, e.max())
    assert np.abs(g["rgb"].astype(int) - o["rgb"].astype(int)).max() <= 1, label
    return e.max()


@pytest.mark.parametrize("shadows", [False, True])
def test_post_matches_the_oracle(renderer, oracle, shadows):
    b = sg.benchmark_batch(21, np.arange(6), res=96, post=True, shadow_res=96 if shadows else 0)
    g = _render(renderer, b)
    o = oracle.render(b, debug=True)
    _check(g, o, f"post shadows={shadows}")
    none = oracle.render(b.with_params(post=None))
    assert np.abs(o["rgb"].astype(int) - none["rgb"].astype(int)).max() > 8   # the pass does something


def test_post_on_ragged_images_with_the_widest_blur(oracle):
    """Widths and heights that are not multiples of the pass's 128-pixel rows and 32 x 32 tiles,
    images narrower than the blur's reach, the 16-pixel truncation (sigma 6) and strong AO; a
    bright light so that bloom has work."""
    res = np.array([37, 130, 64, 17, 200, 96])
    b = sg.hand_batch(22, np.arange(6), res_per_sample=res, cams_per_sample=np.array([1, 2, 1, 3, 1, 2]))
    post = np.tile(np.array([[1.5, 1.0, 6.0, 0.0]], np.float32), (b.n_samples, 1))
    post[1, 2] = 2.5
    post[3] = [0.7, 0.5, 0.8, 0.0]
    light = b.light.copy()
    light[:, :, 3] *= 6.0
    b = b.with_params(post=post, light=light, grading=sg.grading_params(22, np.arange(6)))
    r = Renderer(b.meshes)
    g = _render(r, b)
    o = oracle.render(b, debug=True)
    _check(g, o, "ragged post")
    assert (o["rgb_linear"] > 1.0).any()


def test_zero_intensities_give_the_unprocessed_bits(renderer):
    b = sg.benchmark_batch(23, np.arange(4), res=80, post=True)
    zero = _render(renderer, b.with_params(post=np.zeros_like(b.post)))
    plain = _render(renderer, b.with_params(post=None))
    for k in plain:
        np.testing.assert_array_equal(zero[k], plain[k], err_msg=k)


def test_plain_and_staged_modes_and_workspace_images_agree(renderer):
    b = sg.benchmark_batch(24, np.arange(4), res=72, post=True)
    db = renderer.upload(b)
    fused = to_numpy(renderer.render(db, rgb_linear=True, rgb_graded=True))
    plain = to_numpy(renderer.render(db, cfg=config(mode=L.ORRB_MODE_PLAIN), rgb_linear=True, rgb_graded=True))
    staged = to_numpy(renderer.render(db, cfg=config(mode=L.ORRB_MODE_STAGED), rgb_linear=True, rgb_graded=True))
    for k in fused:
        np.testing.assert_array_equal(plain[k], fused[k], err_msg=k)
        np.testing.assert_array_equal(staged[k], fused[k], err_msg=k)
    # only rgb requested: depth, normal and the linear colour live in the workspace
    out = renderer.alloc_outputs(b.total_pixels)
    rgb_only = {"rgb": out["rgb"]}
    got = to_numpy(renderer.render(db, out=rgb_only))
    torch.cuda.synchronize()
    assert renderer.status() == 0
    np.testing.assert_array_equal(got["rgb"], fused["rgb"])


def test_entry_points_that_cannot_run_the_pass_reject_it(renderer):
    b = sg.benchmark_batch(25, np.arange(2), res=48, post=True)
    db = renderer.upload(b)
    shape = L.orrb_batch_shape.from_buffer_copy(db.shape)
    shape.post_effects = 0
    out = renderer.alloc_outputs(b.total_pixels)
    outs = L.orrb_outputs(*[out[k].data_ptr() if k in out else None for k in
                            ("rgb", "depth", "normal", "seg", "rgb_linear", "gbuffer", "tracker", "shadow_map",
                             "rgb_graded")])
    ws = renderer.workspace(db.shape, config())
    with pytest.raises(L.OrrbError) as e:
        L.orrb_render_batch(renderer.ctx, shape, db.desc, outs, config(), ws.data_ptr(), ws.numel(),
                            torch.cuda.current_stream().cuda_stream)
    assert e.value.status == L.ORRB_ERR_INVALID_ARG
    with pytest.raises(L.OrrbError) as e:
        L.orrb_render_batch_noalloc(renderer.ctx, db.shape, db.desc, outs, config(), None,
                                    torch.cuda.current_stream().cuda_stream)
    assert e.value.status == L.ORRB_ERR_UNSUPPORTED
    g = renderer.render(db, rgb_linear=True, gbuffer=True)
    with pytest.raises(L.OrrbError) as e:
        renderer.shade_backward(db, g["gbuffer"], torch.zeros_like(g["rgb_linear"]), grading=True)
    assert e.value.status == L.ORRB_ERR_UNSUPPORTED
