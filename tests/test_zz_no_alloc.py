"""The allocation-free entry point, orrb_render_batch_noalloc.

It exists for callers that may not call cudaMalloc: code running inside another
runtime that owns the GPU's memory pool (a framework's custom op, a simulator's
render callback), where the pool holds the memory or an allocation could
synchronise the device mid-pipeline.  Instead of a caller workspace it uses one
static device array inside the library.  This test calls it through the C-ABI
twice in a row (two different batches, so stale contents of the shared array
would show) and checks each result against the workspace-based entry point,
orrb_render_batch, at the renderer's parity tolerances -- in practice the two
are bit-identical, since both run the same kernel.  It also checks the
rejection of a shape whose scratch slot cannot fit in the static array.

The file name makes pytest collect it last.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_11633_b300 import lib as L
from paper_1906_11633_b300 import scenegen as sg
from paper_1906_11633_b300.render import Renderer, config, to_numpy
from tests.parity import f16_ordered


def _outs(out):
    return L.orrb_outputs(*[out[k].data_ptr() if k in out else None
                            for k in ("rgb", "depth", "normal", "seg", "rgb_linear", "gbuffer")])


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    r = Renderer(sg.hand_meshes())
    stream = torch.cuda.current_stream().cuda_stream
    status = torch.full((1,), 0xFF, dtype=torch.int32, device="cuda")
    for seed, res in ((11, 200), (12, 128)):
        b = sg.hand_batch(seed, np.arange(6), res=res)
        db = r.upload(b)
        ref = to_numpy(r.render(db, rgb_linear=True))
        out = r.alloc_outputs(db.total_pixels, rgb_linear=True)
        for v in out.values():
            v.fill_(0x5A)
        L.orrb_render_batch_noalloc(r.ctx, db.shape, db.desc, _outs(out), config(), status.data_ptr(), stream)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        got = to_numpy(out)
        np.testing.assert_array_equal(got["seg"], ref["seg"])
        np.testing.assert_array_equal(got["depth"], ref["depth"])
        assert np.abs(got["rgb"].astype(int) - ref["rgb"].astype(int)).max() <= 1
        assert np.abs(got["rgb_linear"] - ref["rgb_linear"]).max() <= 1e-4
        ulp = np.abs(f16_ordered(got["normal"]) - f16_ordered(ref["normal"]))
        assert ulp.max() <= 1


def test_noalloc_rejects_shapes_beyond_its_static_scratch():
    r = Renderer(sg.hand_meshes())
    b = sg.hand_batch(0, np.arange(1), res=64)
    db = r.upload(b)
    shape = L.orrb_batch_shape(db.shape.n_samples, db.shape.n_cams, 1 << 26, db.shape.max_inst_per_sample,
                               db.shape.max_cams_per_sample, db.shape.max_width, db.shape.max_height,
                               db.shape.total_pixels)
    out = r.alloc_outputs(db.total_pixels)
    with pytest.raises(L.OrrbError) as e:
        L.orrb_render_batch_noalloc(r.ctx, shape, db.desc, _outs(out), config(), None,
                                    torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 2
    assert "static scratch" in str(e.value)


def test_noalloc_shadows_count_every_tap_like_the_shortcut():
    """With shadows the workspace entry point settles lit and umbra points from the maps'
    neighbourhood table; the allocation-free one has no room for it and counts all nine taps every
    time.  Maps, G-buffer words (the tap counts) and channels must agree exactly."""
    r = Renderer(sg.hand_meshes())
    stream = torch.cuda.current_stream().cuda_stream
    status = torch.full((1,), 0xFF, dtype=torch.int32, device="cuda")
    b = sg.benchmark_batch(14, np.arange(4), res=96, shadow_res=128)
    db = r.upload(b)
    ref = to_numpy(r.render(db, rgb_linear=True, gbuffer=True))
    out = r.alloc_outputs(db.total_pixels, rgb_linear=True, gbuffer=True)
    out["shadow_map"] = r.alloc_shadow_maps(db)
    outs = _outs(out)
    outs.shadow_map = out["shadow_map"].data_ptr()
    L.orrb_render_batch_noalloc(r.ctx, db.shape, db.desc, outs, config(), status.data_ptr(), stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = to_numpy(out)
    cast = np.arange(4)[None, :] < b.light_meta[:, :1]
    np.testing.assert_array_equal(got["shadow_map"][cast], ref["shadow_map"][cast])
    words = got["gbuffer"][6].view(np.int32)
    np.testing.assert_array_equal(words, ref["gbuffer"][6].view(np.int32))
    assert (words[words >= 0] > 0xff).mean() > 0.05
    for k in ("rgb", "rgb_linear", "depth", "seg", "normal"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
