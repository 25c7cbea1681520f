"""Exact depth ties and the narrowest supported spot cone on the GPU, against the oracle.

- Coplanar quads: two instances of one quad mesh at the same pose give every covered pixel two
  fragments of bit-equal depth; the (depth, key) order gives each pixel to the lower primitive id,
  so the first instance in the list wins everywhere, and swapping the list swaps the winner.  A
  smaller quad in the same plane overlapping a larger one ties only where they overlap.  Every
  pixel is one of these exact ties, so `seg` is compared with the oracle outright (no tie
  allowance), in fused and plain launches.
- Spot cones: the GPU folds 1/(cos_i - cos_o) into the cone axis, which amplifies the rounding of
  the cosine by that factor; at the narrowest ramp the library supports, cos_i - cos_o = 0.01, the
  channels still match the oracle within the contract (rgb_linear 1e-4, rgb8 1 LSB).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_11633_b300 import lib as L
from paper_1906_11633_b300 import scenegen as sg
from paper_1906_11633_b300.render import Renderer, config, to_numpy
from tests import scenes
from tests.parity import compare


@pytest.fixture(scope="module")
def oracle():
    from oracle import oracle as orc
    orc.build()
    return orc


def _quads(order, second_half=1.0):
    big = sg.quad_mesh([(-1, -1, 0), (1, -1, 0), (1, 1, 0), (-1, 1, 0)], (0, 0, 1))
    # (a quad that sticks out past the large one's edge at x = 1: it ties where they overlap)
    h = second_half
    small = sg.quad_mesh([(0.4, -h, 0), (1.3, -h, 0), (1.3, 0.3, 0), (0.4, 0.3, 0)], (0, 0, 1))
    cam = scenes.camera_down((0.1, 0.05, 3.0), 48, 40, fovy_deg=50)
    meshes = [big, small] if second_half != 1.0 else [big]
    inst = [0, 1] if second_half != 1.0 else [0, 0]
    seg = np.array([7, 9])
    return scenes.single_sample(meshes, list(np.array(inst)[order]), [scenes.identity_pose()] * 2, [cam],
                                seg=seg[order], lights=[((0.2, 0.1, 1.5), 1.0)])


@pytest.mark.parametrize("mode", [L.ORRB_MODE_FUSED, L.ORRB_MODE_PLAIN])
def test_coplanar_ties_go_to_the_lower_primitive(oracle, mode):
    for second_half, order in [(1.0, [0, 1]), (1.0, [1, 0]), (0.6, [0, 1]), (0.6, [1, 0])]:
        b = _quads(order, second_half)
        r = Renderer(b.meshes)
        g = to_numpy(r.render(r.upload(b), cfg=config(mode=mode), rgb_linear=True))
        torch.cuda.synchronize()
        assert r.status() == 0
        o = oracle.render(b, debug=True)
        hit = o["prim"] >= 0
        assert hit.sum() > 300
        np.testing.assert_array_equal(g["seg"], o["seg"])          # outright, ties included
        np.testing.assert_array_equal(g["depth"], o["depth"])
        first = np.array([7, 9])[order][0]
        if second_half == 1.0:                                    # identical quads: the first wins
            assert np.all(g["seg"][hit] == first)
        else:                                                     # both show; the overlap is the first's
            assert set(np.unique(g["seg"][hit])) == {7, 9}
            overlap = (o["prim"] >= 0) & (o["depth2"] == o["depth"])
            assert overlap.sum() > 30 and np.all(g["seg"][overlap] == first)
        assert np.abs(g["rgb"].astype(int) - o["rgb"].astype(int)).max() <= 1


def test_narrowest_spot_cone_ramp_matches_the_oracle(oracle):
    b = sg.benchmark_batch(12, np.arange(6), res=96, grading=False)
    spot = b.light_spot.copy()
    spot[:, :, 4] = spot[:, :, 3] + 0.01       # cos_i - cos_o = 0.01 on every light
    b = b.with_params(light_spot=spot)
    r = Renderer(b.meshes)
    g = to_numpy(r.render(r.upload(b), rgb_linear=True))
    torch.cuda.synchronize()
    assert r.status() == 0
    o = oracle.render(b, debug=True)
    # the ramp is crossed by many pixels, so the amplified rounding is exercised
    compare(g, o, "narrow spot ramp")
    assert np.abs(g["rgb_linear"] - o["rgb_linear"]).max() <= 1e-4
