"""The algorithmic FP32 operation count of the roofline, pinned to the oracle's own arithmetic.

The oracle tallies, beside its code, the fp32 operations of the per-pixel steps (G-buffer
interpolation, shading, grading, quantisation) that depend on the pixel, and once per image those
that depend on the image only.  bench.py's roofline computes the same count from a G-buffer with
per-term constants; these tests require the two to agree on scenes that exercise every term: point
lights with specular lobes, directional lights, orthographic cameras, spot cones (and a null cone),
emission and colour grading.  A one-pixel scene pins the constants themselves by hand.
"""

import numpy as np
import pytest

import bench
from paper_1906_11633_b300 import scenegen as sg
from tests import scenes


def _bench_count(oracle, b):
    o = oracle.render(b, gbuffer=True, flops=True)
    return o["flops"], bench.alg_flops(b, o["gb_pos"], o["gb_nrm"], o["gb_mat"]), o


def _directional_ortho(b):
    light = b.light.copy()
    d = light[:, :, :3].astype(np.float64)
    d /= np.maximum(np.linalg.norm(d, axis=-1, keepdims=True), 1e-9)
    light[:, :, :3] = d.astype(np.float32)
    meta = b.light_meta.copy()
    meta[:, 1] = sg.LIGHT_DIRECTIONAL
    intr = b.cam_intr.copy()
    ortho = np.arange(len(intr)) % 2 == 1
    intr[ortho, 0] = intr[ortho, 1] = 64 / 0.7
    intr[ortho, 5] = sg.CAM_ORTHOGRAPHIC
    return b.with_params(light=light, light_meta=meta, cam_intr=intr)


def _null_cone(b):
    spot = b.light_spot.copy()
    spot[:, 1, 4] = spot[:, 1, 3]      # light 1: inner = outer, a null cone that lights nothing
    return b.with_params(light_spot=spot)


@pytest.mark.parametrize("kind", ["hand", "tiny", "dir_ortho", "spot_grade", "null_cone"])
def test_bench_count_equals_the_oracle_tally(oracle, kind):
    if kind == "hand":
        b = sg.hand_batch(2, np.arange(6), res=64)
    elif kind == "tiny":
        b = sg.tiny_batch(3, n_samples=4, res=48)
    elif kind == "dir_ortho":
        b = _directional_ortho(sg.hand_batch(4, np.arange(4), res=64))
    elif kind == "spot_grade":
        b = sg.benchmark_batch(5, np.arange(4), res=64)
        assert b.grading is not None and b.light_spot is not None
    else:
        b = _null_cone(sg.benchmark_batch(6, np.arange(3), res=64))
    want, got, o = _bench_count(oracle, b)
    assert (o["gb_mat"] >= 0).sum() > 1000
    # the lit test n . L > 0 is taken in fp64 by the bench and in fp32 by the oracle: a pixel whose
    # n . L is within rounding of 0 may count differently (21 operations each)
    assert abs(got - want) <= max(21 * 4, 1e-5 * want), (got, want)


def _one_pixel(lights, light_type=sg.LIGHT_POINT, specular=0.5, ortho=False):
    # a 1x1 image whose pixel sees the plane z = 0 from 1 m above
    view, intr, wh = scenes.camera_down((0.0, 0.0, 1.0), 1, 1, px_per_m=1.0 if ortho else None,
                                        fovy_deg=None if ortho else 45.0)
    return scenes.single_sample([sg.plane_mesh(1, 1)], [0], [scenes.identity_pose()], [(view, intr, wh)],
                                lights=lights, light_type=light_type, specular=specular, shininess=8.0)


def test_one_pixel_counts_by_hand(oracle):
    # per image: the two reciprocal focal lengths (2) and 2^EV (1); the pixel: 43 for the G-buffer
    # (3 conversions, 3 perspective products, 15 for the interpolated normal, 6 for its length, 1
    # test, 3 divisions, 4 + 5 for the pixel ray, 3 for the position), 12 for the view vector, 15
    # for ambient, emission and exposure, 18 for three quantisations and 3 binary16 conversions
    base = 3 + 43 + 12 + 15 + 18 + 3
    o = oracle.render(_one_pixel([]), flops=True)
    assert o["seg"][0] == 1 and o["flops"] == base
    # a point light above the pixel: 18 per image to move it to view space; per pixel 13 for the
    # light vector, its length and the falloff, 1 for the shadow factor, 6 for n . L with its
    # clamp, 1 test, and since it lights the surface 9 + 12 for the half vector and the lobe; then
    # 12 for the colour sums
    o = oracle.render(_one_pixel([((0.0, 0.0, 0.5), 1.0)]), flops=True)
    assert o["flops"] == base + 18 + 13 + 1 + 6 + 1 + 9 + 12 + 12
    # the same light below the plane lights nothing: no half vector, no lobe
    o = oracle.render(_one_pixel([((0.0, 0.0, -0.5), 1.0)]), flops=True)
    assert o["flops"] == base + 18 + 13 + 1 + 6 + 1 + 12
    # an orthographic camera: no perspective products (3), a position of one negation (1 instead
    # of 3) and no view vector (12)
    o = oracle.render(_one_pixel([], ortho=True), flops=True)
    assert o["seg"][0] == 1 and o["flops"] == base - 3 - 2 - 12
