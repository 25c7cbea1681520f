"""Pins of the oracle's fp64 shading (the primal that the adjoint differentiates and that finite
differences are taken of) against things other than itself.

1. The fp64 shading of a rendered G-buffer equals the fp32 forward's rgb_linear of the same
   render, element by element: both evaluate the shading of step 10 (Blinn-Phong over point,
   directional or spot lights, emission, shadow factors of step 16, exposure) from the randomized
   material and light parameters of Sec. 4.3.1, but in separately written code (fp32 in the
   renderer, fp64 in the adjoint's primal).  A term dropped, transposed or mis-signed in either
   one shows up as a difference far above fp32 rounding.  Checked on the hand scene (1-4 point
   lights with specular lobes), the benchmark-like scene (three spot lights, emissive block) and
   the same scene with shadow maps (tap counts in the G-buffer material word).
2. Closed forms under a camera that is rotated and translated (so that a light moved to view
   space without the view translation, or with the rotation transposed, fails): the mirror
   configuration of a point light (the half vector equals the normal) gives the lobe
   k_s I / d^2 at any shininess plus the Lambert term rho I (n . v) / d^2; a spot light aimed at
   the point at full cone gives the same; one aimed away gives the ambient term alone.
"""

import numpy as np
import pytest

from paper_1906_11633_b300 import scenegen as sg
from tests import scenes

# fp32 forward against fp64: every value is below ~4 and passes through ~60 fp32 operations and
# one powf with an exponent of at most 128, so the fp32 result carries a relative error of a few
# 1e-7 (up to 128 x that in the lobe): 1e-5 absolute leaves a margin of several times that.
TOL_F32 = 1e-5


def _check_forward(oracle, b):
    o = oracle.render(b, gbuffer=True)
    rgb64 = oracle.shade_f64(b, o["gb_pos"], o["gb_nrm"], o["gb_mat"])
    ref = o["rgb_linear"].astype(np.float64)
    fg = o["gb_mat"] >= 0
    assert fg.sum() > 0.3 * fg.size
    err = np.abs(rgb64 - ref)
    assert err.max() <= TOL_F32, (err.max(), np.unravel_index(err.argmax(), err.shape))
    # background pixels carry the background colour on both sides
    assert np.array_equal(rgb64[~fg], ref[~fg])
    return o


def test_f64_shading_equals_forward_hand_point_lights(oracle):
    b = sg.hand_batch(5, np.arange(4), res=48)
    assert (b.material[:, :, 3] > 0).any() and (b.light_meta[:, 0] >= 2).any()
    _check_forward(oracle, b)


def test_f64_shading_equals_forward_spot_lights_and_emission(oracle):
    b = sg.benchmark_batch(6, np.arange(4), res=48)
    assert b.light_spot is not None and (b.emission > 0).any()
    _check_forward(oracle, b)


def test_f64_shading_equals_forward_with_shadow_factors(oracle):
    b = sg.benchmark_batch(7, np.arange(3), res=48, shadow_res=64)
    o = _check_forward(oracle, b)
    taps = (o["gb_mat"][o["gb_mat"] >= 0] >> 8) & 0xfff
    assert (taps != 0).any(), "the scene must have shadowed taps for the check to cover them"


def test_f64_shading_equals_forward_directional_lights(oracle):
    b = sg.tiny_batch(8, n_samples=3, res=40)
    b = b.with_params(material=b.material.copy())
    b.material[:, :2, 3] = 0.6
    b.material[:, :2, 4] = 20.0
    _check_forward(oracle, b)


# ---- closed forms -----------------------------------------------------------------------------

def _euler(rx, ry, rz):
    cx, sx, cy, sy, cz, sz = np.cos(rx), np.sin(rx), np.cos(ry), np.sin(ry), np.cos(rz), np.sin(rz)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def _mirror_case(alpha, ks, rho, I, d, ev, amb, spot=None):
    """One pixel whose G-buffer point P (view space) has unit normal n; a point light at
    P + d L_hat with L_hat the mirror of the view direction about n, so H = n.  Returns the fp64
    shading of that pixel and the closed form."""
    R = _euler(0.3, -0.5, 1.1)      # camera-from-world rotation
    t = np.array([0.4, -0.7, 1.3])  # camera-from-world translation
    view = np.concatenate([R, t[:, None]], 1)
    P = np.array([0.05, -0.08, -0.9])
    n = np.array([0.2, 0.3, 0.9])
    n /= np.linalg.norm(n)
    v = -P / np.linalg.norm(P)
    Lhat = 2.0 * np.dot(n, v) * n - v
    Lview = P + d * Lhat
    Lworld = R.T @ (Lview - t)      # so that R Lworld + t = Lview
    b = scenes.single_sample([sg.plane_mesh(1, 1)], [0], [scenes.identity_pose()],
                             [(view, sg.perspective_intrinsics(1, 1, 45.0), (1, 1))],
                             lights=[(Lworld, I)], light_type=sg.LIGHT_SPOT if spot is not None else sg.LIGHT_POINT,
                             albedo=rho, specular=ks, shininess=alpha, ev=ev, ambient=amb,
                             spots=None if spot is None else [spot(R, Lworld, P, t)])
    gb_pos = P.astype(np.float32)[None]
    gb_nrm = n.astype(np.float32)[None]
    gb_mat = np.zeros(1, np.int32)
    rgb = oracle_shade(b, gb_pos, gb_nrm, gb_mat)
    # the closed form from the float32 values the oracle reads: the G-buffer point and normal, the
    # camera matrix and the world light position, the light taken to view space exactly
    P32, n32 = gb_pos[0].astype(np.float64), gb_nrm[0].astype(np.float64)
    V32 = b.cam_view[0].astype(np.float64)
    L32 = V32[:, :3] @ b.light[0, 0, :3].astype(np.float64) + V32[:, 3]
    return rgb[0], P32, n32, L32, v


oracle_shade = None


@pytest.fixture(autouse=True)
def _bind(oracle):
    global oracle_shade
    oracle_shade = oracle.shade_f64


@pytest.mark.parametrize("alpha", [1.0, 7.5, 128.0])
def test_point_light_mirror_lobe_closed_form(alpha):
    ks, rho, I, d, ev = 0.75, np.array([0.0, 0.0, 0.0]), 1.5, 0.8, 0.25
    rgb, P, n, Lview, v = _mirror_case(alpha, ks, rho, I, d, ev, amb=(0.0, 0.0, 0.0))
    d_exact = np.linalg.norm(Lview - P)
    # the mirror: H = n / |n|, so n . H = |n| (1 up to the float32 rounding of the stored normal)
    expect = 2.0 ** ev * ks * np.linalg.norm(n) ** alpha * I / d_exact ** 2
    # (every parameter is exact in float32; the float32 rounding of the G-buffer point moves the
    # half vector off the normal by ~1e-7 rad, which lowers the lobe by a relative ~alpha * 1e-14)
    assert np.allclose(rgb, expect, rtol=1e-9, atol=0), (rgb, expect)


def test_point_light_mirror_lambert_and_ambient_closed_form():
    ks, rho, I, d, ev, amb = 0.375, np.array([0.25, 0.5, 0.875]), 1.25, 0.6, -0.5, np.array([0.0625, 0.03125, 0.125])
    rgb, P, n, Lview, v = _mirror_case(16.0, ks, rho, I, d, ev, amb=amb)
    dist = np.linalg.norm(Lview - P)
    L = (Lview - P) / dist
    ndl = np.dot(n, L)
    assert abs(ndl - np.dot(n, v)) < 1e-6   # the mirror: n . L = n . v
    expect = 2.0 ** ev * (amb * rho + I / dist ** 2 * (rho * ndl + ks * np.linalg.norm(n) ** 16.0))
    assert np.allclose(rgb, expect, rtol=1e-9, atol=0), (rgb, expect)


def _spot_at(R, Lworld, P, t, cos_o=0.9, cos_i=0.95, away=False):
    # world axis from the light towards the point (or the opposite way)
    Pw = R.T @ (P - t)
    a = Pw - Lworld
    a /= np.linalg.norm(a)
    return (-a if away else a, cos_o, cos_i)


def test_spot_light_full_cone_equals_point_light():
    ks, rho, I, d, ev, amb = 0.5, np.array([0.375, 0.625, 0.125]), 0.875, 0.7, 0.0, np.array([0.0, 0.0, 0.0])
    rgb_spot, P, n, Lview, _ = _mirror_case(9.0, ks, rho, I, d, ev, amb=amb, spot=_spot_at)
    rgb_point, *_ = _mirror_case(9.0, ks, rho, I, d, ev, amb=amb)
    dist = np.linalg.norm(Lview - P)
    expect = I / dist ** 2 * (rho * np.dot(n, (Lview - P) / dist) + ks * np.linalg.norm(n) ** 9.0)
    assert np.allclose(rgb_spot, expect, rtol=1e-9, atol=0)
    assert np.allclose(rgb_point, expect, rtol=1e-9, atol=0)


def test_spot_light_aimed_away_leaves_ambient():
    amb, rho = np.array([0.125, 0.25, 0.375]), np.array([0.5, 0.5, 0.5])
    rgb, *_ = _mirror_case(9.0, 0.5, rho, 0.875, 0.7, 1.0, amb=amb,
                           spot=lambda R, Lw, P, t: _spot_at(R, Lw, P, t, away=True))
    assert np.allclose(rgb, 2.0 * amb * rho, rtol=1e-12, atol=0)
