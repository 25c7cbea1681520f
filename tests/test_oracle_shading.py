"""Pins of the oracle's shading (randomized material / light / exposure, Sec. 4.3.1) and channel
encodings (Sec. 4.4) against closed forms and library routines."""

import math

import numpy as np
import pytest

from paper_1906_11633_b300 import scenegen as sg
from tests import scenes

PLANE = sg.plane_mesh(50.0, 50.0)


def _plane_down(h=1.5, W=33, H=31, **kw):
    cam = scenes.camera_down((0.0, 0.0, h), W, H, fovy_deg=60)
    return scenes.single_sample([PLANE], [0], [scenes.identity_pose()], [cam], **kw)


@pytest.mark.parametrize("theta_deg", [0.0, 30.0, 60.0, 89.0, 95.0, 150.0])
def test_lambert_directional(oracle, theta_deg):
    """rgb = rho * I * cos(theta) for a directional light at angle theta to the plane normal (0 beyond 90 deg)."""
    th = math.radians(theta_deg)
    d = (-math.sin(th), 0.0, -math.cos(th))        # direction the light travels
    rho, I = (0.8, 0.45, 0.2), 1.7
    b = _plane_down(lights=[(d, I)], light_type=sg.LIGHT_DIRECTIONAL, albedo=rho)
    o = oracle.render(b)
    exp = np.array(rho) * I * max(0.0, math.cos(th))
    np.testing.assert_allclose(o["rgb_linear"], np.tile(exp, (b.total_pixels, 1)), atol=1e-6)
    if theta_deg > 90:
        assert (o["rgb_linear"] == 0).all()


def test_point_light_inverse_square(oracle):
    """A point light right above the pixel seen along the camera axis: rgb = rho * I / d^2."""
    W = H = 65          # odd: the centre pixel's centre is on the optical axis
    for d in (0.3, 0.7, 1.2):
        b = _plane_down(h=2.0, W=W, H=H, lights=[((0.0, 0.0, d), 0.9)], albedo=(0.5, 0.25, 1.0))
        o = oracle.render(b)
        c = (H // 2) * W + W // 2
        np.testing.assert_allclose(o["rgb_linear"][c], np.array([0.5, 0.25, 1.0]) * 0.9 / d ** 2, rtol=1e-6)


def test_blinn_phong_mirror_configuration(oracle):
    """Camera, light and surface point on one normal: n = L = V = H, so spec = k_s exactly and
    rgb = 2^EV (ambient*rho + I/d^2 (rho + k_s))."""
    W = H = 65
    for ks, alpha, ev in ((0.7, 1.0, 0.0), (0.3, 64.0, 1.0), (1.0, 128.0, -0.5)):
        rho, amb, I, d = np.array([0.2, 0.6, 0.9]), np.array([0.05, 0.02, 0.08]), 0.8, 0.6
        b = _plane_down(h=2.0, W=W, H=H, lights=[((0.0, 0.0, d), I)], albedo=rho, specular=ks, shininess=alpha,
                        ev=ev, ambient=amb)
        o = oracle.render(b)
        c = (H // 2) * W + W // 2
        exp = 2.0 ** ev * (amb * rho + I / d ** 2 * (rho + ks))
        np.testing.assert_allclose(o["rgb_linear"][c], exp, rtol=2e-6)


def test_shininess_one_is_a_cosine_lobe(oracle):
    """alpha = 1: spec = k_s * (n . H); every pixel against an fp64 closed form from the plane geometry."""
    W, H, h = 40, 36, 1.2
    lp = np.array([0.3, -0.2, 0.5])
    b = _plane_down(h=h, W=W, H=H, lights=[(lp, 0.6)], albedo=(0.3, 0.3, 0.3), specular=0.9, shininess=1.0)
    o = oracle.render(b)
    fx, fy, cx, cy = b.cam_intr[0, :4].astype(np.float64)
    xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    # view = world - eye (camera looks straight down with R = I); plane point P = h * ray
    P = np.stack([h * (xs - cx) / fx, -h * (ys - cy) / fy, -h * np.ones_like(xs)], -1)
    Lv = (lp - np.array([0, 0, h])) - P
    d2 = (Lv ** 2).sum(-1)
    L = Lv / np.sqrt(d2)[..., None]
    V = -P / np.linalg.norm(P, axis=-1, keepdims=True)
    Hh = (L + V) / np.linalg.norm(L + V, axis=-1, keepdims=True)
    ndl = np.clip(L[..., 2], 0, None)
    ndh = np.clip(Hh[..., 2], 0, None)
    rgb = 0.6 / d2 * (0.3 * ndl + np.where(ndl > 0, 0.9 * ndh, 0.0))
    np.testing.assert_allclose(o["rgb_linear"].reshape(H, W, 3), np.repeat(rgb[..., None], 3, -1), rtol=2e-5)


def test_exposure_is_an_exact_power_of_two(oracle):
    base = sg.hand_batch(11, np.arange(1), res=48)
    o0 = oracle.render(base)
    for ev in (-1.0, 1.0, 2.0):
        b = base.with_params(exposure_ev=base.exposure_ev * 0 + np.float32(ev))
        b0 = base.with_params(exposure_ev=base.exposure_ev * 0)
        r0 = oracle.render(b0)["rgb_linear"]
        r = oracle.render(b)["rgb_linear"]
        fg = oracle.render(b, gbuffer=True)["gb_mat"] >= 0
        np.testing.assert_array_equal(r[fg], np.float32(2.0 ** ev) * r0[fg])
    assert o0["rgb_linear"].shape[0] == base.total_pixels


def test_normals_are_unit_and_planes_are_exact(oracle):
    b = sg.hand_batch(5, np.arange(2), res=64)
    o = oracle.render(b, gbuffer=True)
    fg = o["gb_mat"] >= 0
    n = o["gb_nrm"][fg].astype(np.float64)
    assert np.abs(np.linalg.norm(n, axis=1) - 1.0).max() < 1e-6
    # table pixels: the normal is R_view (0, 0, 1)
    seg = o["seg"]
    for c in range(b.n_cams):
        sl = slice(b.img_offset[c], b.img_offset[c] + 64 * 64)
        table = seg[sl] == 1
        expn = b.cam_view[c, :, 2].astype(np.float64)
        assert np.abs(o["gb_nrm"][sl][table] - expn).max() < 2e-7


def test_binary16_matches_numpy():
    from oracle import oracle as orc
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-1, 1, 4000), rng.standard_normal(2000) * 1e-5, rng.standard_normal(1000) * 1e4,
                        [0.0, -0.0, 1.0, -1.0, 65504.0, 65520.0, 1e9, 5.96e-8, 2.98e-8, 2.99e-8, 6.1e-5, np.inf, -np.inf]])
    x = x.astype(np.float32)
    got = orc.f32_to_f16_bits(x)
    with np.errstate(over="ignore"):                       # 65520, 1e9 and the infinities go to inf
        want = x.astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(got, want)


def test_quantisation_rounds_half_up(oracle):
    vals = np.array([-0.5, 0.0, 0.5 / 255, 0.49 / 255, 0.5, 1.0, 7.0], np.float32)
    rgb8 = []
    for v in vals:
        b = _plane_down(W=3, H=3, background=(v, v, v))
        b = b.with_params(inst_offset=np.array([0, 0], np.int32), inst_mesh=b.inst_mesh[:0], inst_pose=b.inst_pose[:0],
                          inst_seg=b.inst_seg[:0], inst_mat_base=b.inst_mat_base[:0])
        rgb8.append(oracle.render(b)["rgb"][0, 0])
    np.testing.assert_array_equal(rgb8, [0, 0, 1, 0, 128, 255, 255])
