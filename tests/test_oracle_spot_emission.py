"""Pins of the oracle's spot lights (the LightRandomizer's spotlight angles, Sec. 4.3.1) and of
material emission (a MuJoCo material's emission, Sec. 4.2), against closed forms from the scene
geometry and against special cases that reduce to already pinned shading:

  a cone wider than every direction is the point light, bit for bit; under a spot aimed straight
  down at a plane every pixel follows rho I cos(theta) / d^2 times the smoothstep of cos(theta)
  across the cone's edge; a spot aimed away, a cone with cos_inner <= cos_outer, an unknown light
  type and a spot without its cone table light nothing; emission alone gives 2^EV e rho; emission
  e on every material equals ambient + e; emission on one slot changes only that slot's pixels.
"""

import math

import numpy as np

from paper_1906_11633_b300 import scenegen as sg
from tests import scenes

PLANE = sg.plane_mesh(50.0, 50.0)


def _plane_down(h=1.5, W=48, H=44, fovy=70.0, **kw):
    cam = scenes.camera_down((0.0, 0.0, h), W, H, fovy_deg=fovy)
    return scenes.single_sample([PLANE], [0], [scenes.identity_pose()], [cam], **kw)


def _plane_points(b, h):
    """fp64 world points of the pixel centres on the z = 0 plane under the straight-down camera."""
    W, H = b.cam_wh[0]
    fx, fy, cx, cy = b.cam_intr[0, :4].astype(np.float64)
    xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    return np.stack([h * (xs - cx) / fx, -h * (ys - cy) / fy, np.zeros_like(xs)], -1)


def _smoothstep(x, cos_o, cos_i):
    t = np.clip((x - cos_o) / (cos_i - cos_o), 0.0, 1.0)
    return t * t * (3.0 - 2.0 * t)


def test_cone_wider_than_every_direction_is_the_point_light(oracle):
    b = sg.hand_batch(3, np.arange(2), res=48)
    n = int(b.light_meta[:, 0].max())
    spot = np.zeros((b.n_samples, 4, 5), np.float32)
    spot[:, :, :3] = (0.0, 0.0, -1.0)
    spot[:, :, 3], spot[:, :, 4] = -2.0, -1.5           # t = (x + 2) / 0.5 >= 2 for every x >= -1
    meta = b.light_meta.copy()
    meta[:, 1] = sg.LIGHT_SPOT
    s = b.with_params(light_meta=meta, light_spot=spot)
    p, q = oracle.render(b), oracle.render(s)
    assert n > 0 and (p["rgb_linear"] > 0).any()
    for k in p:
        np.testing.assert_array_equal(q[k], p[k], err_msg=k)


def test_spot_aimed_down_follows_the_cone_profile(oracle):
    h_cam, h_l, I, rho = 2.0, 0.8, 0.7, np.array([0.9, 0.5, 0.3])
    for outer, inner in ((30.0, 20.0), (40.0, 36.0)):
        cos_o, cos_i = math.cos(math.radians(outer)), math.cos(math.radians(inner))
        b = _plane_down(h=h_cam, lights=[((0.0, 0.0, h_l), I)], light_type=sg.LIGHT_SPOT, albedo=rho,
                        spots=[((0.0, 0.0, -1.0), cos_o, cos_i)])
        rgb = oracle.render(b)["rgb_linear"].reshape(44, 48, 3).astype(np.float64)
        P = _plane_points(b, h_cam)
        d2 = P[..., 0] ** 2 + P[..., 1] ** 2 + h_l ** 2
        cos_t = h_l / np.sqrt(d2)             # the angle off the spot axis equals the angle of incidence
        exp = (I * cos_t / d2 * _smoothstep(cos_t, np.float32(cos_o), np.float32(cos_i)))[..., None] * rho
        inside, outside = cos_t > cos_i + 1e-4, cos_t < cos_o - 1e-4
        ramp = ~inside & ~outside
        assert inside.sum() > 20 and outside.sum() > 20 and ramp.sum() > 20
        np.testing.assert_allclose(rgb[inside], exp[inside], rtol=2e-6)
        assert (rgb[outside] == 0).all()
        # the ramp: fp32 rounding of the cosine is amplified by 1 / (cos_i - cos_o)
        tol = 3e-6 * I / h_l ** 2 * 1.5 / (cos_i - cos_o)
        assert np.abs(rgb[ramp] - exp[ramp]).max() < tol


def test_spots_that_light_nothing(oracle):
    base = dict(h=1.5, lights=[((0.1, 0.0, 0.6), 0.8)], albedo=(0.5, 0.5, 0.5), ambient=(0.01, 0.02, 0.03))
    dark = oracle.render(_plane_down(**{**base, "lights": []}))["rgb_linear"]
    assert (dark > 0).all()
    cases = [
        dict(light_type=sg.LIGHT_SPOT, spots=[((0.0, 0.0, 1.0), 0.5, 0.9)]),     # aimed away from the plane
        dict(light_type=sg.LIGHT_SPOT, spots=[((0.0, 0.0, -1.0), 0.8, 0.8)]),    # cos_inner == cos_outer
        dict(light_type=sg.LIGHT_SPOT, spots=[((0.0, 0.0, -1.0), 0.9, 0.5)]),    # cos_inner < cos_outer
        dict(light_type=sg.LIGHT_SPOT),                                          # no cone table
        dict(light_type=5),                                                      # unknown type
    ]
    for kw in cases:
        got = oracle.render(_plane_down(**base, **kw))["rgb_linear"]
        np.testing.assert_array_equal(got, dark, err_msg=str(kw))


def test_emission_alone_is_two_to_ev_times_emission_times_albedo(oracle):
    rho, e, ev = np.array([0.8, 0.4, 0.2]), 0.35, 0.5
    b = _plane_down(albedo=rho, ev=ev, emission=e)
    rgb = oracle.render(b)["rgb_linear"]
    np.testing.assert_allclose(rgb, np.tile(2.0 ** ev * e * rho, (b.total_pixels, 1)), rtol=1e-6)


def test_emission_adds_like_ambient(oracle):
    b = sg.hand_batch(9, np.arange(2), res=40)
    e = 0.125                                  # exact in fp32, and so are ambient + e below
    with_e = oracle.render(b.with_params(emission=np.full((2, 32), e, np.float32)))["rgb_linear"]
    amb = oracle.render(b.with_params(ambient=b.ambient + np.float32(e)))["rgb_linear"]
    np.testing.assert_allclose(with_e, amb, rtol=1e-6, atol=1e-7)


def test_emission_on_one_slot_changes_only_its_pixels(oracle):
    b = sg.hand_batch(9, np.arange(1), res=48)
    o = oracle.render(b, gbuffer=True)
    em = np.zeros((1, 32), np.float32)
    em[0, 1] = 0.5                             # the block's first face
    got = oracle.render(b.with_params(emission=em))["rgb_linear"]
    slot = o["gb_mat"] == 1
    assert slot.sum() > 0
    np.testing.assert_array_equal(got[~slot], o["rgb_linear"][~slot])
    assert (got[slot] > o["rgb_linear"][slot]).all()
