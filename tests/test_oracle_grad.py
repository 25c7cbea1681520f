"""Pins of the oracle's shading adjoint (gradients of an image loss w.r.t. the randomized material,
light and exposure parameters, Sec. 4.3.1, at fixed visibility).

L = sum over pixels and channels of (rgb_linear - target)^2, so dL/drgb = 2 (rgb - target).
The analytic fp64 adjoint is checked against fp64 central differences (h = 1e-4) of the fp64
shading of the same G-buffer, and against closed forms.
"""

import math

import numpy as np
import pytest

from paper_1906_11633_b300 import scenegen as sg
from tests import scenes

H_FD = 1e-4


def _setup(batch, oracle, seed=0):
    o = oracle.render(batch, gbuffer=True)
    gb = (o["gb_pos"], o["gb_nrm"], o["gb_mat"])
    mat_t, light_t, ev_t = sg.perturb_params(batch, seed)
    tgt = oracle.shade_f64(batch, *gb, material=mat_t, light=light_t, exposure_ev=ev_t)
    return gb, tgt


def _loss(oracle, batch, gb, tgt, m, l, e):
    rgb = oracle.shade_f64(batch, *gb, material=m, light=l, exposure_ev=e)
    fg = gb[2] >= 0
    return ((rgb[fg] - tgt[fg]) ** 2).sum()


def _rel(g, ref):
    scale = max(np.abs(ref).max(), 1e-30)
    return np.abs(g - ref) / np.maximum(np.abs(ref), 1e-3 * scale)


@pytest.mark.parametrize("kind", ["hand", "tiny_dir"])
def test_adjoint_matches_central_differences(oracle, kind):
    if kind == "hand":
        b = sg.hand_batch(21, np.arange(2), res=40)
    else:
        b = sg.tiny_batch(4, n_samples=2, res=40)
        b = b.with_params(material=b.material.copy())
        b.material[:, :2, 3] = 0.4      # add a specular lobe to exercise the directional-light path
        b.material[:, :2, 4] = 12.0
    gb, tgt = _setup(b, oracle)
    m = b.material.astype(np.float64)
    l = b.light.astype(np.float64)
    e = b.exposure_ev.astype(np.float64)
    rgb = oracle.shade_f64(b, *gb, material=m, light=l, exposure_ev=e)
    g = 2.0 * (rgb - tgt)
    g[gb[2] < 0] = 0.0
    dm, dl, de = oracle.shade_backward_f64(b, *gb, g, material=m, light=l, exposure_ev=e)

    rng = np.random.default_rng(0)
    S = b.n_samples
    checks = []
    used = [np.unique(gb[2][(gb[2] >= 0) & (np.repeat(b.cam_sample, b.cam_wh[:, 0] * b.cam_wh[:, 1]) == s)])
            for s in range(S)]
    for s in range(S):
        for mat in rng.choice(used[s], min(4, len(used[s])), replace=False):
            for k in range(4):
                checks.append(("m", (s, mat, k), dm[s, mat, k]))
        for li in range(b.light_meta[s, 0]):
            for k in range(4):
                checks.append(("l", (s, li, k), dl[s, li, k]))
        checks.append(("e", (s,), de[s]))
    fd, an = [], []
    for kind_, idx, a in checks:
        vals = []
        for sgn in (1, -1):
            mm, ll, ee = m.copy(), l.copy(), e.copy()
            arr = {"m": mm, "l": ll, "e": ee}[kind_]
            arr[idx] += sgn * H_FD
            vals.append(_loss(oracle, b, gb, tgt, mm, ll, ee))
        fd.append((vals[0] - vals[1]) / (2 * H_FD))
        an.append(a)
    fd, an = np.array(fd), np.array(an)
    assert np.abs(an).max() > 0
    assert _rel(an, fd).max() < 1e-4, (_rel(an, fd).max(), checks[int(np.argmax(_rel(an, fd)))])


def test_exposure_and_albedo_closed_forms(oracle):
    """dL/dEV = ln2 * sum 2(rgb - t) rgb;  Lambert: dL/drho_c = sum_px 2(rgb - t)_c 2^EV E ndl."""
    th = math.radians(40.0)
    d = (-math.sin(th), 0.0, -math.cos(th))
    b = scenes.single_sample([sg.plane_mesh(50, 50)], [0], [scenes.identity_pose()],
                             [scenes.camera_down((0, 0, 1.5), 20, 18, fovy_deg=60)],
                             lights=[(d, 1.3)], light_type=sg.LIGHT_DIRECTIONAL, albedo=(0.4, 0.5, 0.6), ev=0.7)
    o = oracle.render(b, gbuffer=True)
    gb = (o["gb_pos"], o["gb_nrm"], o["gb_mat"])
    rgb = oracle.shade_f64(b, *gb)
    tgt = np.full_like(rgb, 0.3)
    g = 2.0 * (rgb - tgt)
    dm, dl, de = oracle.shade_backward_f64(b, *gb, g)
    np.testing.assert_allclose(de[0], math.log(2.0) * (g * rgb).sum(), rtol=1e-12)
    scale = 2.0 ** 0.7
    exp = (g * scale * 1.3 * math.cos(th)).sum(0)
    np.testing.assert_allclose(dm[0, 0, :3], exp, rtol=1e-6)   # direction stored as fp32
    # directional intensity: dL/dI = sum 2(rgb-t) . rgb / I
    np.testing.assert_allclose(dl[0, 0, 3], (g * rgb).sum() / np.float32(1.3), rtol=1e-10)


def test_unused_parameters_have_exactly_zero_gradient(oracle):
    b = sg.hand_batch(2, np.arange(1), res=32)
    gb, tgt = _setup(b, oracle)
    rgb = oracle.shade_f64(b, *gb)
    g = 2.0 * (rgb - tgt)
    g[gb[2] < 0] = 0
    dm, dl, de = oracle.shade_backward_f64(b, *gb, g)
    used = np.unique(gb[2][gb[2] >= 0])
    unused = np.setdiff1d(np.arange(32), used)
    assert len(unused) > 0
    assert (dm[0, unused] == 0).all()
    assert (dl[0, b.light_meta[0, 0]:] == 0).all()


@pytest.mark.parametrize("shadow_res", [0, 64])
def test_spot_and_emission_adjoint_matches_central_differences(oracle, shadow_res):
    """The benchmark-like scene: three spot lights (the cone factor depends on the light position)
    and emissive block faces, with and without shadow maps (the shadow factors, carried in the
    G-buffer, stay fixed); light, exposure and emission gradients against fp64 differences."""
    b = sg.benchmark_batch(5, np.arange(2), res=40, grading=False, shadow_res=shadow_res)
    b = b.with_params(emission=b.emission + np.float32(0.05))     # every slot emissive
    o = oracle.render(b, gbuffer=True)
    gb = (o["gb_pos"], o["gb_nrm"], o["gb_mat"])
    m, l = b.material.astype(np.float64), b.light.astype(np.float64)
    e, em = b.exposure_ev.astype(np.float64), b.emission.astype(np.float64)
    mat_t, light_t, ev_t = sg.perturb_params(b, 1)
    tgt = oracle.shade_f64(b, *gb, material=mat_t, light=light_t, exposure_ev=ev_t, emission=em * 0.7)
    fg = gb[2] >= 0

    def loss(mm, ll, ee, emm):
        rgb = oracle.shade_f64(b, *gb, material=mm, light=ll, exposure_ev=ee, emission=emm)
        return ((rgb[fg] - tgt[fg]) ** 2).sum()

    rgb = oracle.shade_f64(b, *gb, material=m, light=l, exposure_ev=e, emission=em)
    g = 2.0 * (rgb - tgt)
    g[~fg] = 0.0
    dm, dl, de, dem = oracle.shade_backward_f64(b, *gb, g, material=m, light=l, exposure_ev=e, emission=em,
                                                return_emission=True)
    # the ramp of some cone crosses pixels of the scene, so the cone term is exercised
    cams = np.repeat(b.cam_sample, b.cam_wh[:, 0] * b.cam_wh[:, 1])
    if shadow_res:
        k = (gb[2][fg] >> 8) & 15
        assert ((k > 0) & (k < 9)).any()                               # partly shadowed pixels
    checks = [("l", (s, li, k), dl[s, li, k]) for s in range(2) for li in range(3) for k in range(4)]
    checks += [("e", (s,), de[s]) for s in range(2)]
    for s in range(2):
        used = np.unique(gb[2][fg & (cams == s)] & 0xff)
        checks += [("em", (s, mat), dem[s, mat]) for mat in used[:6]]
        checks += [("m", (s, mat, k), dm[s, mat, k]) for mat in used[:3] for k in range(3)]
    fd, an = [], []
    for kind_, idx, a in checks:
        vals = []
        for sgn in (1, -1):
            arrs = {"m": m.copy(), "l": l.copy(), "e": e.copy(), "em": em.copy()}
            arrs[kind_][idx] += sgn * H_FD
            vals.append(loss(arrs["m"], arrs["l"], arrs["e"], arrs["em"]))
        fd.append((vals[0] - vals[1]) / (2 * H_FD))
        an.append(a)
    fd, an = np.array(fd), np.array(an)
    assert np.abs(an).max() > 0
    assert _rel(an, fd).max() < 1e-4, (_rel(an, fd).max(), checks[int(np.argmax(_rel(an, fd)))])
    # emission closed form: dL/de = 2^EV sum_px g . rho over the slot's pixels
    s, mat = 0, int(np.unique(gb[2][fg & (cams == 0)] & 0xff)[0])
    px = fg & (cams == s) & ((gb[2] & 0xff) == mat)
    np.testing.assert_allclose(dem[s, mat], 2.0 ** e[s] * (g[px] @ m[s, mat, :3]).sum(), rtol=1e-10)
