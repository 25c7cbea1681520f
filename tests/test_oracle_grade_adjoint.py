"""Pins of the oracle's colour-grading adjoint (a loss on the graded colour, the post-processing
randomizer of Sec. 4.3.1).

- The fp64 grading equals the fp32 forward's grading (rgb8 within 1 LSB of its quantisation).
- Its adjoint matches fp64 central differences (h = 1e-4) for every grading parameter (hue,
  saturation, contrast, brightness, temperature, tint, grain amplitude) and, through the grading,
  for albedo, light and exposure.
- Closed forms: brightness collects the sum of dL/dc' over every pixel (background included); at
  the identity grading the colour's gradient passes unchanged and the hue's equals the sum of
  dL/dc' . (axis x c).
"""

import numpy as np
import pytest

from paper_1906_11633_b300 import scenegen as sg

H_FD = 1e-4
NAMES = ["hue", "saturation", "contrast", "brightness", "temperature", "tint", "grain"]


def _rel(g, ref, scale):
    return abs(g - ref) / max(abs(ref), 1e-3 * scale)


def _setup(oracle, seed=0):
    b = sg.benchmark_batch(seed, np.arange(2), res=40)
    o = oracle.render(b, gbuffer=True)
    gb = (o["gb_pos"], o["gb_nrm"], o["gb_mat"])
    rng = np.random.default_rng(seed)
    target = oracle.graded_shade_f64(b, *gb) + rng.normal(0.0, 0.05, (b.total_pixels, 3))
    return b, o, gb, target


def _loss(oracle, b, gb, target, grading=None, **params):
    c = oracle.graded_shade_f64(b, *gb, grading=grading, **params)
    return ((c - target) ** 2).sum()


def test_fp64_grading_equals_the_forward(oracle):
    b, o, gb, _ = _setup(oracle, 1)
    c = oracle.graded_shade_f64(b, *gb)
    q = np.floor(np.clip(c, 0.0, 1.0) * 255.0 + 0.5).astype(int)
    assert np.abs(q - o["rgb"].astype(int)).max() <= 1


def test_grading_adjoint_matches_central_differences(oracle):
    b, o, gb, target = _setup(oracle, 2)
    g0 = b.grading.astype(np.float64)
    c = oracle.graded_shade_f64(b, *gb, grading=g0)
    d = 2.0 * (c - target)
    dm, dl, de, dg = oracle.graded_backward_f64(b, *gb, d, grading=g0)
    scale = np.abs(dg[:, :7]).max()
    for s in range(b.n_samples):
        for j, name in enumerate(NAMES):
            gp, gm = g0.copy(), g0.copy()
            gp[s, j] += H_FD
            gm[s, j] -= H_FD
            fd = (_loss(oracle, b, gb, target, grading=gp) - _loss(oracle, b, gb, target, grading=gm)) / (2 * H_FD)
            assert _rel(dg[s, j], fd, scale) < 1e-4, (s, name, dg[s, j], fd)
    assert np.all(dg[:, 7] == 0.0)
    # through the grading: exposure, an albedo channel and a light coordinate
    m0, l0, e0 = (b.material.astype(np.float64), b.light.astype(np.float64), b.exposure_ev.astype(np.float64))
    checks = [("ev", (0,), de[0]), ("albedo", (1, 2, 1), dm[1, 2, 1]), ("light", (0, 1, 2), dl[0, 1, 2])]
    for kind, idx, got in checks:
        args = []
        for sgn in (1.0, -1.0):
            m, l, e = m0.copy(), l0.copy(), e0.copy()
            {"ev": e, "albedo": m, "light": l}[kind][idx] += sgn * H_FD
            args.append(_loss(oracle, b, gb, target, grading=g0, material=m, light=l, exposure_ev=e))
        fd = (args[0] - args[1]) / (2 * H_FD)
        assert abs(got - fd) <= 1e-4 * max(abs(fd), 1e-3), (kind, got, fd)


def test_grading_adjoint_closed_forms(oracle):
    b, o, gb, _ = _setup(oracle, 3)
    rng = np.random.default_rng(3)
    d = rng.normal(size=(b.total_pixels, 3))
    # brightness: every pixel's three channels
    _, _, _, dg = oracle.graded_backward_f64(b, *gb, d)
    per_img = (b.cam_wh[:, 0] * b.cam_wh[:, 1]).astype(np.int64)
    owner = np.repeat(b.cam_sample, per_img)
    for s in range(b.n_samples):
        assert np.isclose(dg[s, 3], d[owner == s].sum(), rtol=1e-12, atol=1e-9)
    # identity grading (no grain): d rgb_linear = dL/dc', and d hue = sum dL/dc' . (axis x c)
    ident = sg.identity_grading(b.n_samples).astype(np.float64)
    ident[:, 6] = 0.0
    lin = oracle.shade_f64(b, *gb)
    dm_i, dl_i, de_i, dg_i = oracle.graded_backward_f64(b, *gb, d, grading=ident)
    dm_l, dl_l, de_l = oracle.shade_backward_f64(b, *gb, d)
    assert np.allclose(dm_i, dm_l, rtol=1e-12, atol=1e-12) and np.allclose(de_i, de_l, rtol=1e-12, atol=1e-12)
    k = 1.0 / np.sqrt(3.0)
    axc = k * np.stack([lin[:, 2] - lin[:, 1], lin[:, 0] - lin[:, 2], lin[:, 1] - lin[:, 0]], axis=1)
    for s in range(b.n_samples):
        assert np.isclose(dg_i[s, 0], (d * axc)[owner == s].sum(), rtol=1e-10, atol=1e-9)
