"""Pins of the oracle's colour-grading epilogue (the post-processing randomizer, Sec. 4.3.1):
each operation checked on its own against what it must do to the ungraded linear colour,
computed here from the oracle's rgb_linear channel (which stays ungraded):

  identity parameters change nothing; a hue rotation by 2 pi / 3 about the grey axis permutes
  the channels (r, g, b) -> (b, r, g); saturation 0 leaves the Rec. 709 luma in every channel;
  contrast 0 leaves mid-grey; brightness adds; temperature and tint scale red / blue and green;
  grain adds the same uniform [-a/2, a/2) offset to all three channels, deterministic, different
  per camera and independent of the batch a sample is rendered in.
"""

import math

import numpy as np
import pytest

from paper_1906_11633_b300 import scenegen as sg


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as o
    o.build()
    return o


@pytest.fixture(scope="module")
def batch():
    return sg.hand_batch(4, np.arange(2), res=48)


def _q(v):
    return np.floor(np.clip(v, 0.0, 1.0) * 255.0 + 0.5).astype(np.int32)


def _graded(orc, batch, **kw):
    g = sg.identity_grading(batch.n_samples)
    names = ["hue", "saturation", "contrast", "brightness", "temperature", "tint", "grain", "seed"]
    for k, v in kw.items():
        g[:, names.index(k)] = v
    o = orc.render(batch.with_params(grading=g))
    return o["rgb"].reshape(-1, 3).astype(np.int32), o["rgb_linear"].reshape(-1, 3).astype(np.float64)


def test_identity_changes_nothing(orc, batch):
    plain = orc.render(batch)
    got = orc.render(batch.with_params(grading=sg.identity_grading(batch.n_samples)))
    for k in plain:
        if k == "rgb_final":  # (the identity's fp32 steps, e.g. Y + 1 * (c - Y), may move the last bit)
            np.testing.assert_allclose(got[k], plain[k], rtol=0, atol=1e-6, err_msg=k)
        else:
            np.testing.assert_array_equal(got[k], plain[k], err_msg=k)


def test_hue_third_turn_permutes_channels(orc, batch):
    rgb, lin = _graded(orc, batch, hue=2.0 * math.pi / 3.0)
    want = _q(lin[:, [2, 0, 1]])
    assert np.abs(rgb - want).max() <= 1
    rgb_full, _ = _graded(orc, batch, hue=2.0 * math.pi)
    assert np.abs(rgb_full - _q(lin)).max() <= 1


def test_saturation_zero_is_rec709_luma(orc, batch):
    rgb, lin = _graded(orc, batch, saturation=0.0)
    y = lin @ np.array([0.2126, 0.7152, 0.0722])
    assert np.abs(rgb - _q(y)[:, None]).max() <= 1
    assert (rgb.max(axis=1) - rgb.min(axis=1)).max() <= 1


def test_contrast_zero_is_mid_grey_and_brightness_adds(orc, batch):
    rgb, _ = _graded(orc, batch, contrast=0.0)
    assert (rgb == 128).all()
    rgb, lin = _graded(orc, batch, brightness=0.07)
    assert np.abs(rgb - _q(lin + 0.07)).max() <= 1


def test_temperature_and_tint_are_channel_gains(orc, batch):
    rgb, lin = _graded(orc, batch, temperature=0.2, tint=-0.15)
    want = _q(lin * np.array([1.2, 0.85, 0.8]))
    assert np.abs(rgb - want).max() <= 1


def test_grain_is_one_uniform_offset_per_pixel(orc, batch):
    a = 0.5
    # contrast 0 makes every pixel mid-grey before the grain, so the grain is all that is left
    rgb, _ = _graded(orc, batch, contrast=0.0, grain=a, seed=12345.0)
    noise = (rgb / 255.0 - 0.5) / a                      # n - 1/2 up to the quantisation (+-0.5/255/a)
    tol = 1.0 / 255.0 / a
    assert (np.ptp(noise, axis=1) <= 2 * tol).all()     # the same offset on r, g and b
    n = noise.mean(axis=1)
    assert n.min() >= -0.5 - tol and n.max() < 0.5 + tol
    assert abs(n.mean()) < 0.03 and abs(n.std() - 1.0 / math.sqrt(12.0)) < 0.03
    hist, _ = np.histogram(n, bins=10, range=(-0.5, 0.5))
    assert hist.min() > 0.5 * hist.mean()
    again, _ = _graded(orc, batch, contrast=0.0, grain=a, seed=12345.0)
    np.testing.assert_array_equal(again, rgb)
    other, _ = _graded(orc, batch, contrast=0.0, grain=a, seed=54321.0)
    assert (other != rgb).any()


def test_grain_differs_per_camera_and_not_per_batch(orc):
    b = sg.hand_batch(6, np.arange(3), res=32, grading=True)
    g = b.grading.copy()
    g[:, 6] = 0.3
    b = b.with_params(grading=g)
    full = orc.render(b)["rgb"].reshape(-1, 32 * 32, 3)
    assert (full[0] != full[1]).any()                   # cameras of one sample: different grain
    alone = orc.render(sg.select_samples(b, [1]))["rgb"].reshape(-1, 32 * 32, 3)
    np.testing.assert_array_equal(alone, full[3:6])
