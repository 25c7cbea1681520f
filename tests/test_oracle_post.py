"""Pins of the oracle's step 17 (ambient occlusion and bloom, the post-processing randomizer of
Sec. 4.3.1) on synthetic images and on rendered batches.

Bloom (b = max(c - 1, 0), a normalised Gaussian of radius sigma, rows then columns, indices
clamped): nothing at or below 1 blooms; an impulse spreads into a symmetric rank-1 kernel whose
neighbouring values fall by exp(-(2i + 1) / (2 sigma^2)), which sums to beta h and ends at
R = min(ceil(3 sigma), 16); a uniformly bright image gains exactly beta h everywhere.
Ambient occlusion (eight fixed offsets, o = max(0, n.v / L - 0.1) / (1 + L^2 / 0.05^2), c *= 1 - a O):
intensity 0 and a plane facing the camera change nothing; a convex sphere occludes nothing; a depth
step seen at a tiny pixel pitch darkens the far side by 1 - a * 0.45 * m / 8, m the offsets that
reach across the step, and leaves the near side alone.
"""

import numpy as np
import pytest

from paper_1906_11633_b300 import scenegen as sg

# the eight sample offsets of step 17 (its definition)
OFFSETS = [(2, 1), (-1, 3), (-4, -1), (1, -4), (5, 2), (-2, 5), (-5, -3), (3, -6)]
ORTHO = [1.0, 1.0, 0.0, 0.0, 0.01, 1.0]


def f16(v):
    return np.asarray(v, np.float32).astype(np.float16).view(np.uint16)


def blank(W, H, value=0.5, depth=0.0):
    col = np.full((W * H, 3), value, np.float32)
    d = np.full(W * H, depth, np.float32)
    n = np.zeros((W * H, 3), np.uint16)
    return col, d, n


@pytest.mark.parametrize("beta,sigma", [(0.7, 1.0), (1.0, 2.5), (0.3, 7.0)])
def test_bloom_of_an_impulse(oracle, beta, sigma):
    W = H = 41
    col, d, n = blank(W, H, 0.0)     # (a dark background keeps the bloom's own float32 precision)
    h = 3.0
    x0 = y0 = 20
    col[y0 * W + x0, 0] = 1.0 + h
    out = oracle.post_image(W, H, ORTHO, [0.0, beta, sigma, 0.0], col, d, n)
    delta = (out[:, 0] - col[:, 0]).astype(np.float64).reshape(H, W)
    assert np.array_equal(out[:, 1:], col[:, 1:])                 # other channels: nothing above 1
    R = min(int(np.ceil(3 * sigma)), 16)
    nz = np.argwhere(delta != 0)
    assert nz[:, 0].min() == y0 - R and nz[:, 0].max() == y0 + R  # support ends at R
    assert nz[:, 1].min() == x0 - R and nz[:, 1].max() == x0 + R
    assert abs(delta.sum() - beta * h) < 1e-5 * beta * h           # mass: the weights are normalised
    assert np.allclose(delta, delta[::-1, :], rtol=1e-5, atol=1e-9)  # symmetric
    assert np.allclose(delta, delta[:, ::-1], rtol=1e-5, atol=1e-9)
    row, colm = delta[y0, :], delta[:, x0]
    assert np.allclose(np.outer(colm, row) / delta[y0, x0], delta, rtol=1e-4, atol=1e-9)  # rank 1
    for i in range(0, R):                                         # Gaussian fall-off along a row
        assert np.isclose(row[x0 + i + 1] / row[x0 + i], np.exp(-(2 * i + 1) / (2 * sigma ** 2)), rtol=1e-4)


def test_bloom_threshold_and_uniform_bright_image(oracle):
    W, H = 23, 17
    col, d, n = blank(W, H)
    rng = np.random.default_rng(0)
    col[:] = rng.uniform(0.0, 1.0, col.shape).astype(np.float32)
    assert np.array_equal(oracle.post_image(W, H, ORTHO, [0, 2.0, 3.0, 0], col, d, n), col)
    h, beta = 0.75, 0.4
    col[:] = 1.0 + h
    out = oracle.post_image(W, H, ORTHO, [0, beta, 4.0, 0], col, d, n)  # clamped borders: the same everywhere
    assert np.allclose(out, 1.0 + h + beta * h, rtol=1e-6)
    assert np.array_equal(oracle.post_image(W, H, ORTHO, [0, 0.0, 4.0, 0], col, d, n), col)   # beta 0
    assert np.array_equal(oracle.post_image(W, H, ORTHO, [0, 1.0, 0.0, 0], col, d, n), col)   # sigma 0


def test_ao_of_a_plane_facing_the_camera_and_of_intensity_zero(oracle):
    W = H = 24
    col, d, n = blank(W, H, 0.6, depth=1.0)
    n[:] = f16([0.0, 0.0, 1.0])
    for intr in (ORTHO, [30.0, 30.0, 12.0, 12.0, 0.01, 0.0]):
        assert np.array_equal(oracle.post_image(W, H, intr, [1.5, 0, 0, 0], col, d, n), col)
    rng = np.random.default_rng(1)
    d[:] = rng.uniform(0.5, 2.0, W * H).astype(np.float32)
    n[:] = f16(rng.normal(size=(W * H, 3)))
    assert np.array_equal(oracle.post_image(W, H, ORTHO, [0.0, 0, 0, 0], col, d, n), col)


def test_ao_of_a_convex_sphere_is_none(oracle):
    """Points Q on a sphere seen from P on it satisfy n_P . (Q - P) = r (n_Q . n_P - 1) <= 0."""
    W = H = 64
    intr = [40.0, 40.0, 32.0, 32.0, 0.01, 1.0]          # orthographic, 40 px per metre
    x = (np.arange(W) + 0.5 - 32.0) / 40.0
    X, Y = np.meshgrid(x, -x)
    r = 0.6
    inside = X ** 2 + Y ** 2 < r ** 2
    Z = np.where(inside, np.sqrt(np.maximum(r ** 2 - X ** 2 - Y ** 2, 0.0)), 0.0)   # front cap, centre at z = -2
    col, d, n = blank(W, H, 0.4)
    d[:] = np.where(inside, 2.0 - Z, 0.0).reshape(-1)
    n[:] = np.where(inside[..., None], f16(np.stack([X, Y, Z], -1) / r), 0).reshape(-1, 3)
    out = oracle.post_image(W, H, intr, [1.5, 0, 0, 0], col, d, n)
    assert np.array_equal(out, col)


def test_ao_of_a_depth_step(oracle):
    """Orthographic at 1e4 px per metre: the far plane (depth 1.05) left of column 20, the near one
    (depth 1.00) from it on, both facing the camera.  A far pixel's sample across the step sees
    v = (tiny, tiny, 0.05): n.v / L = 1 - O(1e-4), o = 0.9 / (1 + 1) = 0.45."""
    W, H, step, a = 40, 30, 20, 0.8
    intr = [1e4, 1e4, 0.0, 0.0, 0.01, 1.0]
    col, d, n = blank(W, H, 0.5)
    xs = np.tile(np.arange(W), H)
    d[:] = np.where(xs < step, 1.05, 1.0).astype(np.float32)
    n[:] = f16([0.0, 0.0, 1.0])
    out = oracle.post_image(W, H, intr, [a, 0, 0, 0], col, d, n).reshape(H, W, 3)
    for y in range(H):
        for x in range(W):
            if x >= step:
                assert np.array_equal(out[y, x], col.reshape(H, W, 3)[y, x])      # near side: untouched
                continue
            m = sum(1 for dx, dy in OFFSETS
                    if 0 <= x + dx < W and 0 <= y + dy < H and x + dx >= step)
            expect = 0.5 * (1.0 - a * 0.45 * m / 8.0)
            assert np.allclose(out[y, x], expect, rtol=1e-3), (x, y, m, out[y, x], expect)
    assert (out[:, step - 1, 0] < 0.5).all() and (out[:, :step - 7, 0] == 0.5).all()


def test_rendered_post_batch_uses_the_image_channels(oracle):
    """In a render, step 17 runs on the image's own linear colour, depth and normal channels and
    step 13 grades its result: post_image over those channels, graded, gives rgb_final."""
    b = sg.benchmark_batch(3, np.arange(2), res=40, post=True)
    o = oracle.render(b)
    none = oracle.render(b.with_params(post=None))
    assert np.array_equal(o["rgb_linear"], none["rgb_linear"]) and np.array_equal(o["depth"], none["depth"])
    ident = b.with_params(grading=sg.identity_grading(b.n_samples) * np.array([1, 1, 1, 1, 1, 1, 0, 1], np.float32))
    oi = oracle.render(ident)
    for c in range(b.n_cams):
        W, H = b.cam_wh[c]
        s = b.cam_sample[c]
        sl = slice(int(b.img_offset[c]), int(b.img_offset[c]) + W * H)
        post = oracle.post_image(W, H, b.cam_intr[c], b.post[s], oi["rgb_linear"][sl], oi["depth"][sl],
                                 oi["normal"][sl])
        assert np.allclose(oi["rgb_final"][sl], post, rtol=1e-6, atol=1e-6)
    assert np.abs(o["rgb"].astype(int) - none["rgb"].astype(int)).max() > 0


def test_zero_post_parameters_change_nothing(oracle):
    b = sg.benchmark_batch(4, np.arange(2), res=40, post=True)
    z = oracle.render(b.with_params(post=np.zeros_like(b.post)))
    none = oracle.render(b.with_params(post=None))
    for k in ("rgb", "rgb_final", "depth", "normal", "seg", "rgb_linear"):
        assert np.array_equal(z[k], none[k]), k
