"""Pins of the oracle's coverage, fill rule, depth and visibility against closed forms.

Readings pinned here (the paper names the channels, Sec. 4.4, but no raster rule):
8 fractional bits, pixel centres at (x+1/2, y+1/2), top-left fill rule,
(depth, key) visibility with key = 2*prim + sub.
"""

import math

import numpy as np
import pytest

from paper_1906_11633_b300 import scenegen as sg
from tests import scenes

FIX = 256


def quad_tris(x0, y0, x1, y1, diag=0):
    """Two screen triangles (fixed point) covering the axis-aligned box, front-facing."""
    a, b, c, d = (x0, y0), (x0, y1), (x1, y1), (x1, y0)
    tris = [(a, b, c), (a, c, d)] if diag == 0 else [(a, b, d), (b, c, d)]
    X = np.array([[v[0] for v in t] for t in tris], np.int64)
    Y = np.array([[v[1] for v in t] for t in tris], np.int64)
    return X, Y


def expected_box(W, H, x0, y0, x1, y1):
    """Pixels whose centres lie in [x0, x1) x [y0, y1) (fixed-point bounds)."""
    cx = FIX * np.arange(W) + FIX // 2
    cy = FIX * np.arange(H) + FIX // 2
    mx = (cx >= x0) & (cx < x1)
    my = (cy >= y0) & (cy < y1)
    return my[:, None] & mx[None, :]


@pytest.mark.parametrize("diag", [0, 1])
def test_quads_on_pixel_centre_lines(oracle, diag):
    rng = np.random.default_rng(1)
    W = H = 24
    for _ in range(40):
        px0, px1 = sorted(rng.choice(W, 2, replace=False))
        py0, py1 = sorted(rng.choice(H, 2, replace=False))
        # corners at (x + 1/2) px: the edges pass exactly through pixel centres
        x0, x1, y0, y1 = (FIX * v + FIX // 2 for v in (px0, px1, py0, py1))
        X, Y = quad_tris(x0, y0, x1, y1, diag)
        key, depth, count = oracle.raster_fixed(W, H, X, Y, np.ones((2, 3)))
        exp = expected_box(W, H, x0, y0, x1, y1)
        assert exp.sum() == (px1 - px0) * (py1 - py0)
        np.testing.assert_array_equal(count, exp.astype(np.int32))
        np.testing.assert_array_equal(key >= 0, exp)


@pytest.mark.parametrize("diag", [0, 1])
def test_quads_with_integer_corners(oracle, diag):
    rng = np.random.default_rng(2)
    W = H = 24
    for _ in range(40):
        px0, px1 = sorted(rng.choice(W + 1, 2, replace=False))
        py0, py1 = sorted(rng.choice(H + 1, 2, replace=False))
        X, Y = quad_tris(FIX * px0, FIX * py0, FIX * px1, FIX * py1, diag)
        _, _, count = oracle.raster_fixed(W, H, X, Y, np.ones((2, 3)))
        assert count.sum() == (px1 - px0) * (py1 - py0)
        assert count.max() <= 1


def _orient(X, Y):
    """Swap vertices 1 and 2 where needed so every triangle has positive area."""
    A = (X[:, 2] - X[:, 0]) * (Y[:, 1] - Y[:, 0]) - (Y[:, 2] - Y[:, 0]) * (X[:, 1] - X[:, 0])
    neg = A < 0
    X[neg, 1], X[neg, 2] = X[neg, 2].copy(), X[neg, 1].copy()
    Y[neg, 1], Y[neg, 2] = Y[neg, 2].copy(), Y[neg, 1].copy()
    return X, Y


def test_jittered_grid_is_watertight(oracle):
    """A jittered triangle grid tiling an axis-aligned box covers each pixel centre of the box exactly once."""
    rng = np.random.default_rng(3)
    W = H = 40
    for trial in range(10):
        x0, y0 = rng.integers(0, 6 * FIX, 2)
        x1, y1 = rng.integers(30 * FIX, 40 * FIX, 2)
        n = 7
        gx = np.linspace(x0, x1, n + 1)
        gy = np.linspace(y0, y1, n + 1)
        PX, PY = np.meshgrid(gx, gy)
        # +-0.2 cell keeps every cell convex, so both diagonals give front-facing triangles
        jit = rng.uniform(-0.2, 0.2, (2, n + 1, n + 1)) * (gx[1] - gx[0])
        PX = np.rint(PX + jit[0]).astype(np.int64)
        PY = np.rint(PY + jit[1]).astype(np.int64)
        PX[:, 0], PX[:, -1] = x0, x1
        PY[0, :], PY[-1, :] = y0, y1
        tris = []
        for i in range(n):
            for j in range(n):
                a, b, c, d = (i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)
                tris += [(a, b, c), (a, c, d)] if rng.random() < 0.5 else [(a, b, d), (b, c, d)]
        X = np.array([[PX[v] for v in t] for t in tris], np.int64)
        Y = np.array([[PY[v] for v in t] for t in tris], np.int64)
        A = (X[:, 2] - X[:, 0]) * (Y[:, 1] - Y[:, 0]) - (Y[:, 2] - Y[:, 0]) * (X[:, 1] - X[:, 0])
        assert (A > 0).all()
        _, _, count = oracle.raster_fixed(W, H, X, Y, np.ones((len(X), 3)))
        exp = expected_box(W, H, x0, y0, x1, y1)
        np.testing.assert_array_equal(count, exp.astype(np.int32), err_msg=f"trial {trial}")


def test_fan_is_watertight(oracle):
    """A fan around an interior point over a polygon boundary covers every inside centre once."""
    rng = np.random.default_rng(4)
    W = H = 32
    for _ in range(10):
        c = np.array([16 * FIX + rng.integers(-FIX, FIX), 16 * FIX + rng.integers(-FIX, FIX)])
        ang = np.sort(rng.uniform(0, 2 * np.pi, 24))
        rad = rng.uniform(8, 14, 24) * FIX
        P = np.stack([c[0] + rad * np.cos(ang), c[1] + rad * np.sin(ang)], 1).astype(np.int64)
        X = np.array([[c[0], P[k, 0], P[(k + 1) % 24, 0]] for k in range(24)], np.int64)
        Y = np.array([[c[1], P[k, 1], P[(k + 1) % 24, 1]] for k in range(24)], np.int64)
        X, Y = _orient(X, Y)
        _, _, count = oracle.raster_fixed(W, H, X, Y, np.ones((24, 3)))
        assert count.max() == 1
        # every centre strictly inside the (star-shaped) polygon is covered
        cx = FIX * np.arange(W) + FIX // 2
        gxx, gyy = np.meshgrid(cx, cx)
        inside = np.ones((H, W), bool)
        for k in range(24):
            ax, ay = X[k, 1], Y[k, 1]
            bx, by = X[k, 2], Y[k, 2]
            e = (gxx - ax) * (by - ay) - (gyy - ay) * (bx - ax)
            inside &= e > 0
        assert np.all(count[inside] == 1)


def test_back_faces_and_degenerates_are_culled(oracle):
    X = np.array([[0, 10 * FIX, 10 * FIX], [0, 5 * FIX, 10 * FIX]], np.int64)
    Y = np.array([[0, 0, 10 * FIX], [0, 5 * FIX, 10 * FIX]], np.int64)   # clockwise on screen; collinear
    _, _, count = oracle.raster_fixed(16, 16, X, Y, np.ones((2, 3)))
    assert count.sum() == 0
    _, _, count = oracle.raster_fixed(16, 16, X[:1, [0, 2, 1]], Y[:1, [0, 2, 1]], np.ones((1, 3)))
    assert count.sum() > 0


def test_coplanar_tie_goes_to_lower_primitive(oracle):
    """Two identical overlapping quads: the first in the list wins everywhere; swapping swaps the winner."""
    X, Y = quad_tris(3 * FIX, 2 * FIX, 12 * FIX + 77, 11 * FIX + 5)
    XX, YY = np.concatenate([X, X]), np.concatenate([Y, Y])
    key, depth, count = oracle.raster_fixed(16, 16, XX, YY, np.full((4, 3), 0.5))
    cov = count > 0
    assert np.all(count[cov] == 2)
    assert np.all(key[cov] < 4)      # keys 0, 2 belong to the first quad
    # full pipeline: two instances of the same quad mesh at the same pose
    quad = sg.quad_mesh([(-1, -1, 0), (1, -1, 0), (1, 1, 0), (-1, 1, 0)], (0, 0, 1))
    cam = scenes.camera_down((0.1, 0.05, 3.0), 32, 32, fovy_deg=50)
    for order in ([0, 1], [1, 0]):
        b = scenes.single_sample([quad], [0, 0], [scenes.identity_pose()] * 2, [cam], seg=np.array([7, 9])[order])
        o = oracle.render(b, debug=True)
        hit = o["prim"] >= 0
        assert hit.sum() > 100
        assert np.all(o["seg"][hit] == (7 if order == [0, 1] else 9))
        assert np.all(o["prim"][hit] < 4)


def test_orthographic_cube_exact_pixel_count(oracle):
    """A side-s cube seen orthographically along -z at f px/m with s*f integer covers exactly (s*f)^2
    pixels wherever it sits on the subpixel grid; its top-face depth is the camera-to-face distance."""
    rng = np.random.default_rng(5)
    cube = sg.box_mesh(0.5, per_face_material=False)
    for _ in range(8):
        f = float(rng.choice([8, 12, 16]))           # 1 m side -> f pixels
        off = rng.uniform(-3, 3, 2) / f               # off-grid centre (metres)
        zc = float(rng.uniform(2.0, 5.0))
        cam = scenes.camera_down((0.0, 0.0, zc), 48, 48, px_per_m=f)
        b = scenes.single_sample([cube], [0], [scenes.pose(t=(off[0], off[1], 0.0))], [cam], seg=[2])
        o = oracle.render(b, gbuffer=True)
        seg = o["seg"].reshape(48, 48)
        assert (seg == 2).sum() == int(f) ** 2
        d = o["depth"][o["seg"] == 2]
        exp = np.float32(zc) - np.float32(0.5)
        assert np.all(np.abs(d - exp) <= 2 * np.spacing(exp))
        n = o["gb_nrm"][o["seg"] == 2]
        np.testing.assert_array_equal(n, np.tile([0.0, 0.0, 1.0], (len(n), 1)).astype(np.float32))


def test_plane_depth_camera_straight_down(oracle):
    plane = sg.plane_mesh(20.0, 20.0)
    for h in (0.37, 1.0, 2.5):
        cam = scenes.camera_down((0.013, -0.021, h), 33, 29, fovy_deg=60)
        b = scenes.single_sample([plane], [0], [scenes.identity_pose()], [cam])
        o = oracle.render(b)
        assert (o["seg"] == 1).all()
        np.testing.assert_allclose(o["depth"], h, rtol=1e-6)


def _tilted_plane(half, pitch, W=64, H=48):
    plane = sg.plane_mesh(half, half)
    th = math.radians(pitch)
    eye = np.array([0.2, -2.0 * math.cos(th), 2.0 * math.sin(th)])
    view, intr, wh = scenes.camera_look(eye, (0.2, 0.0, 0.0), W, H, 50.0)
    return scenes.single_sample([plane], [0], [scenes.identity_pose()], [(view, intr, wh)])


def _rays(b, W, H):
    fx, fy, cx, cy = b.cam_intr[0, :4].astype(np.float64)
    xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    return np.stack([(xs - cx) / fx, -(ys - cy) / fy, -np.ones_like(xs)], -1)


def test_plane_depth_tilted_camera_closed_form(oracle):
    """depth(x, y) = (n_v . t) / (n_v . (u_x, u_y, -1)) for the plane z = 0 seen by a pitched camera.

    Vertices are snapped to 1/256 px while keeping their exact 1/w, which shifts the interpolated
    1/w of a triangle spanning hundreds of pixels (and a factor ~10 in 1/w) by up to ~1e-4
    relative; the exact comparison against the snapped triangle is the next test."""
    W, H = 64, 48
    for pitch in (20.0, 35.0, 55.0):
        b = _tilted_plane(40.0, pitch, W, H)
        o = oracle.render(b)
        V = b.cam_view[0].astype(np.float64)
        nv = V[:, :3] @ np.array([0.0, 0.0, 1.0])
        t = V[:, 3]
        ray = _rays(b, W, H)
        denom = ray @ nv
        depth = (nv @ t) / denom
        # world hit point: p_w = R^T (depth * ray - t); the plane ends at |x|, |y| = 40 m
        pw = np.einsum("ji,hwj->hwi", V[:, :3], depth[..., None] * ray - t)
        inside = (denom < 0) & (np.abs(pw[..., 0]) < 39.0) & (np.abs(pw[..., 1]) < 39.0)
        missed = (denom >= 0) | (np.abs(pw[..., 0]) > 41.0) | (np.abs(pw[..., 1]) > 41.0)
        got = o["depth"].reshape(H, W)
        assert inside.sum() > W * H // 3
        assert np.all(got[inside] > 0) and np.all(got[missed] == 0)
        np.testing.assert_allclose(got[inside], depth[inside], rtol=2e-3)


def test_plane_depth_matches_snapped_triangle_exactly(oracle):
    """Given the snapped vertices (X/256, Y/256) and their 1/w, depth is 1 / (the affine function of
    screen position through those three points), to 1e-6: an independent plane fit in fp64."""
    W, H = 64, 48
    for pitch in (35.0, 55.0):
        b = _tilted_plane(2.0, pitch, W, H)
        o = oracle.render(b, debug=True)
        assert o["counters"][2] == 0
        V = b.cam_view[0]
        fx, fy, cx, cy = b.cam_intr[0, :4]
        m = b.meshes[0]
        f32 = np.float32
        # the snapped inputs: fp32 view transform, 1/w and projection as the renderer defines them
        pc = [((V[i, 0] * m.pos[:, 0] + V[i, 1] * m.pos[:, 1]) + V[i, 2] * m.pos[:, 2]) + V[i, 3] for i in range(3)]
        iw = (f32(1.0) / (-pc[2])).astype(f32)
        xs = (cx + fx * (pc[0] * iw)).astype(f32)
        ys = (cy - fy * (pc[1] * iw)).astype(f32)
        X = np.rint(xs * f32(256)).astype(np.float64) / 256.0
        Y = np.rint(ys * f32(256)).astype(np.float64) / 256.0
        got = o["depth"].reshape(H, W)
        prim = (o["prim"] // 2).reshape(H, W)
        px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
        for t in range(m.n_tris):
            v = m.idx[t]
            A = np.stack([X[v], Y[v], np.ones(3)], 1)
            coef = np.linalg.solve(A, iw[v].astype(np.float64))
            sel = prim == t
            assert sel.sum() > 50
            exp = 1.0 / (coef[0] * px[sel] + coef[1] * py[sel] + coef[2])
            np.testing.assert_allclose(got[sel], exp, rtol=1e-6)


def test_near_plane_clipping_keeps_the_visible_part(oracle):
    """The tiny workload's 10 m plane passes behind the camera: it is clipped, not dropped or culled."""
    b = sg.tiny_batch(0, n_samples=2)
    o = oracle.render(b, debug=True)
    assert o["counters"][2] > 0          # clipped triangles
    assert o["counters"][3] == 0         # none dropped by the guard band
    seg = o["seg"].reshape(2, 64, 64)
    assert (seg[:, -1, :] == 1).all()    # the bottom row looks at the near part of the plane
