"""Brute-force fp64 ray casting against the oracle on small scenes.

A ray from the camera centre through each pixel centre is intersected
(Moller-Trumbore, fp64, world space) with every front-facing triangle; the
nearest hit beyond the near plane must be the oracle's winning primitive, its
distance along the view axis the oracle's depth, and the barycentric
interpolation of the world normals at the hit the oracle's normal.  This is an
independent formulation (3-D rays instead of 2-D edge functions) of the
transform, projection, pixel-centre, y-flip, culling, clipping, depth and
perspective-correct interpolation conventions.  Pixels whose centre lies within
a small distance of a projected triangle edge (where the 1/512 px vertex
snapping may move coverage) or whose two nearest hits are within 1e-5 in depth
are counted and excluded.
"""

import numpy as np
import pytest

from paper_1906_11633_b300 import scenegen as sg

EDGE_EPS_PX = 0.02


def _world_tris(batch, s):
    tris, nrms, prim_ids, segs = [], [], [], []
    prim = 0
    for inst in range(batch.inst_offset[s], batch.inst_offset[s + 1]):
        m = batch.meshes[batch.inst_mesh[inst]]
        P = batch.inst_pose[inst].astype(np.float64)
        pw = m.pos.astype(np.float64) @ P[:, :3].T + P[:, 3]
        nw = m.nrm.astype(np.float64) @ P[:, :3].T
        tris.append(pw[m.idx.astype(np.int64)])
        nrms.append(nw[m.idx.astype(np.int64)])
        prim_ids.append(prim + np.arange(m.n_tris))
        segs.append(np.full(m.n_tris, batch.inst_seg[inst]))
        prim += m.n_tris
    return np.concatenate(tris), np.concatenate(nrms), np.concatenate(prim_ids), np.concatenate(segs)


def raycast_image(batch, c):
    s = batch.cam_sample[c]
    W, H = batch.cam_wh[c]
    V = batch.cam_view[c].astype(np.float64)
    fx, fy, cx, cy, near, _ = batch.cam_intr[c].astype(np.float64)
    R, t = V[:, :3], V[:, 3]
    T, N, prim, seg = _world_tris(batch, s)
    # view-space vertices, for culling, bounding boxes and edge distances
    Tv = T @ R.T + t
    e1, e2 = T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]
    eye = -R.T @ t
    fn = np.cross(e1, e2)
    front = np.einsum("ij,ij->i", fn, eye - T[:, 0]) > 0
    best = np.full((H, W), np.inf)
    second = np.full((H, W), np.inf)
    best_prim = np.full((H, W), -1, np.int64)
    best_n = np.zeros((H, W, 3))
    best_seg = np.zeros((H, W), np.int64)
    ambiguous = np.zeros((H, W), bool)
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    for k in np.nonzero(front)[0]:
        z = Tv[k, :, 2]
        if np.all(z > -near):
            continue
        if np.all(z <= -near):
            xs = cx + fx * Tv[k, :, 0] / -z
            ys = cy - fy * Tv[k, :, 1] / -z
            x0, x1 = int(max(0, np.floor(xs.min() - 1))), int(min(W, np.ceil(xs.max() + 1)))
            y0, y1 = int(max(0, np.floor(ys.min() - 1))), int(min(H, np.ceil(ys.max() + 1)))
            if x0 >= x1 or y0 >= y1:
                continue
            sl = (slice(y0, y1), slice(x0, x1))
            # distance of each pixel centre to the three projected edges
            for a, b in ((0, 1), (1, 2), (2, 0)):
                ex, ey = xs[b] - xs[a], ys[b] - ys[a]
                L = np.hypot(ex, ey)
                if L == 0:
                    continue
                d = np.abs((px[sl] - xs[a]) * ey - (py[sl] - ys[a]) * ex) / L
                tpar = ((px[sl] - xs[a]) * ex + (py[sl] - ys[a]) * ey) / (L * L)
                ambiguous[sl] |= (d < EDGE_EPS_PX) & (tpar > -0.01) & (tpar < 1.01)
        else:
            sl = (slice(0, H), slice(0, W))
        # rays through the pixel centres of the box, world space
        dv = np.stack([(px[sl] - cx) / fx, -(py[sl] - cy) / fy, -np.ones_like(px[sl])], -1)
        dw = dv @ R  # R^T dv
        pvec = np.cross(dw, e2[k])
        det = pvec @ e1[k]
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / det
            tvec = eye - T[k, 0]
            u = (pvec @ tvec) * inv
            qvec = np.cross(tvec, e1[k])
            v = np.einsum("j,...j->...", qvec, dw) * inv
            tt = (qvec @ e2[k]) * inv
        hit = (np.abs(det) > 1e-300) & (u >= 0) & (v >= 0) & (u + v <= 1) & (tt >= near)
        # depth along the view axis equals tt because dv has z = -1
        if not hit.any():
            continue
        depth = np.where(hit, tt, np.inf)
        bsl, ssl = best[sl], second[sl]
        closer = depth < bsl
        ssl[closer] = bsl[closer]
        ssl[~closer] = np.minimum(ssl[~closer], depth[~closer])
        bsl[closer] = depth[closer]
        best_prim[sl][closer] = prim[k]
        best_seg[sl][closer] = seg[k]
        n = (1 - u - v)[..., None] * N[k, 0] + u[..., None] * N[k, 1] + v[..., None] * N[k, 2]
        best_n[sl][closer] = (n @ R.T)[closer]
        best[sl], second[sl] = bsl, ssl
    nl = np.linalg.norm(best_n, axis=-1, keepdims=True)
    best_n = np.divide(best_n, nl, out=np.zeros_like(best_n), where=nl > 0)
    with np.errstate(invalid="ignore"):
        ties = np.isfinite(second) & (np.abs(second - best) <= 1e-5 * best)
    return best_prim, best, best_n, best_seg, ambiguous | ties


@pytest.mark.parametrize("kind", ["tiny", "hand"])
def test_oracle_matches_raycast(oracle, kind):
    if kind == "tiny":
        b = sg.tiny_batch(7, n_samples=3, res=48)
    else:
        b = sg.hand_batch(3, np.arange(2), res=56, n_cams=3)
    o = oracle.render(b, gbuffer=True, debug=True)
    total_amb = 0
    total_px = 0
    errs = []
    for c in range(b.n_cams):
        W, H = b.cam_wh[c]
        sl = slice(b.img_offset[c], b.img_offset[c] + W * H)
        prim, depth, nrm, seg, amb = raycast_image(b, c)
        got_prim = np.where(o["prim"][sl] >= 0, o["prim"][sl] // 2, -1).reshape(H, W)
        ok = ~amb
        total_amb += amb.sum()
        total_px += W * H
        np.testing.assert_array_equal(got_prim[ok], prim[ok])
        np.testing.assert_array_equal(o["seg"][sl].reshape(H, W)[ok], np.where(prim[ok] >= 0, seg[ok], 0))
        vis = ok & (prim >= 0)
        np.testing.assert_allclose(o["depth"][sl].reshape(H, W)[vis], depth[vis], rtol=2e-3)
        gn = o["gb_nrm"][sl].reshape(H, W, 3)[vis]
        errs.append(np.abs(gn - nrm[vis]).max(-1))
    assert total_amb < 0.05 * total_px, (total_amb, total_px)
    # snapping moves the vertices of 1-2 px sliver triangles by up to 1/512 px, which moves
    # their barycentrics (and so the interpolated normal) by up to ~1e-2 on a handful of pixels
    e = np.concatenate(errs)
    assert np.percentile(e, 99) < 1e-3 and e.max() < 3e-2


def test_normal_interpolation_is_perspective_correct(oracle):
    """One large triangle with three different vertex normals, strongly tilted so 1/w varies by
    ~4x across it: the oracle's normal equals the fp64 barycentric normal at the ray hit."""
    from tests import scenes
    corners = np.array([(-1.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 6.0, 0.0)])
    nv = np.array([(0.6, -0.3, 0.74), (-0.5, 0.2, 0.84), (0.1, 0.7, 0.7)])
    nv /= np.linalg.norm(nv, axis=1, keepdims=True)
    mesh = sg.Mesh(corners.astype(np.float32), nv.astype(np.float32), np.array([[0, 1, 2]], np.uint32),
                   np.zeros(1, np.uint8))
    cam = scenes.camera_look((0.0, -1.5, 0.8), (0.0, 2.0, 0.0), 96, 96, 70.0)
    b = scenes.single_sample([mesh], [0], [scenes.identity_pose()], [cam])
    o = oracle.render(b, gbuffer=True, debug=True)
    prim, depth, nrm, seg, amb = raycast_image(b, 0)
    vis = (~amb) & (prim >= 0)
    assert vis.sum() > 1000
    got = o["gb_nrm"].reshape(96, 96, 3)[vis]
    np.testing.assert_allclose(got, nrm[vis], atol=3e-4)
    d = depth[vis]
    assert d.max() / d.min() > 3.0
