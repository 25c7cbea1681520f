"""Seeded synthetic scenes and randomizer parameters -- renderer INPUTS only.

This module builds what a caller hands to the renderer: meshes that are shared
by every sample of a batch (Single Scene Multiple States, Sec. 3) and the
per-sample state and randomization parameters that the paper's randomizer
components draw (Sec. 4.3.1: joint positions, camera jitter, light positions
and intensities, material tint/specular/glossiness, a post-processing scalar).
It holds none of the renderer's arithmetic: no transform into view space, no
projection, rasterisation or shading happens here.  The CUDA path and the CPU
oracle both consume the arrays it produces.

Determinism (Sec. 4.3): every random number is a Philox4x32-10 output keyed by
(seed, stream) with counter (sample index, block).  Each randomizer owns one
stream, so a sample's parameters do not depend on which other samples share
its batch, nor on how many draws another randomizer makes.

Workload shapes (the paper's Shadow-Hand scene, Sec. 5, is not available; a
procedural capsule hand of the same scale stands in for it):
  tiny_batch    -- unit cube on a 10 m plane, 64x64, 1 directional light
  hand_batch    -- 24 capsule links + 5 cm block + 1 m table, 3 cameras
  benchmark_batch -- the hand scene lit and coloured the way the paper's benchmark
                  configures it (Sec. 5): 3 spot lights placed by LightSetup with
                  LightRandomizer levels and cones, FixedHue block materials with
                  emission, camera jitter or orbit, post-processing grading
  uneven_batch  -- 1..156 capsule links per scene, mixed square resolutions
  perturb_params-- target parameters for the differentiation workload
  poisson_requests -- request stream for the serving loop
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional, List, Sequence

import numpy as np

MAX_LIGHTS = 4
MAX_MATERIALS = 32
CAM_PERSPECTIVE = 0
CAM_ORTHOGRAPHIC = 1
LIGHT_POINT = 0
LIGHT_DIRECTIONAL = 1
LIGHT_SPOT = 2

# One stream per randomizer, so the draws of one never shift another's.
STREAM_MESHES = 1
STREAM_JOINTS = 2
STREAM_BLOCK = 3
STREAM_CAMERA = 4
STREAM_LIGHTS = 5
STREAM_MATERIALS = 6
STREAM_POST = 7
STREAM_SCENE = 8
STREAM_TARGET = 9
STREAM_REQUESTS = 10
STREAM_GRADING = 11
STREAM_FIXED_HUE = 12
STREAM_LIGHT_SETUP = 13
STREAM_LIGHT_LEVELS = 14
STREAM_ORBIT = 15
STREAM_POST_EFFECTS = 16

# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
# easy as 1, 2, 3", SC 2011): 10 rounds of two 32x32->64 multiplies with a
# Weyl-sequence key schedule.
# --------------------------------------------------------------------------
_PHILOX_M0 = 0xD2511F53
_PHILOX_M1 = 0xCD9E8D57
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32-10 block function on broadcastable uint32 counter arrays."""
    c = np.broadcast_arrays(*[np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3)])
    x0, x1, x2, x3 = [v.copy() for v in c]
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    m0 = np.uint64(_PHILOX_M0)
    m1 = np.uint64(_PHILOX_M1)
    for _ in range(10):
        p0 = x0 * m0
        p1 = x2 * m1
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        x0, x1, x2, x3 = hi1 ^ x1 ^ np.uint64(k0), lo1, hi0 ^ x3 ^ np.uint64(k1), lo0
        k0 = (k0 + _PHILOX_W0) & 0xFFFFFFFF
        k1 = (k1 + _PHILOX_W1) & 0xFFFFFFFF
    return tuple(v.astype(np.uint32) for v in (x0, x1, x2, x3))


def uniform(seed: int, stream: int, samples, n: int) -> np.ndarray:
    """[len(samples), n] float64 draws in (0, 1), keyed (seed, stream), counter (sample, block)."""
    samples = np.asarray(samples, dtype=np.int64).reshape(-1)
    nb = (n + 3) // 4
    s = samples[:, None]
    b = np.arange(nb, dtype=np.int64)[None, :]
    out = philox4x32_10(s & 0xFFFFFFFF, b, s >> 32, 0, seed, stream)
    u = np.stack(out, axis=-1).reshape(len(samples), nb * 4)[:, :n]
    return (u.astype(np.float64) + 0.5) * (1.0 / 4294967296.0)


# --------------------------------------------------------------------------
# Meshes (shared across samples).  Triangles are wound counter-clockwise seen
# from outside, i.e. the face normal (b-a)x(c-a) points out of the body.
# --------------------------------------------------------------------------
@dataclass
class Mesh:
    pos: np.ndarray      # [V, 3] float32, object space (metres)
    nrm: np.ndarray      # [V, 3] float32, unit vertex normals
    idx: np.ndarray      # [T, 3] uint32, vertex indices
    tri_mat: np.ndarray  # [T] uint8, material index relative to the instance's base

    @property
    def n_verts(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.idx.shape[0])


def _orient_outward(pos: np.ndarray, nrm: np.ndarray, idx: np.ndarray) -> np.ndarray:
    a, b, c = pos[idx[:, 0]], pos[idx[:, 1]], pos[idx[:, 2]]
    fn = np.cross(b - a, c - a)
    vn = nrm[idx[:, 0]] + nrm[idx[:, 1]] + nrm[idx[:, 2]]
    flip = np.einsum("ij,ij->i", fn, vn) < 0
    out = idx.copy()
    out[flip, 1], out[flip, 2] = idx[flip, 2], idx[flip, 1]
    return out


def _finish(pos, nrm, idx, tri_mat) -> Mesh:
    pos = np.asarray(pos, np.float64)
    nrm = np.asarray(nrm, np.float64)
    nrm = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    idx = _orient_outward(pos, nrm, np.asarray(idx, np.int64))
    return Mesh(pos.astype(np.float32), nrm.astype(np.float32),
                idx.astype(np.uint32), np.asarray(tri_mat, np.uint8))


def capsule_mesh(radius: float, length: float, n_around: int = 16) -> Mesh:
    """Capsule along +x: segment [0, length], hemispherical caps of `radius`.

    11 rings of `n_around` vertices (pole, 3 cap rings, equator at x=0, a
    middle ring, equator at x=length, 3 cap rings, pole): 176 vertices and
    320 triangles for n_around = 16.  The 32 triangles touching a pole ring are
    degenerate (two coincident vertices) and are culled by the renderer.
    """
    rings = []
    for i in range(5):          # left cap, pole -> equator
        phi = 0.5 * math.pi * i / 4
        rings.append((-radius * math.cos(phi), radius * math.sin(phi), (-math.cos(phi), math.sin(phi))))
    rings.append((0.5 * length, radius, (0.0, 1.0)))
    for i in range(5):          # right cap, equator -> pole
        phi = 0.5 * math.pi * (4 - i) / 4
        rings.append((length + radius * math.cos(phi), radius * math.sin(phi), (math.cos(phi), math.sin(phi))))
    pos, nrm = [], []
    for x, rho, (nx, nr) in rings:
        for j in range(n_around):
            psi = 2.0 * math.pi * j / n_around
            cs, sn = math.cos(psi), math.sin(psi)
            pos.append((x, rho * cs, rho * sn))
            nrm.append((nx, nr * cs, nr * sn))
    idx = []
    for i in range(len(rings) - 1):
        for j in range(n_around):
            j1 = (j + 1) % n_around
            a, b = i * n_around + j, i * n_around + j1
            c, d = (i + 1) * n_around + j1, (i + 1) * n_around + j
            idx.append((a, b, c))
            idx.append((a, c, d))
    # outward orientation: ring order runs along +x and psi turns about +x
    idx = np.asarray(idx, np.int64)
    pos = np.asarray(pos, np.float64)
    nrm = np.asarray(nrm, np.float64)
    # decide the winding from a non-degenerate band, then apply it uniformly
    a, b, c = pos[idx[40, 0]], pos[idx[40, 1]], pos[idx[40, 2]]
    if np.dot(np.cross(b - a, c - a), nrm[idx[40, 0]] + nrm[idx[40, 1]] + nrm[idx[40, 2]]) < 0:
        idx = idx[:, [0, 2, 1]]
    return Mesh(pos.astype(np.float32), (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32),
                idx.astype(np.uint32), np.zeros(len(idx), np.uint8))


def box_mesh(half: float, per_face_material: bool = True) -> Mesh:
    """Axis-aligned cube centred at the origin: 24 vertices (flat faces), 12 triangles."""
    pos, nrm, idx, mat = [], [], [], []
    for face, (axis, sgn) in enumerate([(0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1)]):
        u, v = [k for k in range(3) if k != axis]
        base = len(pos)
        for cu, cv in [(-1, -1), (1, -1), (1, 1), (-1, 1)]:
            p = [0.0, 0.0, 0.0]
            p[axis] = sgn * half
            p[u] = cu * half
            p[v] = cv * half
            n = [0.0, 0.0, 0.0]
            n[axis] = float(sgn)
            pos.append(p)
            nrm.append(n)
        idx += [(base, base + 1, base + 2), (base, base + 2, base + 3)]
        mat += [face if per_face_material else 0] * 2
    return _finish(pos, nrm, idx, mat)


def plane_mesh(half_x: float, half_y: float) -> Mesh:
    """Plane z = 0 facing +z: 4 vertices, 2 triangles."""
    pos = [(-half_x, -half_y, 0), (half_x, -half_y, 0), (half_x, half_y, 0), (-half_x, half_y, 0)]
    nrm = [(0, 0, 1)] * 4
    return _finish(pos, nrm, [(0, 1, 2), (0, 2, 3)], [0, 0])


def quad_mesh(corners, normal) -> Mesh:
    """Planar quad with the given 4 corners (counter-clockwise about `normal`)."""
    return _finish(corners, [normal] * 4, [(0, 1, 2), (0, 2, 3)], [0, 0])


# --------------------------------------------------------------------------
# Batch description (host numpy arrays, the layout the C-ABI takes)
# --------------------------------------------------------------------------
@dataclass
class Batch:
    meshes: List[Mesh]
    inst_offset: np.ndarray    # [B+1] int32, CSR of instances per sample
    inst_mesh: np.ndarray      # [I] uint32, index into `meshes`
    inst_pose: np.ndarray      # [I, 3, 4] float32, world-from-object (rigid)
    inst_seg: np.ndarray       # [I] uint8, segmentation id
    inst_mat_base: np.ndarray  # [I] int16, first material slot of the instance
    cam_offset: np.ndarray     # [B+1] int32, CSR of cameras per sample
    cam_sample: np.ndarray     # [C] int32, owning sample of each camera
    cam_view: np.ndarray       # [C, 3, 4] float32, camera-from-world (OpenGL axes)
    cam_intr: np.ndarray       # [C, 6] float32: fx, fy, cx, cy, near, type
    cam_wh: np.ndarray         # [C, 2] int32: width, height
    img_offset: np.ndarray     # [C] int64, first pixel of each image in the flat outputs
    light: np.ndarray          # [B, 4, 4] float32: position (or direction) xyz, intensity
    light_meta: np.ndarray     # [B, 2] int32: count, type
    material: np.ndarray       # [B, 32, 5] float32: albedo rgb, specular, shininess
    exposure_ev: np.ndarray    # [B] float32
    ambient: np.ndarray        # [B, 3] float32
    background: np.ndarray     # [B, 3] float32
    sample_ids: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    # [B, 8] float32 colour-grading epilogue (hue, saturation, contrast, brightness, temperature,
    # tint, grain amplitude, grain seed: an integer below 2^24), or None for none
    grading: Optional[np.ndarray] = None
    # [B, 4, 5] float32 cones of spot lights (light type 2): world axis xyz (unit), cos of the outer
    # and of the inner half-angle; or None
    light_spot: Optional[np.ndarray] = None
    # [B, 32] float32 material emission e (the emitted colour is e * albedo), or None for none
    emission: Optional[np.ndarray] = None
    # [B, 4] float32 post-processing: ambient-occlusion intensity, bloom intensity, bloom radius
    # (pixels), 0; or None for none
    post: Optional[np.ndarray] = None
    # shadows: per light shadow_faces shadow cameras (one for a spot light, six cube faces for a
    # point light, one orthographic for a directional light), views [B, 4, F, 3, 4]
    # (camera-from-world) and intrinsics [B, 4, F, 7] (fx, fy, cx, cy, near, depth bias, type:
    # 0 perspective, 1 orthographic; fx == 0: that face casts none), rendered
    # into square maps of side shadow_res; None / 0 for no shadows
    shadow_view: Optional[np.ndarray] = None
    shadow_intr: Optional[np.ndarray] = None
    shadow_res: int = 0
    shadow_faces: int = 1

    @property
    def n_samples(self) -> int:
        return int(self.inst_offset.shape[0] - 1)

    @property
    def n_cams(self) -> int:
        return int(self.cam_wh.shape[0])

    @property
    def n_inst(self) -> int:
        return int(self.inst_mesh.shape[0])

    @property
    def total_pixels(self) -> int:
        return int((self.cam_wh[:, 0].astype(np.int64) * self.cam_wh[:, 1]).sum())

    def tris_per_sample(self) -> np.ndarray:
        nt = np.array([m.n_tris for m in self.meshes], np.int64)
        per_inst = nt[self.inst_mesh]
        return np.add.reduceat(per_inst, self.inst_offset[:-1]) if self.n_inst else np.zeros(self.n_samples, np.int64)

    def tri_images(self) -> int:
        tps = self.tris_per_sample()
        cams = np.diff(self.cam_offset)
        return int((tps * cams).sum())

    def with_params(self, **kw) -> "Batch":
        return replace(self, **kw)


def concat_batches(batches: Sequence[Batch]) -> Batch:
    """Concatenate batches that share the same mesh list (SSMS)."""
    meshes = batches[0].meshes
    for b in batches:
        assert b.meshes is meshes or len(b.meshes) == len(meshes)
    inst_counts = np.concatenate([np.diff(b.inst_offset) for b in batches])
    cam_counts = np.concatenate([np.diff(b.cam_offset) for b in batches])
    cam_sample = []
    base = 0
    for b in batches:
        cam_sample.append(b.cam_sample + base)
        base += b.n_samples
    wh = np.concatenate([b.cam_wh for b in batches])
    return Batch(
        meshes=meshes,
        inst_offset=np.concatenate([[0], np.cumsum(inst_counts)]).astype(np.int32),
        inst_mesh=np.concatenate([b.inst_mesh for b in batches]),
        inst_pose=np.concatenate([b.inst_pose for b in batches]),
        inst_seg=np.concatenate([b.inst_seg for b in batches]),
        inst_mat_base=np.concatenate([b.inst_mat_base for b in batches]),
        cam_offset=np.concatenate([[0], np.cumsum(cam_counts)]).astype(np.int32),
        cam_sample=np.concatenate(cam_sample).astype(np.int32),
        cam_view=np.concatenate([b.cam_view for b in batches]),
        cam_intr=np.concatenate([b.cam_intr for b in batches]),
        cam_wh=wh,
        img_offset=_img_offsets(wh),
        light=np.concatenate([b.light for b in batches]),
        light_meta=np.concatenate([b.light_meta for b in batches]),
        material=np.concatenate([b.material for b in batches]),
        exposure_ev=np.concatenate([b.exposure_ev for b in batches]),
        ambient=np.concatenate([b.ambient for b in batches]),
        background=np.concatenate([b.background for b in batches]),
        sample_ids=np.concatenate([b.sample_ids for b in batches]),
        grading=_concat_opt(batches, "grading", identity_grading),
        light_spot=_concat_opt(batches, "light_spot", lambda n: np.zeros((n, MAX_LIGHTS, 5), np.float32)),
        emission=_concat_opt(batches, "emission", lambda n: np.zeros((n, MAX_MATERIALS), np.float32)),
        post=_concat_opt(batches, "post", lambda n: np.zeros((n, 4), np.float32)),
        shadow_view=_concat_opt(batches, "shadow_view",
                                lambda n: np.zeros((n, MAX_LIGHTS, _shadow_kind(batches)[1], 3, 4), np.float32)),
        shadow_intr=_concat_opt(batches, "shadow_intr",
                                lambda n: np.zeros((n, MAX_LIGHTS, _shadow_kind(batches)[1], 7), np.float32)),
        shadow_res=_shadow_kind(batches)[0],
        shadow_faces=_shadow_kind(batches)[1],
    )


def _shadow_kind(batches):
    """(shadow_res, shadow_faces) shared by the batches with shadows."""
    kinds = {(b.shadow_res, b.shadow_faces) for b in batches if b.shadow_view is not None}
    assert len(kinds) <= 1, "batches with shadows must share one shadow-map size and face count"
    return kinds.pop() if kinds else (0, 1)


def _concat_opt(batches, name, neutral):
    """Concatenate an optional per-sample array; batches without it contribute `neutral(n_samples)`."""
    if all(getattr(b, name) is None for b in batches):
        return None
    return np.concatenate([getattr(b, name) if getattr(b, name) is not None else neutral(b.n_samples)
                           for b in batches])


def select_samples(batch: Batch, idx: Sequence[int]) -> Batch:
    """Sub-batch holding samples `idx` (in that order) of `batch`."""
    parts = []
    for s in idx:
        i0, i1 = batch.inst_offset[s], batch.inst_offset[s + 1]
        c0, c1 = batch.cam_offset[s], batch.cam_offset[s + 1]
        wh = batch.cam_wh[c0:c1]
        parts.append(Batch(
            meshes=batch.meshes,
            inst_offset=np.array([0, i1 - i0], np.int32),
            inst_mesh=batch.inst_mesh[i0:i1], inst_pose=batch.inst_pose[i0:i1],
            inst_seg=batch.inst_seg[i0:i1], inst_mat_base=batch.inst_mat_base[i0:i1],
            cam_offset=np.array([0, c1 - c0], np.int32), cam_sample=np.zeros(c1 - c0, np.int32),
            cam_view=batch.cam_view[c0:c1], cam_intr=batch.cam_intr[c0:c1], cam_wh=wh,
            img_offset=_img_offsets(wh),
            light=batch.light[s:s + 1], light_meta=batch.light_meta[s:s + 1],
            material=batch.material[s:s + 1], exposure_ev=batch.exposure_ev[s:s + 1],
            ambient=batch.ambient[s:s + 1], background=batch.background[s:s + 1],
            sample_ids=batch.sample_ids[s:s + 1] if len(batch.sample_ids) else np.array([s]),
            grading=batch.grading[s:s + 1] if batch.grading is not None else None,
            light_spot=batch.light_spot[s:s + 1] if batch.light_spot is not None else None,
            emission=batch.emission[s:s + 1] if batch.emission is not None else None,
            post=batch.post[s:s + 1] if batch.post is not None else None,
            shadow_view=batch.shadow_view[s:s + 1] if batch.shadow_view is not None else None,
            shadow_intr=batch.shadow_intr[s:s + 1] if batch.shadow_intr is not None else None,
            shadow_res=batch.shadow_res,
            shadow_faces=batch.shadow_faces,
        ))
    return concat_batches(parts)


def _img_offsets(wh: np.ndarray) -> np.ndarray:
    px = wh[:, 0].astype(np.int64) * wh[:, 1].astype(np.int64)
    return np.concatenate([[0], np.cumsum(px)[:-1]]).astype(np.int64) if len(px) else np.zeros(0, np.int64)


# --------------------------------------------------------------------------
# Rigid-transform helpers (float64, inputs only)
# --------------------------------------------------------------------------
def _rot(axis: str, ang: np.ndarray) -> np.ndarray:
    ang = np.asarray(ang, np.float64)
    c, s = np.cos(ang), np.sin(ang)
    o, z = np.ones_like(ang), np.zeros_like(ang)
    if axis == "x":
        m = [[o, z, z], [z, c, -s], [z, s, c]]
    elif axis == "y":
        m = [[c, z, s], [z, o, z], [-s, z, c]]
    else:
        m = [[c, -s, z], [s, c, z], [z, z, o]]
    return np.moveaxis(np.array(m), [0, 1], [-2, -1])


def _hom(R: np.ndarray, t) -> np.ndarray:
    R = np.asarray(R, np.float64)
    T = np.zeros(R.shape[:-2] + (4, 4))
    T[..., :3, :3] = R
    T[..., :3, 3] = t
    T[..., 3, 3] = 1.0
    return T


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera-from-world rotation rows (right, up, back) for OpenGL axes."""
    eye, target, up = (np.asarray(v, np.float64) for v in (eye, target, up))
    f = target - eye
    f = f / np.linalg.norm(f, axis=-1, keepdims=True)
    r = np.cross(f, up)
    r = r / np.linalg.norm(r, axis=-1, keepdims=True)
    u = np.cross(r, f)
    return np.stack([r, u, -f], axis=-2)


def view_matrix(R: np.ndarray, eye) -> np.ndarray:
    eye = np.asarray(eye, np.float64)
    t = -np.einsum("...ij,...j->...i", R, eye)
    return np.concatenate([R, t[..., None]], axis=-1)


def perspective_intrinsics(width: int, height: int, fovy_deg: float, near: float = 0.01) -> np.ndarray:
    f = 0.5 * height / math.tan(math.radians(fovy_deg) / 2.0)
    return np.array([f, f, 0.5 * width, 0.5 * height, near, CAM_PERSPECTIVE], np.float64)


def _square_intrinsics(res: np.ndarray, fovy_deg: float, near: float = 0.01):
    """Perspective intrinsics [C, 6] and sizes [C, 2] of square images of side res[c]."""
    res = np.asarray(res, np.float64)
    f = 0.5 * res / math.tan(math.radians(fovy_deg) / 2.0)
    intr = np.stack([f, f, 0.5 * res, 0.5 * res, np.full_like(res, near), np.full_like(res, CAM_PERSPECTIVE)], -1)
    wh = np.stack([res, res], -1).astype(np.int32)
    return intr.reshape(-1, 6), wh.reshape(-1, 2)


def orthographic_intrinsics(width: int, height: int, px_per_m: float, near: float = 0.01) -> np.ndarray:
    return np.array([px_per_m, px_per_m, 0.5 * width, 0.5 * height, near, CAM_ORTHOGRAPHIC], np.float64)


# --------------------------------------------------------------------------
# Tiny workload: unit cube at random yaw on a 10 m plane
# --------------------------------------------------------------------------
def tiny_meshes() -> List[Mesh]:
    return [plane_mesh(5.0, 5.0), box_mesh(0.5, per_face_material=False)]


def tiny_batch(seed: int, n_samples: int = 8, res: int = 64, meshes=None, shadow_res: int = 0) -> Batch:
    """The tiny workload; with `shadow_res` > 0 its directional light casts shadows from an
    orthographic map of that side over the central 6 x 6 m of the plane."""
    meshes = meshes if meshes is not None else tiny_meshes()
    ids = np.arange(n_samples, dtype=np.int64)
    B = n_samples
    yaw = 2.0 * math.pi * uniform(seed, STREAM_BLOCK, ids, 1)[:, 0]
    pose = np.zeros((B, 2, 3, 4))
    pose[:, 0, :, :3] = np.eye(3)
    pose[:, 1, :, :3] = _rot("z", yaw)
    pose[:, 1, :, 3] = (0.0, 0.0, 0.5)
    pitch = math.radians(30.0)
    eye = np.array([0.0, -4.0 * math.cos(pitch), 4.0 * math.sin(pitch)])
    view = view_matrix(look_at(eye, (0.0, 0.0, 0.0)), eye)
    mat = np.zeros((B, MAX_MATERIALS, 5))
    mat[:, :, 4] = 1.0
    mat[:, :2, :3] = uniform(seed, STREAM_MATERIALS, ids, 6).reshape(B, 2, 3)
    light = np.zeros((B, MAX_LIGHTS, 4))
    d = np.array([-0.3, -0.5, -0.8])
    light[:, 0, :3] = d / np.linalg.norm(d)
    light[:, 0, 3] = 1.0
    wh = np.tile([[res, res]], (B, 1)).astype(np.int32)
    return Batch(
        meshes=meshes,
        inst_offset=(np.arange(B + 1) * 2).astype(np.int32),
        inst_mesh=np.tile([0, 1], B).astype(np.uint32),
        inst_pose=pose.reshape(-1, 3, 4).astype(np.float32),
        inst_seg=np.tile([1, 2], B).astype(np.uint8),
        inst_mat_base=np.tile([0, 1], B).astype(np.int16),
        cam_offset=np.arange(B + 1, dtype=np.int32),
        cam_sample=np.arange(B, dtype=np.int32),
        cam_view=np.tile(view[None], (B, 1, 1)).astype(np.float32),
        cam_intr=np.tile(perspective_intrinsics(res, res, 60.0)[None], (B, 1)).astype(np.float32),
        cam_wh=wh,
        img_offset=_img_offsets(wh),
        light=light.astype(np.float32),
        light_meta=np.tile([[1, LIGHT_DIRECTIONAL]], (B, 1)).astype(np.int32),
        material=mat.astype(np.float32),
        exposure_ev=np.zeros(B, np.float32),
        ambient=np.zeros((B, 3), np.float32),
        background=np.zeros((B, 3), np.float32),
        sample_ids=ids,
        **(_directional_shadows(light, shadow_res) if shadow_res > 0 else {}),
    )


def _directional_shadows(light, res):
    """An orthographic shadow camera for light 0 (directional) of every tiny sample."""
    B = len(light)
    view, intr = directional_shadow_camera(light[0, 0, :3], (0.0, 0.0, 0.5), 3.0, res)
    sv = np.zeros((B, MAX_LIGHTS, 1, 3, 4))
    si = np.zeros((B, MAX_LIGHTS, 1, 7))
    sv[:, 0, 0], si[:, 0, 0] = view, intr
    return dict(shadow_view=sv.astype(np.float32), shadow_intr=si.astype(np.float32), shadow_res=int(res),
                shadow_faces=1)


# --------------------------------------------------------------------------
# Hand-like workload: 24 capsule links on a 5-finger kinematic tree
# --------------------------------------------------------------------------
N_LINKS = 24
HAND_BASE = np.array([-0.10, 0.0, 0.10])
BLOCK_CENTRE = np.array([0.02, 0.0, 0.16])
CAMERA_TARGET = np.array([0.0, 0.0, 0.10])
# (azimuth deg, elevation deg) of the three rig cameras, 0.5 m from the target
CAMERA_RIG = [(-60.0, 40.0), (60.0, 40.0), (180.0, 55.0)]
CAMERA_DIST = 0.5
FOVY_DEG = 45.0


def link_dims(seed: int = 0):
    u = uniform(seed, STREAM_MESHES, [0], 2 * N_LINKS)[0]
    radius = 0.008 + 0.004 * u[:N_LINKS]
    length = 0.02 + 0.03 * u[N_LINKS:]
    return radius, length


def hand_meshes(seed: int = 0) -> List[Mesh]:
    """Mesh 0 table (1x1 m), mesh 1 block (5 cm, 6 face materials), meshes 2..25 capsule links."""
    radius, length = link_dims(seed)
    return [plane_mesh(0.5, 0.5), box_mesh(0.025)] + [capsule_mesh(r, l) for r, l in zip(radius, length)]


def _hand_tree(length):
    """(parent, offset xyz, fixed yaw deg, hinge axis) per link; parents precede children."""
    L = length
    tree = [(-1, (0.0, 0.0, 0.0), 0.0, "y")]
    for y in (0.022, 0.0, -0.022):
        tree.append((0, (L[0], y, 0.0), 0.0, "z"))
    starts = [(1, (0.3 * L[1], 0.018, 0.0), 50.0), (1, (L[1], 0.005, 0.0), 0.0), (2, (L[2], 0.0, 0.0), 0.0),
              (3, (L[3], 0.005, 0.0), 0.0), (3, (L[3], -0.012, 0.0), -15.0)]
    for parent, off, yaw in starts:
        first = len(tree)
        tree.append((parent, off, yaw, "z"))
        for k in range(1, 4):
            prev = first + k - 1
            tree.append((prev, (L[prev], 0.0, 0.0), 0.0, "y"))
    assert len(tree) == N_LINKS
    return tree


def _forward_kinematics(tree, base: np.ndarray, angles: np.ndarray) -> np.ndarray:
    """World-from-link transforms [B, n, 4, 4] from hinge angles [B, n]."""
    B, n = angles.shape
    T = np.zeros((B, n, 4, 4))
    for l, (parent, off, yaw, axis) in enumerate(tree):
        local = _hom(_rot("z", np.full(B, math.radians(yaw))) @ _rot(axis, angles[:, l]), np.asarray(off))
        T[:, l] = (base if parent < 0 else T[:, parent]) @ local
    return T


def _rig_views(seed: int, ids: np.ndarray, n_cams: np.ndarray, jitter: bool = True):
    """Jittered camera-from-world matrices for the first n_cams[s] rig cameras of each sample."""
    ids = np.asarray(ids)
    n_cams = np.asarray(n_cams, dtype=np.int64)
    K = len(CAMERA_RIG)
    u = uniform(seed, STREAM_CAMERA, ids, 6 * K).reshape(len(ids), K, 6)
    az = np.radians([a for a, _ in CAMERA_RIG])
    el = np.radians([e for _, e in CAMERA_RIG])
    eye0 = CAMERA_TARGET + CAMERA_DIST * np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], -1)
    R0 = look_at(eye0, np.broadcast_to(CAMERA_TARGET, eye0.shape))             # [K, 3, 3]
    sel = np.arange(K)[None, :] < n_cams[:, None]                            # [S, K]
    s_idx, k_idx = np.nonzero(sel)
    j = u[s_idx, k_idx]                                                       # [C, 6]
    eye = eye0[k_idx]
    R = R0[k_idx]
    if jitter:
        eye = eye + 0.02 * (2.0 * j[:, :3] - 1.0)
        ang = np.radians(3.0) * (2.0 * j[:, 3:] - 1.0)
        R = _rot("x", ang[:, 0]) @ _rot("y", ang[:, 1]) @ _rot("z", ang[:, 2]) @ R
    views = view_matrix(R, eye)
    return views.reshape(-1, 3, 4), s_idx.astype(np.int32)


def _lights(seed: int, ids: np.ndarray):
    B = len(ids)
    u = uniform(seed, STREAM_LIGHTS, ids, 1 + 4 * MAX_LIGHTS)
    count = 1 + np.minimum((u[:, 0] * 4).astype(np.int64), 3)
    v = u[:, 1:].reshape(B, MAX_LIGHTS, 4)
    light = np.zeros((B, MAX_LIGHTS, 4))
    light[..., 0] = -0.5 + v[..., 0]
    light[..., 1] = -0.5 + v[..., 1]
    light[..., 2] = 0.3 + 0.7 * v[..., 2]
    light[..., 3] = 0.05 + 0.20 * v[..., 3]
    light[np.arange(MAX_LIGHTS)[None, :] >= count[:, None]] = 0.0
    meta = np.stack([count, np.full(B, LIGHT_POINT)], axis=1)
    return light.astype(np.float32), meta.astype(np.int32)


def _materials(seed: int, ids: np.ndarray):
    B = len(ids)
    u = uniform(seed, STREAM_MATERIALS, ids, 5 * MAX_MATERIALS).reshape(B, MAX_MATERIALS, 5)
    mat = np.empty((B, MAX_MATERIALS, 5))
    mat[..., :3] = u[..., :3]
    mat[..., 3] = u[..., 3]
    mat[..., 4] = np.exp(u[..., 4] * math.log(128.0))   # log-uniform shininess in [1, 128]
    return mat.astype(np.float32)


def _post(seed: int, ids: np.ndarray):
    u = uniform(seed, STREAM_POST, ids, 7)
    ev = (u[:, 0] - 0.5).astype(np.float32)
    ambient = (0.1 * u[:, 1:4]).astype(np.float32)
    background = u[:, 4:7].astype(np.float32)
    return ev, ambient, background


def identity_grading(n: int) -> np.ndarray:
    """Grading parameters that leave the image unchanged."""
    g = np.zeros((n, 8), np.float32)
    g[:, 1] = 1.0   # saturation
    g[:, 2] = 1.0   # contrast
    return g


def grading_params(seed: int, sample_ids) -> np.ndarray:
    """Per-sample post-processing (the paper's post-processing randomizer, Sec. 4.3.1): hue shift
    U(+-0.1) rad, saturation U[0.8, 1.2], contrast U[0.8, 1.2], brightness U(+-0.05), temperature
    U(+-0.1), tint U(+-0.1), grain amplitude U[0, 0.05], and a grain seed (integer below 2^24)."""
    ids = np.asarray(sample_ids, dtype=np.int64).reshape(-1)
    u = uniform(seed, STREAM_GRADING, ids, 8)
    g = np.empty((len(ids), 8), np.float32)
    g[:, 0] = 0.1 * (2.0 * u[:, 0] - 1.0)
    g[:, 1] = 0.8 + 0.4 * u[:, 1]
    g[:, 2] = 0.8 + 0.4 * u[:, 2]
    g[:, 3] = 0.05 * (2.0 * u[:, 3] - 1.0)
    g[:, 4] = 0.1 * (2.0 * u[:, 4] - 1.0)
    g[:, 5] = 0.1 * (2.0 * u[:, 5] - 1.0)
    g[:, 6] = 0.05 * u[:, 6]
    g[:, 7] = np.floor(u[:, 7] * 16777216.0)   # an integer below 2^24, exact in float32
    return g


def post_params(seed: int, sample_ids) -> np.ndarray:
    """Per-sample ambient occlusion and bloom (the rest of the post-processing randomizer, Sec.
    4.3.1): AO intensity U[0, 1.5], bloom intensity U[0, 1], bloom radius U[1, 6] pixels."""
    ids = np.asarray(sample_ids, dtype=np.int64).reshape(-1)
    u = uniform(seed, STREAM_POST_EFFECTS, ids, 3)
    q = np.zeros((len(ids), 4), np.float32)
    q[:, 0] = 1.5 * u[:, 0]
    q[:, 1] = u[:, 1]
    q[:, 2] = 1.0 + 5.0 * u[:, 2]
    return q


def hand_batch(seed: int, sample_ids, res: int = 200, n_cams: int = 3, meshes=None, res_per_sample=None,
               cams_per_sample=None, grading: bool = False, shadow_res: int = 0) -> Batch:
    """Hand-like scenes: table, block, 24 capsule links posed by hinge angles U(+-60 deg); with
    `shadow_res` > 0 every point light casts shadows from six cube-face maps of that side."""
    ids = np.asarray(sample_ids, dtype=np.int64).reshape(-1)
    B = len(ids)
    meshes = meshes if meshes is not None else hand_meshes(0)
    radius, length = link_dims(0)
    tree = _hand_tree(length)
    ang = math.radians(60.0) * (2.0 * uniform(seed, STREAM_JOINTS, ids, N_LINKS) - 1.0)
    base = _hom(np.eye(3), HAND_BASE)
    links = _forward_kinematics(tree, base, ang)
    ub = uniform(seed, STREAM_BLOCK, ids, 4)
    block = _hom(_rot("z", 2.0 * math.pi * ub[:, 0]), BLOCK_CENTRE[None, :] + 0.01 * (2.0 * ub[:, 1:4] - 1.0))
    n_inst = 2 + N_LINKS
    pose = np.zeros((B, n_inst, 3, 4))
    pose[:, 0, :, :3] = np.eye(3)
    pose[:, 1] = block[:, :3, :]
    pose[:, 2:] = links[:, :, :3, :]
    cams = np.full(B, n_cams) if cams_per_sample is None else np.asarray(cams_per_sample)
    res_s = np.full(B, res) if res_per_sample is None else np.asarray(res_per_sample)
    views, owner = _rig_views(seed, ids, cams)
    intr, wh = _square_intrinsics(res_s[owner], FOVY_DEG)
    light, meta = _lights(seed, ids)
    ev, ambient, background = _post(seed, ids)
    return Batch(
        meshes=meshes,
        inst_offset=(np.arange(B + 1) * n_inst).astype(np.int32),
        inst_mesh=np.tile(np.arange(n_inst), B).astype(np.uint32),
        inst_pose=pose.reshape(-1, 3, 4).astype(np.float32),
        inst_seg=np.tile(np.concatenate([[1, 2], 3 + np.arange(N_LINKS)]), B).astype(np.uint8),
        inst_mat_base=np.tile(np.concatenate([[0, 1], 7 + np.arange(N_LINKS)]), B).astype(np.int16),
        cam_offset=np.concatenate([[0], np.cumsum(cams)]).astype(np.int32),
        cam_sample=owner,
        cam_view=views.astype(np.float32),
        cam_intr=intr.astype(np.float32),
        cam_wh=wh,
        img_offset=_img_offsets(wh),
        light=light, light_meta=meta,
        material=_materials(seed, ids),
        exposure_ev=ev, ambient=ambient, background=background,
        sample_ids=ids,
        grading=grading_params(seed, ids) if grading else None,
        **(_cube_shadows(light, meta, shadow_res) if shadow_res > 0 else {}),
    )


def _cube_shadows(light, meta, res):
    """Cube-face shadow cameras for every point light of every sample (zero rows elsewhere)."""
    B = len(light)
    sv, si = point_shadow_cameras(light[..., :3].astype(np.float64), res)     # [B, 4, 6, ...]
    on = (np.arange(MAX_LIGHTS)[None, :] < meta[:, :1]) & (meta[:, 1:2] == LIGHT_POINT)
    sv = np.where(on[..., None, None, None], sv, 0.0)
    si = np.where(on[..., None, None], si, 0.0)
    return dict(shadow_view=sv.reshape(B, MAX_LIGHTS, 6, 3, 4).astype(np.float32),
                shadow_intr=si.reshape(B, MAX_LIGHTS, 6, 7).astype(np.float32), shadow_res=int(res), shadow_faces=6)


# --------------------------------------------------------------------------
# The paper's randomizer and set-up components (Sec. 4.3.1, 4.3.2) as parameter samplers
# --------------------------------------------------------------------------
def hsv_to_rgb(hsv) -> np.ndarray:
    """HSV in [0, 1]^3 (hue wraps) to RGB, the hexcone model (Smith, SIGGRAPH 1978)."""
    hsv = np.asarray(hsv, np.float64)
    h, sat, v = hsv[..., 0] % 1.0, hsv[..., 1], hsv[..., 2]
    h6 = h * 6.0
    sector = np.floor(h6)
    f = h6 - sector
    p, q, t = v * (1.0 - sat), v * (1.0 - sat * f), v * (1.0 - sat * (1.0 - f))
    k = sector.astype(np.int64) % 6
    r = np.choose(k, [v, q, p, p, t, v])
    g = np.choose(k, [t, v, v, q, p, p])
    b = np.choose(k, [p, p, t, v, v, q])
    return np.stack([r, g, b], -1)


def glossiness_to_shininess(g) -> np.ndarray:
    """Glossiness in [0, 1] to the Blinn-Phong exponent 128^g in [1, 128]."""
    return np.exp(np.asarray(g, np.float64) * math.log(128.0))


def fixed_hue_materials(seed: int, sample_ids, hsv, radius=(0.03, 0.15, 0.15),
                        clamp=((0.0, 1.0), (0.2, 1.0), (0.2, 1.0)), specular=(0.0, 0.6), glossiness=(0.3, 0.9),
                        emissive_prob=0.15, emissive_power=(0.1, 0.6)):
    """FixedHueMaterialRandomizer (Sec. 4.3.1): materials near calibrated HSV colours [K, 3].

    Per sample and colour: each HSV component uniform within its radius of the calibrated value,
    then clamped to its range (hue wraps instead); specular (the metallic level) and glossiness
    uniform in their ranges; emissive with probability `emissive_prob`, at a power uniform in
    `emissive_power`.  Returns albedo [B, K, 3], specular [B, K], shininess [B, K], emission [B, K].
    """
    ids = np.asarray(sample_ids, dtype=np.int64).reshape(-1)
    hsv = np.asarray(hsv, np.float64).reshape(-1, 3)
    K = len(hsv)
    u = uniform(seed, STREAM_FIXED_HUE, ids, 7 * K).reshape(len(ids), K, 7)
    h = hsv + np.asarray(radius) * (2.0 * u[..., :3] - 1.0)
    h[..., 0] %= 1.0
    for c in (1, 2):
        h[..., c] = np.clip(h[..., c], clamp[c][0], clamp[c][1])
    albedo = hsv_to_rgb(h)
    ks = specular[0] + (specular[1] - specular[0]) * u[..., 3]
    alpha = glossiness_to_shininess(glossiness[0] + (glossiness[1] - glossiness[0]) * u[..., 4])
    emission = np.where(u[..., 5] < emissive_prob,
                        emissive_power[0] + (emissive_power[1] - emissive_power[0]) * u[..., 6], 0.0)
    return albedo, ks, alpha, emission


def light_setup(seed: int, sample_ids, n_lights: int, target, distance=(0.35, 0.6), height=(0.4, 0.7)):
    """LightSetup (Sec. 4.3.2): `n_lights` lights about `target`, each at a horizontal distance and
    a height above it uniform in the ranges, spread evenly in azimuth from a uniform offset, and
    each pointed at the target (LookAt).  Returns positions [B, n, 3] and unit axes [B, n, 3]."""
    ids = np.asarray(sample_ids, dtype=np.int64).reshape(-1)
    u = uniform(seed, STREAM_LIGHT_SETUP, ids, 1 + 2 * n_lights)
    az = 2.0 * math.pi * (u[:, :1] + np.arange(n_lights)[None, :] / n_lights)
    d = distance[0] + (distance[1] - distance[0]) * u[:, 1:1 + n_lights]
    hgt = height[0] + (height[1] - height[0]) * u[:, 1 + n_lights:]
    target = np.asarray(target, np.float64)
    pos = target + np.stack([d * np.cos(az), d * np.sin(az), hgt], -1)
    axis = target - pos
    return pos, axis / np.linalg.norm(axis, axis=-1, keepdims=True)


def light_levels(seed: int, sample_ids, n_lights: int, total=(0.5, 1.0), weight=(0.5, 1.0),
                 outer_deg=(25.0, 45.0), softness=(0.1, 0.4)):
    """LightRandomizer (Sec. 4.3.1): the total illumination uniform in `total`, split over the
    lights in proportion to relative weights uniform in `weight`; spot cones with an outer
    half-angle uniform in `outer_deg` and an inner one `1 - softness` times it.  Returns
    intensities [B, n] (summing to the total), cos outer [B, n] and cos inner [B, n]."""
    ids = np.asarray(sample_ids, dtype=np.int64).reshape(-1)
    u = uniform(seed, STREAM_LIGHT_LEVELS, ids, 1 + 3 * n_lights)
    T = total[0] + (total[1] - total[0]) * u[:, :1]
    w = weight[0] + (weight[1] - weight[0]) * u[:, 1:1 + n_lights]
    intensity = T * w / w.sum(axis=1, keepdims=True)
    outer = np.radians(outer_deg[0] + (outer_deg[1] - outer_deg[0]) * u[:, 1 + n_lights:1 + 2 * n_lights])
    inner = outer * (1.0 - (softness[0] + (softness[1] - softness[0]) * u[:, 1 + 2 * n_lights:]))
    return intensity, np.cos(outer), np.cos(inner)


def orbit_views(seed: int, sample_ids, n_cams: int, poi, radius=(0.4, 0.6), elevation_deg=(20.0, 70.0)):
    """CameraRandomizer, Orbit mode (Sec. 4.3.1): every camera at a radius and elevation uniform in
    the ranges and a uniform azimuth about the point of interest, looking at it.  Returns
    camera-from-world matrices [B * n_cams, 3, 4] and their samples [B * n_cams]."""
    ids = np.asarray(sample_ids, dtype=np.int64).reshape(-1)
    u = uniform(seed, STREAM_ORBIT, ids, 3 * n_cams).reshape(len(ids), n_cams, 3)
    r = radius[0] + (radius[1] - radius[0]) * u[..., 0]
    el = np.radians(elevation_deg[0] + (elevation_deg[1] - elevation_deg[0]) * u[..., 1])
    az = 2.0 * math.pi * u[..., 2]
    poi = np.asarray(poi, np.float64)
    eye = poi + r[..., None] * np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], -1)
    eye = eye.reshape(-1, 3)
    views = view_matrix(look_at(eye, np.broadcast_to(poi, eye.shape)), eye)
    return views, np.repeat(np.arange(len(ids)), n_cams).astype(np.int32)


def spot_shadow_cameras(pos, axis, cos_outer, res: int, near: float = 0.05, bias: float = 0.004,
                        margin: float = 1.1):
    """A perspective shadow camera per spot light: at the light, looking along its axis, with a
    square field of view of `margin` times the outer cone.  Returns views [..., 3, 4] and
    intrinsics [..., 6] (fx, fy, cx, cy, near, bias)."""
    pos, axis = np.asarray(pos, np.float64), np.asarray(axis, np.float64)
    up = np.where(np.abs(axis[..., 2:3]) > 0.99, np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]))
    f = axis / np.linalg.norm(axis, axis=-1, keepdims=True)
    r = np.cross(f, up)
    r /= np.linalg.norm(r, axis=-1, keepdims=True)
    R = np.stack([r, np.cross(r, f), -f], axis=-2)
    half = np.minimum(np.arccos(np.clip(cos_outer, -1.0, 1.0)) * margin, np.radians(80.0))
    fx = 0.5 * res / np.tan(half)
    intr = np.stack([fx, fx, np.full_like(fx, 0.5 * res), np.full_like(fx, 0.5 * res), np.full_like(fx, near),
                     np.full_like(fx, bias), np.zeros_like(fx)], -1)
    return view_matrix(R, pos), intr


# the face looking down first: lights hang above the scene, and the lookup tries faces in order
CUBE_FACES = np.array([[0, 0, -1], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1]], np.float64)


def point_shadow_cameras(pos, res: int, near: float = 0.02, bias: float = 0.004):
    """Six cube-face shadow cameras per point light (looking along -z, +x, -x, +y, -y, +z with
    90 deg fields of view).  pos [..., 3] -> views [..., 6, 3, 4], intrinsics [..., 6, 7]."""
    pos = np.asarray(pos, np.float64)
    views, intr = [], []
    for d in CUBE_FACES:
        up = np.array([0.0, 1.0, 0.0]) if abs(d[2]) > 0 else np.array([0.0, 0.0, 1.0])
        f = np.broadcast_to(d, pos.shape)
        r = np.cross(f, up)
        r = r / np.linalg.norm(r, axis=-1, keepdims=True)
        R = np.stack([r, np.cross(r, f), -f], axis=-2)
        views.append(view_matrix(R, pos))
        intr.append(np.broadcast_to(np.array([0.5 * res, 0.5 * res, 0.5 * res, 0.5 * res, near, bias, 0.0]),
                                    pos.shape[:-1] + (7,)))
    return np.stack(views, axis=-3), np.stack(intr, axis=-2)


def directional_shadow_camera(direction, target, half_extent: float, res: int, distance: float = 5.0,
                              near: float = 0.05, bias: float = 0.01):
    """An orthographic shadow camera for a directional light travelling along `direction`: placed
    `distance` back from `target` and looking along the light, its square map covering
    +-half_extent metres.  Returns the view [3, 4] and intrinsics [7]."""
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    up = np.array([0.0, 1.0, 0.0]) if abs(d[2]) > 0.99 else np.array([0.0, 0.0, 1.0])
    r = np.cross(d, up)
    r /= np.linalg.norm(r)
    R = np.stack([r, np.cross(r, d), -d])
    eye = np.asarray(target, np.float64) - distance * d
    f = 0.5 * res / half_extent
    return view_matrix(R, eye), np.array([f, f, 0.5 * res, 0.5 * res, near, bias, 1.0])


# the block's six calibrated face colours (HSV): red, orange, yellow, green, blue, purple
BLOCK_HSV = np.array([[0.00, 0.85, 0.80], [0.08, 0.85, 0.85], [0.15, 0.80, 0.85],
                      [0.33, 0.70, 0.60], [0.60, 0.75, 0.70], [0.78, 0.60, 0.60]])
N_SPOTS = 3


def benchmark_batch(seed: int, sample_ids, res: int = 200, n_cams: int = 3, orbit: bool = False,
                    grading: bool = True, meshes=None, shadow_res: int = 0, post: bool = False) -> Batch:
    """The hand scene configured like the paper's benchmark (Sec. 5): three spot lights placed by
    LightSetup about the block with LightRandomizer levels and cones, FixedHue materials (with
    emission) for the block's faces, the material randomizer for the hand and the table, camera
    jitter (or orbit), post-processing grading; with `shadow_res` > 0 every spot light casts
    shadows from a shadow map of that side; with `post` ambient occlusion and bloom too."""
    b = hand_batch(seed, sample_ids, res=res, n_cams=n_cams, meshes=meshes, grading=grading)
    ids = b.sample_ids
    B = len(ids)
    pos, axis = light_setup(seed, ids, N_SPOTS, BLOCK_CENTRE)
    inten, cos_o, cos_i = light_levels(seed, ids, N_SPOTS)
    light = np.zeros((B, MAX_LIGHTS, 4))
    light[:, :N_SPOTS, :3] = pos
    light[:, :N_SPOTS, 3] = inten
    spot = np.zeros((B, MAX_LIGHTS, 5))
    spot[:, :N_SPOTS, :3] = axis
    spot[:, :N_SPOTS, 3] = cos_o
    spot[:, :N_SPOTS, 4] = cos_i
    meta = np.tile([[N_SPOTS, LIGHT_SPOT]], (B, 1))
    mat = b.material.astype(np.float64).copy()
    albedo, ks, alpha, emis = fixed_hue_materials(seed, ids, BLOCK_HSV)
    mat[:, 1:7, :3], mat[:, 1:7, 3], mat[:, 1:7, 4] = albedo, ks, alpha
    emission = np.zeros((B, MAX_MATERIALS))
    emission[:, 1:7] = emis
    kw = dict(light=light.astype(np.float32), light_meta=meta.astype(np.int32),
              light_spot=spot.astype(np.float32), material=mat.astype(np.float32),
              emission=emission.astype(np.float32))
    if post:
        kw.update(post=post_params(seed, ids))
    if orbit:
        views, owner = orbit_views(seed, ids, n_cams, BLOCK_CENTRE)
        kw.update(cam_view=views.astype(np.float32), cam_sample=owner)
    if shadow_res > 0:
        sv, si = spot_shadow_cameras(pos, axis, cos_o, shadow_res)
        shadow_view = np.zeros((B, MAX_LIGHTS, 1, 3, 4))
        shadow_intr = np.zeros((B, MAX_LIGHTS, 1, 7))
        shadow_view[:, :N_SPOTS, 0], shadow_intr[:, :N_SPOTS, 0] = sv, si
        kw.update(shadow_view=shadow_view.astype(np.float32), shadow_intr=shadow_intr.astype(np.float32),
                  shadow_res=int(shadow_res), shadow_faces=1)
    return b.with_params(**kw)


# --------------------------------------------------------------------------
# Uneven workload: 1..156 capsule links per scene on a random tree
# --------------------------------------------------------------------------
UNEVEN_RES = (64, 128, 200, 256, 512)


def uneven_layout(seed: int, sample_ids):
    """Per scene: target triangle count (log-uniform [1k, 50k]) -> links, resolution, cameras."""
    ids = np.asarray(sample_ids, dtype=np.int64).reshape(-1)
    u = uniform(seed, STREAM_SCENE, ids, 3)
    T = np.exp(math.log(1000.0) + u[:, 0] * (math.log(50000.0) - math.log(1000.0)))
    n_links = np.maximum(1, np.rint((T - 14.0) / 320.0)).astype(np.int64)
    res = np.asarray(UNEVEN_RES)[np.minimum((u[:, 1] * len(UNEVEN_RES)).astype(np.int64), len(UNEVEN_RES) - 1)]
    cams = 1 + np.minimum((u[:, 2] * 3).astype(np.int64), 2)
    return n_links, res, cams


def uneven_batch(seed: int, sample_ids, meshes=None) -> Batch:
    ids = np.asarray(sample_ids, dtype=np.int64).reshape(-1)
    B = len(ids)
    meshes = meshes if meshes is not None else hand_meshes(0)
    radius, length = link_dims(0)
    n_links, res, cams = uneven_layout(seed, ids)
    max_links = int(n_links.max()) if B else 0
    ua = uniform(seed, STREAM_JOINTS, ids, 2 * max(max_links, 1))
    ub = uniform(seed, STREAM_BLOCK, ids, 4)
    inst_mesh, pose, seg, mbase, counts = [], [], [], [], []
    for s in range(B):
        n = int(n_links[s])
        T = np.zeros((n, 4, 4))
        for i in range(n):
            mesh_i = i % N_LINKS
            parent = -1 if i == 0 else int(ua[s, 2 * i] * i)
            if parent < 0:
                off, P = np.zeros(3), _hom(np.eye(3), HAND_BASE)
            else:
                off, P = np.array([length[parent % N_LINKS], 0.0, 0.0]), T[parent]
            axis = "y" if i % 2 == 0 else "z"
            ang = math.radians(60.0) * (2.0 * ua[s, 2 * i + 1] - 1.0)
            T[i] = P @ _hom(_rot(axis, np.array(ang)), off)
            inst_mesh.append(2 + mesh_i)
            seg.append(3 + i)
            mbase.append(7 + (i % 25))
        block = _hom(_rot("z", np.array(2.0 * math.pi * ub[s, 0])), BLOCK_CENTRE + 0.01 * (2.0 * ub[s, 1:4] - 1.0))
        pose_s = [np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1), block[:3, :]] + [t[:3, :] for t in T]
        pose += pose_s
        inst_mesh[len(inst_mesh) - n:len(inst_mesh) - n] = [0, 1]
        seg[len(seg) - n:len(seg) - n] = [1, 2]
        mbase[len(mbase) - n:len(mbase) - n] = [0, 1]
        counts.append(n + 2)
    views, owner = _rig_views(seed, ids, cams)
    intr, wh = _square_intrinsics(res[owner], FOVY_DEG)
    light, meta = _lights(seed, ids)
    ev, ambient, background = _post(seed, ids)
    return Batch(
        meshes=meshes,
        inst_offset=np.concatenate([[0], np.cumsum(counts)]).astype(np.int32),
        inst_mesh=np.asarray(inst_mesh, np.uint32),
        inst_pose=np.asarray(pose).astype(np.float32),
        inst_seg=np.asarray(seg, np.uint8),
        inst_mat_base=np.asarray(mbase, np.int16),
        cam_offset=np.concatenate([[0], np.cumsum(cams)]).astype(np.int32),
        cam_sample=owner,
        cam_view=views.astype(np.float32),
        cam_intr=intr.astype(np.float32),
        cam_wh=wh,
        img_offset=_img_offsets(wh),
        light=light, light_meta=meta,
        material=_materials(seed, ids),
        exposure_ev=ev, ambient=ambient, background=background,
        sample_ids=ids,
    )


# --------------------------------------------------------------------------
# Differentiation workload: target parameters perturbed from the base ones
# --------------------------------------------------------------------------
def perturb_params(batch: Batch, seed: int):
    """(material, light, exposure_ev) perturbed: albedo +-0.2 (clamped to [0,1]),
    light position +-5 cm, intensity x U(0.7, 1.3), exposure +-0.5 EV."""
    ids = batch.sample_ids if len(batch.sample_ids) else np.arange(batch.n_samples)
    B = batch.n_samples
    u = uniform(seed, STREAM_TARGET, ids, 3 * MAX_MATERIALS + 4 * MAX_LIGHTS + 1)
    mat = batch.material.astype(np.float64).copy()
    mat[..., :3] = np.clip(mat[..., :3] + 0.2 * (2.0 * u[:, :3 * MAX_MATERIALS].reshape(B, MAX_MATERIALS, 3) - 1.0), 0.0, 1.0)
    v = u[:, 3 * MAX_MATERIALS:3 * MAX_MATERIALS + 4 * MAX_LIGHTS].reshape(B, MAX_LIGHTS, 4)
    light = batch.light.astype(np.float64).copy()
    active = np.arange(MAX_LIGHTS)[None, :] < batch.light_meta[:, :1]
    light[..., :3] += np.where(active[..., None], 0.05 * (2.0 * v[..., :3] - 1.0), 0.0)
    light[..., 3] *= np.where(active, 0.7 + 0.6 * v[..., 3], 1.0)
    ev = batch.exposure_ev.astype(np.float64) + (u[:, -1] - 0.5)
    return mat.astype(np.float32), light.astype(np.float32), ev.astype(np.float32)


# --------------------------------------------------------------------------
# Serving workload: Poisson request stream
# --------------------------------------------------------------------------
SERVE_RES = (64, 128, 200, 256)


@dataclass
class Request:
    rid: int
    arrival_s: float
    n_samples: int
    res: int
    n_cams: int
    first_sample: int


def poisson_requests(seed: int, rate_hz: float, duration_s: float, max_samples: int = 64) -> List[Request]:
    """Arrivals of a Poisson process (exponential gaps); request size U{1..max_samples},
    resolution U(SERVE_RES), cameras U{1..3}; sample ids are consecutive and never reused."""
    n_max = int(rate_hz * duration_s * 1.5 + 64)
    u = uniform(seed, STREAM_REQUESTS, np.arange(n_max), 4)
    gaps = -np.log(u[:, 0]) / rate_hz
    t = np.cumsum(gaps)
    reqs, first = [], 0
    for i in range(n_max):
        if t[i] > duration_s:
            break
        n = 1 + min(int(u[i, 1] * max_samples), max_samples - 1)
        res = SERVE_RES[min(int(u[i, 2] * len(SERVE_RES)), len(SERVE_RES) - 1)]
        cams = 1 + min(int(u[i, 3] * 3), 2)
        reqs.append(Request(i, float(t[i]), n, res, cams, first))
        first += n
    return reqs


def request_batch(seed: int, req: Request, meshes=None) -> Batch:
    ids = np.arange(req.first_sample, req.first_sample + req.n_samples)
    return hand_batch(seed, ids, res=req.res, n_cams=req.n_cams, meshes=meshes)
