"""ctypes wrapper of the plain CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this module.  It compiles ``orrb_oracle.c`` with gcc (fp32 forward with no
FMA contraction, fp64 shading adjoint) and runs it over images with a pool of
host threads; the C code releases nothing shared, so images are independent.

Inputs are the numpy arrays of a ``scenegen.Batch``; outputs are numpy arrays
laid out like the renderer's channels (flat over all pixels of all images).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "orrb_oracle.c")
HDR = os.path.join(HERE, "orrb_oracle.h")
LIB = os.path.join(HERE, "_build", "liborrb_oracle.so")
CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle if the shared object is missing or older than its sources."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    stale = force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if stale:
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Meshes(C.Structure):
    _fields_ = [("n_meshes", C.c_int32), ("vert_offset", C.c_void_p), ("tri_offset", C.c_void_p),
                ("pos", C.c_void_p), ("nrm", C.c_void_p), ("idx", C.c_void_p), ("tri_mat", C.c_void_p)]


_BATCH_ARRAYS = ("inst_offset", "inst_mesh", "inst_pose", "inst_seg", "inst_mat_base",
                 "cam_offset", "cam_sample", "cam_view", "cam_intr", "cam_wh", "img_offset",
                 "light", "light_meta", "material", "exposure_ev", "ambient", "background", "grading", "light_spot",
                 "emission", "shadow_view", "shadow_intr", "shadow_map")


class _Batch(C.Structure):
    _fields_ = [("n_samples", C.c_int32)] + [(n, C.c_void_p) for n in _BATCH_ARRAYS] + [("shadow_res", C.c_int32),
                                                                                        ("shadow_faces", C.c_int32),
                                                                                        ("post", C.c_void_p)]


class _Outputs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in (
        "rgb", "depth", "normal", "seg", "rgb_linear", "gb_pos", "gb_nrm", "gb_mat", "prim", "depth2", "counters",
        "tracker")] + [("tracker_stride", C.c_int32), ("flops", C.c_void_p), ("rgb_final", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_render.argtypes = [C.POINTER(_Meshes), C.POINTER(_Batch), C.c_int32, C.c_int32, C.POINTER(_Outputs)]
            L.orc_render.restype = C.c_int
            L.orc_raster_fixed.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_raster_fixed.restype = C.c_int
            L.orc_f32_to_f16.argtypes = [C.c_float]
            L.orc_post_image.argtypes = [C.c_int32, C.c_int32] + [C.c_void_p] * 5
            L.orc_post_image.restype = C.c_int
            L.orc_f32_to_f16.restype = C.c_uint16
            L.orc_shade_f64.argtypes = [C.POINTER(_Batch), C.c_int32, C.c_int32] + [C.c_void_p] * 9
            L.orc_shade_f64.restype = None
            L.orc_shade_backward_f64.argtypes = [C.POINTER(_Batch), C.c_int32, C.c_int32] + [C.c_void_p] * 13
            L.orc_shade_backward_f64.restype = None
            L.orc_grade_f64.argtypes = [C.POINTER(_Batch), C.c_int32, C.c_int32] + [C.c_void_p] * 3
            L.orc_grade_f64.restype = None
            L.orc_grade_backward_f64.argtypes = [C.POINTER(_Batch), C.c_int32, C.c_int32] + [C.c_void_p] * 5
            L.orc_grade_backward_f64.restype = None
            L.orc_render_shadow_maps.argtypes = [C.POINTER(_Meshes), C.POINTER(_Batch), C.c_int32, C.c_int32,
                                                 C.c_void_p]
            L.orc_render_shadow_maps.restype = C.c_int
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _opt(batch, name):
    """An optional float32 parameter array of the batch, or None."""
    a = getattr(batch, name, None)
    return None if a is None else _c(a, np.float32)


class _Pinned:
    """Keeps the contiguous numpy copies alive while C holds their pointers."""

    def __init__(self, batch):
        ms = batch.meshes
        self.vo = _c(np.concatenate([[0], np.cumsum([m.n_verts for m in ms])]), np.int32)
        self.to = _c(np.concatenate([[0], np.cumsum([m.n_tris for m in ms])]), np.int32)
        self.pos = _c(np.concatenate([m.pos for m in ms]), np.float32)
        self.nrm = _c(np.concatenate([m.nrm for m in ms]), np.float32)
        self.idx = _c(np.concatenate([m.idx for m in ms]), np.uint32)
        self.tm = _c(np.concatenate([m.tri_mat for m in ms]), np.uint8)
        self.meshes = _Meshes(len(ms), _p(self.vo), _p(self.to), _p(self.pos), _p(self.nrm), _p(self.idx), _p(self.tm))
        self.arrs = dict(
            inst_offset=_c(batch.inst_offset, np.int32), inst_mesh=_c(batch.inst_mesh, np.uint32),
            inst_pose=_c(batch.inst_pose, np.float32), inst_seg=_c(batch.inst_seg, np.uint8),
            inst_mat_base=_c(batch.inst_mat_base, np.int16), cam_offset=_c(batch.cam_offset, np.int32),
            cam_sample=_c(batch.cam_sample, np.int32), cam_view=_c(batch.cam_view, np.float32),
            cam_intr=_c(batch.cam_intr, np.float32), cam_wh=_c(batch.cam_wh, np.int32),
            img_offset=_c(batch.img_offset, np.int64), light=_c(batch.light, np.float32),
            light_meta=_c(batch.light_meta, np.int32), material=_c(batch.material, np.float32),
            exposure_ev=_c(batch.exposure_ev, np.float32), ambient=_c(batch.ambient, np.float32),
            background=_c(batch.background, np.float32),
            grading=_opt(batch, "grading"), light_spot=_opt(batch, "light_spot"), emission=_opt(batch, "emission"),
            shadow_view=_opt(batch, "shadow_view"), shadow_intr=_opt(batch, "shadow_intr"), shadow_map=None)
        self.shadow_res = int(getattr(batch, "shadow_res", 0) or 0)
        self.shadow_faces = int(getattr(batch, "shadow_faces", 1) or 1)
        self.post = _opt(batch, "post")
        self.batch = _Batch(batch.n_samples, *[_p(self.arrs[n]) for n in _BATCH_ARRAYS], self.shadow_res,
                            self.shadow_faces, _p(self.post))

    def set_shadow_maps(self, maps):
        """Point the lookups of step 16 at `maps` ([S, 4, F, R, R] float32, kept alive here)."""
        self.arrs["shadow_map"] = maps
        self.batch.shadow_map = _p(maps)


def _chunks(n_cams: int, threads: int):
    k = max(1, min(n_cams, threads * 4))
    edges = np.linspace(0, n_cams, k + 1).astype(int)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def shadow_maps(batch, threads: int | None = None, pin=None):
    """The shadow maps of step 15, [n_samples, 4, F, R, R] float32 (zero for faces without shadow), or None."""
    pin = pin or _Pinned(batch)
    R = pin.shadow_res
    if R <= 0 or pin.arrs["shadow_view"] is None or pin.arrs["shadow_intr"] is None:
        return None
    maps = np.zeros((batch.n_samples, 4, pin.shadow_faces, R, R), np.float32)
    threads = threads or default_threads()
    L = lib()

    def run(rng):
        if L.orc_render_shadow_maps(C.byref(pin.meshes), C.byref(pin.batch), rng[0], rng[1], _p(maps)) != 0:
            raise MemoryError("oracle: allocation failed")

    chunks = _chunks(batch.n_samples, threads)
    if threads == 1 or len(chunks) == 1:
        for c in chunks:
            run(c)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, chunks))
    return maps


def render(batch, threads: int | None = None, gbuffer: bool = False, debug: bool = False, cams=None,
           tracker: bool = False, flops: bool = False):
    """Oracle render of a batch.  Returns a dict of numpy channel arrays.

    `cams`: optional (begin, end) camera range; pixels of other images stay zero.
    `tracker`: also the per (camera, instance) rows [n_cams, max instances per sample, 8] of step 14.
    A batch with shadow cameras also returns its shadow maps (step 15) as "shadow_map".
    `flops`: also the number of fp32 operations of steps 9-13 and 16 (the oracle's own per-block
    tallies: per visible pixel what depends on the pixel, once per image what depends on the image
    only), as "flops".
    """
    L = lib()
    pin = _Pinned(batch)
    maps = shadow_maps(batch, threads, pin)
    if maps is not None:
        pin.set_shadow_maps(maps)
    N = batch.total_pixels
    out = dict(rgb=np.zeros((N, 3), np.uint8), depth=np.zeros(N, np.float32), normal=np.zeros((N, 3), np.uint16),
               seg=np.zeros(N, np.uint8), rgb_linear=np.zeros((N, 3), np.float32),
               rgb_final=np.zeros((N, 3), np.float32))
    if gbuffer:
        out.update(gb_pos=np.zeros((N, 3), np.float32), gb_nrm=np.zeros((N, 3), np.float32),
                   gb_mat=np.zeros(N, np.int32))
    if debug:
        out.update(prim=np.zeros(N, np.int64), depth2=np.zeros(N, np.float32))
    stride = int(np.diff(batch.inst_offset).max()) if batch.n_samples else 0
    if tracker:
        out["tracker"] = np.zeros((batch.n_cams, stride, 8), np.int32)
    threads = threads or default_threads()
    c0, c1 = cams if cams is not None else (0, batch.n_cams)
    chunks = [(a + c0, b + c0) for a, b in _chunks(c1 - c0, threads)]
    counters = np.zeros((len(chunks), 4), np.int64)
    nflops = np.zeros((len(chunks), 1), np.int64)

    def run(i):
        o = _Outputs(*[_p(out.get(n)) for n, _ in _Outputs._fields_[:-5]], _p(counters[i]), _p(out.get("tracker")),
                     stride, _p(nflops[i]) if flops else None, _p(out["rgb_final"]))
        rc = L.orc_render(C.byref(pin.meshes), C.byref(pin.batch), chunks[i][0], chunks[i][1], C.byref(o))
        if rc != 0:
            raise MemoryError("oracle: allocation failed")

    if threads == 1 or len(chunks) == 1:
        for i in range(len(chunks)):
            run(i)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, range(len(chunks))))
    out["counters"] = counters.sum(0)
    if flops:
        out["flops"] = int(nflops.sum())
    if maps is not None:
        out["shadow_map"] = maps
    return out


def post_image(W: int, H: int, intr, q, col, depth, normal):
    """Step 17 on one W x H image: returns the post-processed colour [W*H, 3] float32 of the linear
    colour `col` [W*H, 3], given the depth channel [W*H], the normal channel's binary16 bits
    [W*H, 3], the camera's (fx, fy, cx, cy, near, type) and q = (AO intensity, bloom intensity,
    bloom radius in pixels, 0)."""
    c = _c(col, np.float32).reshape(-1, 3).copy()
    d = _c(depth, np.float32).reshape(-1)
    n = _c(normal, np.uint16).reshape(-1, 3)
    i = _c(intr, np.float32).reshape(6)
    qq = _c(q, np.float32).reshape(4)
    assert len(c) == len(d) == len(n) == W * H
    if lib().orc_post_image(W, H, _p(i), _p(qq), _p(c), _p(d), _p(n)) != 0:
        raise MemoryError("oracle: allocation failed")
    return c


def raster_fixed(W: int, H: int, X, Y, iw, ortho: bool = False):
    """Coverage/visibility of snapped triangles.

    Returns (key [H,W] int64, depth [H,W] f32, fragment count [H,W] int32)."""
    X = _c(X, np.int32).reshape(-1, 3)
    Y = _c(Y, np.int32).reshape(-1, 3)
    iw = _c(iw, np.float32).reshape(-1, 3)
    prim = np.zeros(W * H, np.int64)
    depth = np.zeros(W * H, np.float32)
    count = np.zeros(W * H, np.int32)
    rc = lib().orc_raster_fixed(W, H, len(X), _p(X), _p(Y), _p(iw), int(ortho), _p(prim), _p(depth), _p(count))
    assert rc == 0
    return prim.reshape(H, W), depth.reshape(H, W), count.reshape(H, W)


def f32_to_f16_bits(x) -> np.ndarray:
    L = lib()
    x = np.asarray(x, np.float32).reshape(-1)
    return np.array([L.orc_f32_to_f16(float(v)) for v in x], np.uint16)


def _params64(batch, material=None, light=None, exposure_ev=None, ambient=None, emission=None):
    m = _c(batch.material if material is None else material, np.float64)
    l = _c(batch.light if light is None else light, np.float64)
    e = _c(batch.exposure_ev if exposure_ev is None else exposure_ev, np.float64)
    a = _c(batch.ambient if ambient is None else ambient, np.float64)
    em = getattr(batch, "emission", None) if emission is None else emission
    return m, l, e, a, None if em is None else _c(em, np.float64)


def shade_f64(batch, gb_pos, gb_nrm, gb_mat, material=None, light=None, exposure_ev=None, ambient=None,
              emission=None):
    """fp64 shading of a fixed G-buffer (the function finite differences are taken of)."""
    pin = _Pinned(batch)
    m, l, e, a, em = _params64(batch, material, light, exposure_ev, ambient, emission)
    gp, gn, gm = _c(gb_pos, np.float32), _c(gb_nrm, np.float32), _c(gb_mat, np.int32)
    rgb = np.zeros((batch.total_pixels, 3), np.float64)
    lib().orc_shade_f64(C.byref(pin.batch), 0, batch.n_cams, _p(gp), _p(gn), _p(gm), _p(m), _p(l), _p(e), _p(a),
                        _p(em), _p(rgb))
    return rgb


def shade_backward_f64(batch, gb_pos, gb_nrm, gb_mat, d_rgb, material=None, light=None, exposure_ev=None,
                       ambient=None, emission=None, return_emission=False):
    """fp64 adjoint: (d_material [S,32,4], d_light [S,4,4], d_ev [S]), plus d_emission [S,32] last
    when `return_emission`."""
    pin = _Pinned(batch)
    m, l, e, a, em = _params64(batch, material, light, exposure_ev, ambient, emission)
    gp, gn, gm = _c(gb_pos, np.float32), _c(gb_nrm, np.float32), _c(gb_mat, np.int32)
    g = _c(d_rgb, np.float64)
    S = batch.n_samples
    dm = np.zeros((S, 32, 4), np.float64)
    dl = np.zeros((S, 4, 4), np.float64)
    de = np.zeros(S, np.float64)
    dem = np.zeros((S, 32), np.float64)
    lib().orc_shade_backward_f64(C.byref(pin.batch), 0, batch.n_cams, _p(gp), _p(gn), _p(gm), _p(m), _p(l), _p(e),
                                 _p(a), _p(em), _p(g), _p(dm), _p(dl), _p(de), _p(dem))
    return (dm, dl, de, dem) if return_emission else (dm, dl, de)


def grade_f64(batch, rgb_in, grading=None):
    """Step 13 in fp64: the graded colour [N, 3] of the linear colour `rgb_in` [N, 3] (grading
    parameters [S, 8], default the batch's)."""
    pin = _Pinned(batch)
    g = _c(batch.grading if grading is None else grading, np.float64)
    x = _c(rgb_in, np.float64)
    out = np.zeros((batch.total_pixels, 3), np.float64)
    lib().orc_grade_f64(C.byref(pin.batch), 0, batch.n_cams, _p(g), _p(x), _p(out))
    return out


def graded_shade_f64(batch, gb_pos, gb_nrm, gb_mat, grading=None, **params):
    """The graded colour of a fixed G-buffer in fp64 (shading of step 10, then step 13)."""
    return grade_f64(batch, shade_f64(batch, gb_pos, gb_nrm, gb_mat, **params), grading)


def graded_backward_f64(batch, gb_pos, gb_nrm, gb_mat, d_graded, grading=None, **params):
    """fp64 adjoint of a loss on the graded colour: (d_material, d_light, d_ev, d_grading [S, 8])."""
    pin = _Pinned(batch)
    g = _c(batch.grading if grading is None else grading, np.float64)
    lin = _c(shade_f64(batch, gb_pos, gb_nrm, gb_mat, **params), np.float64)
    dO = _c(d_graded, np.float64)
    d_lin = np.zeros((batch.total_pixels, 3), np.float64)
    dg = np.zeros((batch.n_samples, 8), np.float64)
    lib().orc_grade_backward_f64(C.byref(pin.batch), 0, batch.n_cams, _p(g), _p(lin), _p(dO), _p(d_lin), _p(dg))
    dm, dl, de = shade_backward_f64(batch, gb_pos, gb_nrm, gb_mat, d_lin, **params)
    return dm, dl, de, dg
