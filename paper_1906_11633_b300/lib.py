"""ctypes binding of liborrb.so: the C-ABI of include/orrb.h, same names, marshalling only.

Loading fails loudly if the in-tree library is missing: there is no fallback
path.  Build it with ``python -m paper_1906_11633_b300.build``.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liborrb.so")

ORRB_OK = 0
ORRB_ERR_INVALID_ARG = 1   # status codes (ORRB_ERR_* of include/orrb.h)
ORRB_ERR_WORKSPACE = 2
ORRB_ERR_CUDA = 3
ORRB_ERR_TIMEOUT = 4
ORRB_ERR_NOT_FOUND = 5
ORRB_ERR_UNSUPPORTED = 6
ORRB_ERR_DEVICE = 7
ORRB_MODE_FUSED = 0
ORRB_MODE_PLAIN = 1
ORRB_MODE_STAGED = 2
ORRB_MAX_LIGHTS = 4
ORRB_MAX_MATERIALS = 32
ORRB_GBUFFER_PLANES = 7
DEFAULT_TILE_W = 256    # the library's defaults for a zero orrb_config field
DEFAULT_TILE_H = 2
DEFAULT_THREADS = 512
ORRB_DEV_BAD_CAMERA = 0x1     # device status word bits (ORRB_DEV_* of include/orrb.h)
ORRB_DEV_BAD_INSTANCE = 0x2
ORRB_DEV_TOO_MANY_TRIS = 0x4
ORRB_DEV_BAD_MATERIAL = 0x8
ORRB_DEV_BAD_LIGHTS = 0x10
ORRB_DEV_DROPPED = 0x20
ORRB_DEV_TIMEOUT = 0x40
DEV_BITS = {0x1: "bad camera", 0x2: "bad instance", 0x4: "too many triangles", 0x8: "bad material",
            0x10: "bad lights", 0x20: "triangle dropped by guard band", 0x40: "a bounded wait between CTAs gave up"}

EXPORTS = ["orrb_create", "orrb_destroy", "orrb_status_string", "orrb_last_error", "orrb_mesh_arena_size",
           "orrb_upload_meshes", "orrb_release_meshes", "orrb_workspace_size", "orrb_render_batch",
           "orrb_read_status", "orrb_backward_workspace_size", "orrb_shade_backward", "orrb_render_batch_noalloc"]


class orrb_mesh_desc(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("nrm", C.c_void_p), ("n_verts", C.c_int32), ("idx", C.c_void_p),
                ("tri_mat", C.c_void_p), ("n_tris", C.c_int32)]


class orrb_batch_shape(C.Structure):
    _fields_ = [("n_samples", C.c_int32), ("n_cams", C.c_int32), ("max_tris_per_sample", C.c_int32),
                ("max_inst_per_sample", C.c_int32), ("max_cams_per_sample", C.c_int32), ("max_width", C.c_int32),
                ("max_height", C.c_int32), ("total_pixels", C.c_int64), ("shadow_res", C.c_int32),
                ("shadow_faces", C.c_int32), ("post_effects", C.c_int32)]


class orrb_batch_desc(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in (
        "inst_offset", "inst_mesh", "inst_pose", "inst_seg", "inst_mat_base", "cam_offset", "cam_sample", "cam_view",
        "cam_intr", "cam_wh", "img_offset", "light", "light_meta", "material", "exposure_ev", "ambient", "background", "grading",
        "light_spot", "emission", "shadow_view", "shadow_intr", "post")]


class orrb_outputs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("rgb", "depth", "normal", "seg", "rgb_linear", "gbuffer", "tracker",
                                          "shadow_map", "rgb_graded")]


class orrb_config(C.Structure):
    _fields_ = [("mode", C.c_int32), ("tile_w", C.c_int32), ("tile_h", C.c_int32), ("threads", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("reserved", C.c_int32), ("wait_cycles", C.c_int64)]


class orrb_param_grads(C.Structure):
    _fields_ = [("d_material", C.c_void_p), ("d_light", C.c_void_p), ("d_exposure", C.c_void_p),
                ("d_emission", C.c_void_p), ("d_grading", C.c_void_p)]


class OrrbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"orrb status {status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load():
    """Load liborrb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: build it with `python -m paper_1906_11633_b300.build`")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        sig = {
            "orrb_create": ([C.c_int, P(C.c_void_p)], C.c_int32),
            "orrb_destroy": ([C.c_void_p], None),
            "orrb_status_string": ([C.c_int32], C.c_char_p),
            "orrb_last_error": ([C.c_void_p, C.c_char_p, C.c_size_t], C.c_int32),
            "orrb_mesh_arena_size": ([P(orrb_mesh_desc), C.c_int32, P(C.c_size_t)], C.c_int32),
            "orrb_upload_meshes": ([C.c_void_p, P(orrb_mesh_desc), C.c_int32, C.c_void_p, C.c_size_t, C.c_void_p],
                                   C.c_int32),
            "orrb_release_meshes": ([C.c_void_p], C.c_int32),
            "orrb_workspace_size": ([C.c_void_p, P(orrb_batch_shape), P(orrb_config), P(C.c_size_t)], C.c_int32),
            "orrb_render_batch": ([C.c_void_p, P(orrb_batch_shape), P(orrb_batch_desc), P(orrb_outputs),
                                   P(orrb_config), C.c_void_p, C.c_size_t, C.c_void_p], C.c_int32),
            "orrb_read_status": ([C.c_void_p, C.c_void_p, C.c_void_p, P(C.c_uint32)], C.c_int32),
            "orrb_render_batch_noalloc": ([C.c_void_p, P(orrb_batch_shape), P(orrb_batch_desc), P(orrb_outputs),
                                           P(orrb_config), C.c_void_p, C.c_void_p], C.c_int32),
            "orrb_backward_workspace_size": ([C.c_void_p, P(orrb_batch_shape), P(C.c_size_t)], C.c_int32),
            "orrb_shade_backward": ([C.c_void_p, P(orrb_batch_shape), P(orrb_batch_desc), C.c_void_p, C.c_void_p,
                                     P(orrb_param_grads), C.c_void_p, C.c_size_t, C.c_void_p], C.c_int32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def last_error(ctx) -> str:
    buf = C.create_string_buffer(512)
    load().orrb_last_error(ctx, buf, len(buf))
    return buf.value.decode(errors="replace")


def check(status: int, ctx=None) -> None:
    if status != ORRB_OK:
        L = load()
        msg = L.orrb_status_string(status).decode()
        if ctx is not None:
            detail = last_error(ctx)
            if detail:
                msg += ": " + detail
        raise OrrbError(status, msg)


# thin wrappers with the C names -------------------------------------------------
def orrb_create(device: int = 0):
    ctx = C.c_void_p()
    check(load().orrb_create(device, C.byref(ctx)))
    return ctx


def orrb_destroy(ctx) -> None:
    load().orrb_destroy(ctx)


def orrb_mesh_arena_size(descs) -> int:
    arr = (orrb_mesh_desc * len(descs))(*descs)
    n = C.c_size_t()
    check(load().orrb_mesh_arena_size(arr, len(descs), C.byref(n)))
    return n.value


def orrb_upload_meshes(ctx, descs, arena_ptr: int, arena_bytes: int, stream: int) -> None:
    arr = (orrb_mesh_desc * len(descs))(*descs)
    check(load().orrb_upload_meshes(ctx, arr, len(descs), C.c_void_p(arena_ptr), arena_bytes, C.c_void_p(stream)), ctx)


def orrb_release_meshes(ctx) -> None:
    check(load().orrb_release_meshes(ctx), ctx)


def orrb_workspace_size(ctx, shape: orrb_batch_shape, cfg: orrb_config) -> int:
    n = C.c_size_t()
    check(load().orrb_workspace_size(ctx, C.byref(shape), C.byref(cfg), C.byref(n)), ctx)
    return n.value


def orrb_render_batch(ctx, shape, desc, outs, cfg, ws_ptr: int, ws_bytes: int, stream: int) -> None:
    check(load().orrb_render_batch(ctx, C.byref(shape), C.byref(desc), C.byref(outs), C.byref(cfg),
                                   C.c_void_p(ws_ptr), ws_bytes, C.c_void_p(stream)), ctx)


def orrb_render_batch_noalloc(ctx, shape, desc, outs, cfg, status_ptr, stream: int) -> None:
    """Render with the library's static scratch instead of a workspace (no device allocation)."""
    check(load().orrb_render_batch_noalloc(ctx, C.byref(shape), C.byref(desc), C.byref(outs), C.byref(cfg),
                                           C.c_void_p(status_ptr), C.c_void_p(stream)), ctx)


def orrb_read_status(ctx, ws_ptr: int, stream: int) -> int:
    v = C.c_uint32()
    check(load().orrb_read_status(ctx, C.c_void_p(ws_ptr), C.c_void_p(stream), C.byref(v)), ctx)
    return v.value


def orrb_backward_workspace_size(ctx, shape) -> int:
    n = C.c_size_t()
    check(load().orrb_backward_workspace_size(ctx, C.byref(shape), C.byref(n)), ctx)
    return n.value


def orrb_shade_backward(ctx, shape, desc, gbuffer_ptr: int, d_rgb_ptr: int, grads, ws_ptr: int, ws_bytes: int,
                        stream: int) -> None:
    check(load().orrb_shade_backward(ctx, C.byref(shape), C.byref(desc), C.c_void_p(gbuffer_ptr),
                                     C.c_void_p(d_rgb_ptr), C.byref(grads), C.c_void_p(ws_ptr), ws_bytes,
                                     C.c_void_p(stream)), ctx)
