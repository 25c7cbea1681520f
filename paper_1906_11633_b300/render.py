"""Torch-level helpers around the C-ABI: device buffers, output tensors, autograd.

PyTorch provides device memory and streams only; every step of rendering runs
in liborrb.so's kernels.  Typical use::

    r = Renderer(batch.meshes)                 # meshes resident once (Sec. 3, SSMS)
    db = r.upload(batch)                       # per-sample state + randomization params
    out = r.render(db)                         # dict of channel tensors (Sec. 4.4)
"""

from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from typing import Dict, Optional

import numpy as np
import torch

from . import lib as L

_DESC_FIELDS = [n for n, _ in L.orrb_batch_desc._fields_]
_DTYPES = dict(inst_offset=torch.int32, inst_mesh=torch.int32, inst_pose=torch.float32, inst_seg=torch.uint8,
               inst_mat_base=torch.int16, cam_offset=torch.int32, cam_sample=torch.int32, cam_view=torch.float32,
               cam_intr=torch.float32, cam_wh=torch.int32, img_offset=torch.int64, light=torch.float32,
               light_meta=torch.int32, material=torch.float32, exposure_ev=torch.float32, ambient=torch.float32,
               background=torch.float32, grading=torch.float32, light_spot=torch.float32, emission=torch.float32,
               shadow_view=torch.float32, shadow_intr=torch.float32, post=torch.float32)
_NP = {torch.int32: np.int32, torch.float32: np.float32, torch.uint8: np.uint8, torch.int16: np.int16,
       torch.int64: np.int64}


def batch_shape(batch) -> L.orrb_batch_shape:
    """Host-side shape of a scenegen.Batch."""
    tps = batch.tris_per_sample()
    return L.orrb_batch_shape(
        n_samples=batch.n_samples, n_cams=batch.n_cams,
        max_tris_per_sample=int(tps.max()) if len(tps) else 0,
        max_inst_per_sample=int(np.diff(batch.inst_offset).max()) if batch.n_samples else 0,
        max_cams_per_sample=int(np.diff(batch.cam_offset).max()) if batch.n_samples else 0,
        max_width=int(batch.cam_wh[:, 0].max()) if batch.n_cams else 1,
        max_height=int(batch.cam_wh[:, 1].max()) if batch.n_cams else 1,
        total_pixels=batch.total_pixels,
        shadow_res=int(getattr(batch, "shadow_res", 0) or 0) if getattr(batch, "shadow_view", None) is not None else 0,
        shadow_faces=int(getattr(batch, "shadow_faces", 1) or 1),
        post_effects=int(getattr(batch, "post", None) is not None))


@dataclass
class DeviceBatch:
    """A batch's arrays as device tensors plus the C descriptor that points at them."""
    shape: L.orrb_batch_shape
    tensors: Dict[str, torch.Tensor]
    desc: L.orrb_batch_desc = field(init=False)

    def __post_init__(self):
        # an optional array (grading, light_spot, emission, shadow cameras) that is absent or None passes
        # a null pointer
        self.desc = L.orrb_batch_desc(*[self.tensors[n].data_ptr() if self.tensors.get(n) is not None else None
                                        for n in _DESC_FIELDS])

    @property
    def total_pixels(self) -> int:
        return int(self.shape.total_pixels)

    @property
    def has_shadows(self) -> bool:
        return int(self.shape.shadow_res) > 0 and self.tensors.get("shadow_view") is not None \
            and self.tensors.get("shadow_intr") is not None

    def with_params(self, **kw) -> "DeviceBatch":
        t = dict(self.tensors)
        t.update(kw)
        return DeviceBatch(self.shape, t)


def host_arrays(batch) -> Dict[str, np.ndarray]:
    """The batch's arrays in the C layout, contiguous, as numpy (an optional array that is None is left out)."""
    return {n: np.ascontiguousarray(getattr(batch, n), dtype=_NP[_DTYPES[n]]) for n in _DESC_FIELDS
            if getattr(batch, n, None) is not None}


def _mesh_descs(meshes):
    keep, descs = [], []
    for m in meshes:
        pos = np.ascontiguousarray(m.pos, np.float32)
        nrm = np.ascontiguousarray(m.nrm, np.float32)
        idx = np.ascontiguousarray(m.idx, np.uint32)
        tm = np.ascontiguousarray(m.tri_mat, np.uint8)
        keep += [pos, nrm, idx, tm]
        descs.append(L.orrb_mesh_desc(pos.ctypes.data, nrm.ctypes.data, len(pos), idx.ctypes.data, tm.ctypes.data,
                                      len(idx)))
    return descs, keep


def config(mode: int = L.ORRB_MODE_FUSED, tile_w: int = 0, tile_h: int = 0, threads: int = 0,
           ctas_per_sm: int = 0, wait_cycles: int = 0) -> L.orrb_config:
    """Launch configuration; 0 picks each default (see orrb_config in include/orrb.h)."""
    return L.orrb_config(mode, tile_w, tile_h, threads, ctas_per_sm, 0, wait_cycles)


class Renderer:
    """Context + resident mesh arena on one GPU."""

    def __init__(self, meshes, device: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("Renderer needs a CUDA device; there is no CPU path")
        self.device = torch.device("cuda", device)
        self.ctx = L.orrb_create(device)
        descs, keep = _mesh_descs(meshes)
        n = L.orrb_mesh_arena_size(descs)
        self.arena = torch.empty(n, dtype=torch.uint8, device=self.device)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        L.orrb_upload_meshes(self.ctx, descs, self.arena.data_ptr(), n, stream)
        del keep
        self._ws: Optional[torch.Tensor] = None
        self._bws: Optional[torch.Tensor] = None

    def close(self):
        if self.ctx is not None:
            L.orrb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- batches --------------------------------------------------------------
    def upload(self, batch, pinned: bool = False, non_blocking: bool = False) -> DeviceBatch:
        arrs = host_arrays(batch)
        t = {}
        for n, a in arrs.items():
            h = torch.from_numpy(a)
            if pinned:
                h = h.pin_memory()
            t[n] = h.to(self.device, non_blocking=non_blocking)
        return DeviceBatch(batch_shape(batch), t)

    def workspace(self, shape, cfg) -> torch.Tensor:
        n = L.orrb_workspace_size(self.ctx, shape, cfg)
        if self._ws is None or self._ws.numel() < n:
            self._ws = torch.empty(n, dtype=torch.uint8, device=self.device)
        return self._ws

    def alloc_outputs(self, n_pixels: int, rgb_linear: bool = False, gbuffer: bool = False,
                      rgb_graded: bool = False):
        d = self.device
        out = dict(rgb=torch.empty((n_pixels, 3), dtype=torch.uint8, device=d),
                   depth=torch.empty(n_pixels, dtype=torch.float32, device=d),
                   normal=torch.empty((n_pixels, 3), dtype=torch.int16, device=d),
                   seg=torch.empty(n_pixels, dtype=torch.uint8, device=d))
        if rgb_linear:
            out["rgb_linear"] = torch.empty((n_pixels, 3), dtype=torch.float32, device=d)
        if gbuffer:
            out["gbuffer"] = torch.empty((L.ORRB_GBUFFER_PLANES, n_pixels), dtype=torch.float32, device=d)
        if rgb_graded:
            out["rgb_graded"] = torch.empty((n_pixels, 3), dtype=torch.float32, device=d)
        return out

    def alloc_shadow_maps(self, db: DeviceBatch) -> torch.Tensor:
        """The shadow-map output [n_samples, 4, F, R, R] of a batch with shadows."""
        R, F = int(db.shape.shadow_res), max(1, int(db.shape.shadow_faces))
        return torch.empty((int(db.shape.n_samples), L.ORRB_MAX_LIGHTS, F, R, R), dtype=torch.float32,
                           device=self.device)

    def render(self, db: DeviceBatch, out=None, cfg: Optional[L.orrb_config] = None, rgb_linear: bool = False,
               gbuffer: bool = False, stream=None, workspace: Optional[torch.Tensor] = None, tracker: bool = False,
               rgb_graded: bool = False):
        """Render `db`; `tracker` adds the per (camera, instance) rows [n_cams, max instances, 8]; a batch
        with shadows also writes (and returns) its shadow maps as "shadow_map"."""
        cfg = cfg or config()
        if out is None:
            out = self.alloc_outputs(db.total_pixels, rgb_linear, gbuffer, rgb_graded)
            if tracker:
                out["tracker"] = torch.empty((int(db.shape.n_cams), int(db.shape.max_inst_per_sample), 8),
                                             dtype=torch.int32, device=self.device)
        if db.has_shadows and "shadow_map" not in out:
            out["shadow_map"] = self.alloc_shadow_maps(db)
        ws = workspace if workspace is not None else self.workspace(db.shape, cfg)
        outs = L.orrb_outputs(*[out[k].data_ptr() if k in out else None
                                for k in ("rgb", "depth", "normal", "seg", "rgb_linear", "gbuffer", "tracker",
                                          "shadow_map", "rgb_graded")])
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        L.orrb_render_batch(self.ctx, db.shape, db.desc, outs, cfg, ws.data_ptr(), ws.numel(), st)
        self._last_ws = ws
        return out

    def status(self, stream=None) -> int:
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        return L.orrb_read_status(self.ctx, self._last_ws.data_ptr(), st)

    def shade_backward(self, db: DeviceBatch, gbuffer: torch.Tensor, d_rgb: torch.Tensor, stream=None,
                       emission: bool = False, grading: bool = False):
        """(d material [S,32,4], d light [S,4,4], d exposure [S]), plus d emission [S,32] when
        `emission`, plus d grading [S,8] last when `grading` (then d_rgb is dL/d rgb_graded, the
        loss being on the graded colour)."""
        n = L.orrb_backward_workspace_size(self.ctx, db.shape)
        if self._bws is None or self._bws.numel() < n:
            self._bws = torch.empty(n, dtype=torch.uint8, device=self.device)
        S = db.shape.n_samples
        dm = torch.empty((S, L.ORRB_MAX_MATERIALS, 4), dtype=torch.float32, device=self.device)
        dl = torch.empty((S, L.ORRB_MAX_LIGHTS, 4), dtype=torch.float32, device=self.device)
        de = torch.empty(S, dtype=torch.float32, device=self.device)
        dem = torch.empty((S, L.ORRB_MAX_MATERIALS), dtype=torch.float32, device=self.device) if emission else None
        dg = torch.empty((S, 8), dtype=torch.float32, device=self.device) if grading else None
        grads = L.orrb_param_grads(dm.data_ptr(), dl.data_ptr(), de.data_ptr(),
                                   dem.data_ptr() if emission else None, dg.data_ptr() if grading else None)
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        d_rgb = d_rgb.contiguous()
        L.orrb_shade_backward(self.ctx, db.shape, db.desc, gbuffer.data_ptr(), d_rgb.data_ptr(), grads,
                              self._bws.data_ptr(), self._bws.numel(), st)
        r = (dm, dl, de) + ((dem,) if emission else ()) + ((dg,) if grading else ())
        return r


class GraphRender:
    """One fused render captured in a CUDA graph and replayed with new batch contents (with shadow
    maps the render is its three launches and a queue reset, all captured).

    The kernel reads every descriptor from device memory, so a batch with the
    same array shapes (a capacity bucket) renders by copying its parameters into
    the captured tensors (`update`) and replaying: one graph launch, no host
    planning, no allocation.
    """

    def __init__(self, renderer: Renderer, db: DeviceBatch, cfg: Optional[L.orrb_config] = None,
                 rgb_linear: bool = False, gbuffer: bool = False):
        self.r, self.db = renderer, db
        self.cfg = cfg or config()
        self.out = renderer.alloc_outputs(db.total_pixels, rgb_linear, gbuffer)
        n = L.orrb_workspace_size(renderer.ctx, db.shape, self.cfg)
        self.ws = torch.empty(n, dtype=torch.uint8, device=renderer.device)
        renderer.render(db, out=self.out, cfg=self.cfg, workspace=self.ws)   # plans and sets attributes
        torch.cuda.synchronize(renderer.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            renderer.render(db, out=self.out, cfg=self.cfg, workspace=self.ws)

    def update(self, batch) -> None:
        """Copy a host batch of identical array shapes into the captured device tensors."""
        arrs = host_arrays(batch)
        for k, a in arrs.items():
            t = self.db.tensors[k]
            if tuple(t.shape) != a.shape:
                raise ValueError(f"{k}: shape {a.shape} differs from the captured {tuple(t.shape)}")
            t.copy_(torch.from_numpy(a), non_blocking=False)

    def replay(self):
        self.graph.replay()
        return self.out


class CapturePipeline:
    """Round-robin pool of render targets with bulk readback (the capture pipeline of Sec. 4.4).

    `depth` slots, each holding device inputs, a workspace, device outputs and pinned
    host outputs for batches of one shape.  `submit` copies a batch's parameters from
    pinned host memory, renders on the compute stream and queues the bulk device-to-host
    copy of all channels on a copy stream, so a batch renders while the previous one is
    still being read back.  A slot is reused `depth` submissions later: read (or copy)
    its host outputs before then.
    """

    def __init__(self, renderer: Renderer, batch, depth: int = 2, cfg: Optional[L.orrb_config] = None):
        self.r = renderer
        self.cfg = cfg or config()
        self.shape = batch_shape(batch)
        self.compute = torch.cuda.Stream(device=renderer.device)
        self.copy = torch.cuda.Stream(device=renderer.device)
        arrs = host_arrays(batch)
        n_ws = L.orrb_workspace_size(renderer.ctx, self.shape, self.cfg)
        self.slots = []
        for _ in range(depth):
            dev_in = {k: torch.empty(a.shape, dtype=_DTYPES[k], device=renderer.device) for k, a in arrs.items()}
            db = DeviceBatch(self.shape, dev_in)
            out = renderer.alloc_outputs(int(self.shape.total_pixels))
            if db.has_shadows:  # the shadow maps are an output too, read back with the channels
                out["shadow_map"] = renderer.alloc_shadow_maps(db)
            self.slots.append(dict(
                db=db, out=out,
                host={k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items()},
                ws=torch.empty(n_ws, dtype=torch.uint8, device=renderer.device),
                rendered=torch.cuda.Event(), done=torch.cuda.Event()))
        self.k = 0

    @staticmethod
    def pin(batch) -> Dict[str, torch.Tensor]:
        """A batch's parameter arrays in pinned host memory (the form `submit` takes)."""
        return {k: torch.from_numpy(a).pin_memory() for k, a in host_arrays(batch).items()}

    def submit(self, pinned: Dict[str, torch.Tensor]):
        slot = self.slots[self.k % len(self.slots)]
        self.k += 1
        self.compute.wait_event(slot["done"])          # its previous readback has finished
        with torch.cuda.stream(self.compute):
            for k, t in slot["db"].tensors.items():
                t.copy_(pinned[k], non_blocking=True)
            self.r.render(slot["db"], out=slot["out"], cfg=self.cfg, stream=self.compute, workspace=slot["ws"])
            slot["rendered"].record(self.compute)
        self.copy.wait_event(slot["rendered"])
        with torch.cuda.stream(self.copy):
            for k, v in slot["out"].items():
                slot["host"][k].copy_(v, non_blocking=True)
            slot["done"].record(self.copy)
        return slot

    @staticmethod
    def result(slot) -> Dict[str, torch.Tensor]:
        slot["done"].synchronize()
        return slot["host"]


class ShadeFn(torch.autograd.Function):
    """rgb = shade(material, light, exposure_ev[, emission][, grading]) at fixed visibility.

    Forward renders the batch with the given parameter tensors (visibility does not depend on
    them) and returns rgb_linear, or with a grading tensor [S,8] the graded colour before
    quantisation (rgb_graded); backward runs the hand-written shading adjoint kernel and returns
    d material [S,32,5] (albedo rgb and specular; shininess gets 0), d light [S,4,4], d exposure
    [S], d emission [S,32] when an emission tensor is given, and d grading [S,8] (hue,
    saturation, contrast, brightness, temperature, tint, grain amplitude; the seed gets 0) when a
    grading tensor is given.
    """

    @staticmethod
    def forward(ctx, material, light, exposure_ev, renderer: Renderer, db: DeviceBatch, emission=None, grading=None):
        kw = dict(material=material.detach().contiguous(), light=light.detach().contiguous(),
                  exposure_ev=exposure_ev.detach().contiguous())
        if emission is not None:
            kw["emission"] = emission.detach().contiguous()
        if grading is not None:
            kw["grading"] = grading.detach().contiguous()
        dbp = db.with_params(**kw)
        out = renderer.render(dbp, rgb_linear=True, gbuffer=True, rgb_graded=grading is not None)
        ctx.renderer = renderer
        ctx.db = dbp
        ctx.emission = emission is not None
        ctx.graded = grading is not None
        ctx.save_for_backward(out["gbuffer"])
        return out["rgb_graded"] if ctx.graded else out["rgb_linear"]

    @staticmethod
    def backward(ctx, g):
        (gbuffer,) = ctx.saved_tensors
        grads = ctx.renderer.shade_backward(ctx.db, gbuffer, g.float(), emission=ctx.emission, grading=ctx.graded)
        dm, dl, de = grads[:3]
        rest = list(grads[3:])
        dem = rest.pop(0) if ctx.emission else None
        dg = rest.pop(0) if ctx.graded else None
        dmat = torch.zeros_like(ctx.db.tensors["material"])
        dmat[..., :4] = dm
        return dmat, dl, de, None, None, dem, dg


def to_numpy(out) -> Dict[str, np.ndarray]:
    r = {k: v.cpu().numpy() for k, v in out.items()}
    if "normal" in r:
        r["normal"] = r["normal"].view(np.uint16)
    return r
