"""Continuous-batching render service (the in-process analogue of the paper's render service, Sec. 4.1).

Requests (a few samples of the resident scene at some resolution and camera
count, each with fresh randomization parameters) arrive on any thread.  A
scheduler thread wakes every `tick_ms`, takes the requests that have arrived,
and -- while an in-flight slot is free and the device-memory budget allows --
packs them into one batch and launches it on one of several CUDA streams, so
a batch admitted while earlier ones are still rendering overlaps with them on
the GPU.  One completion thread per stream waits for that stream's batches in
order and stamps each request with the time its outputs became ready.  The
meshes stay resident for the life of the server (SSMS, Sec. 3).

A request's result does not depend on what it was batched with: the renderer
computes every pixel from its own sample's inputs only.

The device work sits behind a small backend interface (`memory_budget`,
`bytes_needed`, `launch`, `wait`, `release`), so the scheduling logic is
testable without a GPU.
"""

from __future__ import annotations

import collections
import itertools
import threading
import time
from dataclasses import dataclass, field
from typing import Any, Dict, List, Optional, Tuple

import numpy as np


@dataclass
class ServeRequest:
    rid: int
    batch: Any                      # scenegen.Batch of this request's samples
    arrival: float = 0.0            # perf_counter() at submission
    done: float = 0.0               # perf_counter() when the outputs were ready
    result: Optional[Dict[str, Any]] = None
    error: Optional[str] = None     # set (and `event` signalled) when the request failed
    batch_id: int = -1
    event: threading.Event = field(default_factory=threading.Event)

    @property
    def latency_ms(self) -> float:
        return 1e3 * (self.done - self.arrival)


@dataclass
class InFlight:
    batch_id: int
    requests: List[ServeRequest]
    handle: Any
    nbytes: int
    stream_index: int


class Server:
    """Scheduler + completion threads around a backend."""

    def __init__(self, backend, n_streams: int = 2, max_inflight: int = 4, tick_ms: float = 2.0,
                 max_batch_samples: int = 1024, memory_budget: Optional[int] = None):
        self.backend = backend
        self.n_streams = n_streams
        self.max_inflight = max_inflight
        self.tick = tick_ms / 1e3
        self.max_batch_samples = max_batch_samples
        self.budget = memory_budget if memory_budget is not None else backend.memory_budget()
        self.pending: collections.deque = collections.deque()
        self.lock = threading.Condition()
        self.inflight: Dict[int, InFlight] = {}
        self.inflight_bytes = 0
        self.per_stream: List[collections.deque] = [collections.deque() for _ in range(n_streams)]
        self.stream_cv = [threading.Condition() for _ in range(n_streams)]
        # (request id, latency ms, samples) of every completed request: only what stats() reads, so
        # that a long-running server holds no request's outputs once its caller has dropped them
        self.completed: List[Tuple[int, float, int]] = []
        self.failed: List[ServeRequest] = []   # requests whose batch failed to launch or to render
        self.max_concurrent = 0
        self.launching = 0    # batches taken from `pending` whose launch has not been recorded yet
        self.batches_launched = 0
        self.rejected_for_memory = 0
        self._ids = itertools.count()
        self._next_stream = 0
        self._stop = False
        self._threads = [threading.Thread(target=self._schedule, daemon=True)]
        self._threads += [threading.Thread(target=self._complete, args=(k,), daemon=True) for k in range(n_streams)]
        for t in self._threads:
            t.start()

    # -- client side ------------------------------------------------------------
    def submit(self, req: ServeRequest) -> ServeRequest:
        req.arrival = time.perf_counter()
        with self.lock:
            self.pending.append(req)
        return req

    def close(self, timeout: float = 60.0) -> None:
        deadline = time.perf_counter() + timeout
        while True:
            with self.lock:
                idle = not self.pending and not self.inflight and not self.launching
            if idle or time.perf_counter() > deadline:
                break
            time.sleep(self.tick)
        self._stop = True
        for cv in self.stream_cv:
            with cv:
                cv.notify_all()
        for t in self._threads:
            t.join(timeout=5.0)

    # -- scheduler ----------------------------------------------------------------
    def _schedule(self) -> None:
        while not self._stop:
            t0 = time.perf_counter()
            self._admit()
            dt = self.tick - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)

    def _admit(self) -> None:
        while True:
            with self.lock:
                if not self.pending or len(self.inflight) >= self.max_inflight:
                    return
                take, n = [], 0
                for req in self.pending:
                    if take and n + req.batch.n_samples > self.max_batch_samples:
                        break
                    take.append(req)
                    n += req.batch.n_samples
                try:
                    need = self.backend.bytes_needed([r.batch for r in take])
                    while len(take) > 1 and self.inflight_bytes + need > self.budget:
                        take.pop()                       # admit a smaller prefix that fits
                        need = self.backend.bytes_needed([r.batch for r in take])
                    invalid = None
                except Exception as e:  # a request the host cannot even size: fail what was taken
                    for _ in take:
                        self.pending.popleft()
                    invalid = e
            if invalid is not None:
                self._fail(take, f"invalid request: {invalid}")
                continue
            with self.lock:
                too_big = not self.inflight and need > self.budget
                if too_big:                          # (a single request) it can never fit: fail it, serve the rest
                    for _ in take:
                        self.pending.popleft()
                elif self.inflight_bytes + need > self.budget:
                    self.rejected_for_memory += 1
                    return                           # wait for an in-flight batch to free memory
            if too_big:
                self._fail(take, f"does not fit in device memory: needs {need} bytes of a {self.budget}-byte budget")
                continue
            with self.lock:  # (counted as launching until it is in flight, so close() waits for it)
                for _ in take:
                    self.pending.popleft()
                bid = next(self._ids)
                k = self._next_stream
                self._next_stream = (k + 1) % self.n_streams
                self.inflight_bytes += need
                self.launching += 1
            try:
                handle = self.backend.launch([r.batch for r in take], k)
            except Exception as e:  # the batch never started: fail its requests, free its budget
                with self.lock:
                    self.inflight_bytes -= need
                    self.launching -= 1
                self._fail(take, f"launch failed: {e}")
                continue
            fl = InFlight(bid, take, handle, need, k)
            for r in take:
                r.batch_id = bid
            with self.lock:
                self.inflight[bid] = fl
                self.launching -= 1
                self.max_concurrent = max(self.max_concurrent, len(self.inflight))
                self.batches_launched += 1
            with self.stream_cv[k]:
                self.per_stream[k].append(fl)
                self.stream_cv[k].notify()

    # -- completion ----------------------------------------------------------------
    def _complete(self, k: int) -> None:
        q, cv = self.per_stream[k], self.stream_cv[k]
        while True:
            with cv:
                while not q and not self._stop:
                    cv.wait(timeout=0.05)
                if not q:
                    return
                fl = q.popleft()
            try:
                results, error = self.backend.wait(fl.handle), None
            except Exception as e:  # the batch ran but its results cannot be trusted
                results, error = [None] * len(fl.requests), f"render failed: {e}"
            now = time.perf_counter()
            for r, res in zip(fl.requests, results):
                r.result = res
                r.error = error
                r.done = now
            try:
                self.backend.release(fl.handle)
            finally:
                with self.lock:
                    self.inflight.pop(fl.batch_id, None)
                    self.inflight_bytes -= fl.nbytes
                    if error:
                        self.failed.extend(fl.requests)
                    else:
                        self.completed.extend((r.rid, r.latency_ms, r.batch.n_samples) for r in fl.requests)
                for r in fl.requests:      # signal only once the bookkeeping is visible to stats()
                    r.event.set()

    def _fail(self, reqs, error: str) -> None:
        now = time.perf_counter()
        for r in reqs:
            r.error = error
            r.done = now
        with self.lock:
            self.failed.extend(reqs)
        for r in reqs:
            r.event.set()

    # -- report ----------------------------------------------------------------------
    def stats(self, wall_s: float) -> Dict[str, float]:
        with self.lock:  # a consistent snapshot while batches may still complete
            done, n_failed = list(self.completed), len(self.failed)
            batches, conc, waits = self.batches_launched, self.max_concurrent, self.rejected_for_memory
        lat = np.array([ms for _, ms, _ in done]) if done else np.zeros(1)
        samples = sum(ns for _, _, ns in done)
        return {"requests": len(done), "samples": samples, "samples_per_s": samples / wall_s,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(lat.max()), "batches": batches, "failed": n_failed,
                "max_concurrent_batches": conc, "memory_waits": waits}


_TD: Dict[Any, Any] = {}


def _torch_dtypes(torch) -> Dict[Any, Any]:
    """numpy dtype -> torch dtype for the parameter arrays' types."""
    if not _TD:
        for n in ("int16", "int32", "int64", "uint8", "float32"):
            _TD[np.dtype(n)] = getattr(torch, n)
    return _TD


class ParamStage:
    """One batch's parameters in one pinned host buffer and one device buffer, each array at a
    256-byte aligned offset, so a launch makes one host-to-device copy instead of page-locking and
    copying every array.  A stage belongs to one in-flight batch from its launch to its release
    (after the batch has finished on the GPU), so neither buffer is rewritten while a copy or the
    render can still read it, and no launch waits for one."""

    def __init__(self, torch, device, nbytes: int):
        self.host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        self.dev = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.host_np = self.host.numpy()

    @property
    def capacity(self) -> int:
        return int(self.host.numel())

    @staticmethod
    def layout(arrs) -> tuple:
        offs, o = {}, 0
        for n, a in arrs.items():
            offs[n] = o
            o = (o + a.nbytes + 255) & ~255
        return offs, max(o, 256)

    def upload(self, torch, arrs, offs, nbytes: int, stream):
        """Device tensors holding `arrs` (name -> contiguous numpy array), copied on `stream`."""
        h = self.host_np
        for n, a in arrs.items():
            h[offs[n]:offs[n] + a.nbytes] = a.reshape(-1).view(np.uint8)
        with torch.cuda.stream(stream):
            self.dev[:nbytes].copy_(self.host[:nbytes], non_blocking=True)
        # (flat views: the renderer reads only each array's address)
        td = _torch_dtypes(torch)
        return {n: self.dev[offs[n]:offs[n] + a.nbytes].view(td[a.dtype]) for n, a in arrs.items()}


class GpuBackend:
    """Packs requests into one batch and renders it on a per-slot CUDA stream.

    Each in-flight batch gets its own workspace and outputs, so batches on
    different streams never share scratch memory.  `readback` copies the
    channels to pinned host memory before the request counts as done.
    """

    def __init__(self, meshes, device: int = 0, n_streams: int = 2, cfg=None, readback: bool = False,
                 reserve_bytes: int = 8 << 30, n_stages: int = 4, stage_bytes: int = 8 << 20):
        import torch

        from . import lib as L
        from .render import Renderer, config
        self.torch, self.L = torch, L
        self.r = Renderer(meshes, device=device)
        self.cfg = cfg or config()
        self.streams = [torch.cuda.Stream(device=self.r.device) for _ in range(n_streams)]
        self.readback = readback
        self.reserve = reserve_bytes
        # workspace bytes ~ a + b * (triangles of the largest sample), fitted from two library queries
        w = [L.orrb_workspace_size(self.r.ctx, L.orrb_batch_shape(1, 1, t, 64, 3, 512, 512, 1 << 18), self.cfg)
             for t in (10000, 20000)]
        self.ws_b = (w[1] - w[0]) / 10000.0
        self.ws_a = w[0] - 10000 * self.ws_b
        # parameter stages, allocated up front (one per batch in flight; 8 MB holds the parameters of
        # about 2,000 samples with shadow cameras); a batch larger than a stage gets a bigger one
        self.stage_bytes = stage_bytes
        self._stage_lock = threading.Lock()
        self._stages = [ParamStage(torch, self.r.device, stage_bytes) for _ in range(n_stages)]

    def memory_budget(self) -> int:
        free, _ = self.torch.cuda.mem_get_info(self.r.device)
        return max(0, free - self.reserve)

    def _shape(self, batches):
        from .render import batch_shape
        from .scenegen import concat_batches
        packed = concat_batches(batches)
        return packed, batch_shape(packed)

    def bytes_needed(self, batches) -> int:
        px = sum(b.total_pixels for b in batches)
        tris = max(int(b.tris_per_sample().max()) for b in batches)
        # outputs (14 B per pixel) + workspace + parameters, + shadow maps (4 B per texel) and their
        # neighbourhood table (4 B + a 1-byte count per texel), + the post pass's images (46 B per
        # pixel) when a request carries ambient occlusion and bloom
        maps = sum(b.n_samples * 4 * b.shadow_faces * b.shadow_res ** 2 * 9
                   for b in batches if getattr(b, "shadow_view", None) is not None)
        post = px * 46 + 256 * 5 if any(getattr(b, "post", None) is not None for b in batches) else 0
        return int(px * 14 + self.ws_a + self.ws_b * tris + sum(b.n_samples for b in batches) * 4096 + maps + post)

    def _take_stage(self, nbytes: int) -> ParamStage:
        with self._stage_lock:
            for i, st in enumerate(self._stages):
                if st.capacity >= nbytes:
                    return self._stages.pop(i)
        return ParamStage(self.torch, self.r.device, max(self.stage_bytes, 1 << int(nbytes - 1).bit_length()))

    def launch(self, batches, k: int):
        torch = self.torch
        from .render import DeviceBatch, host_arrays
        with torch.cuda.nvtx.range("serve: pack batch"):  # (a timeline range; no-op without a profiler)
            packed, shape = self._shape(batches)
            arrs = host_arrays(packed)
            offs, nbytes = ParamStage.layout(arrs)
        s = self.streams[k]
        stage = self._take_stage(nbytes)
        try:
            t = stage.upload(torch, arrs, offs, nbytes, s)
            with torch.cuda.stream(s):
                db = DeviceBatch(shape, t)
                n_ws = self.L.orrb_workspace_size(self.r.ctx, shape, self.cfg)
                ws = torch.empty(n_ws, dtype=torch.uint8, device=self.r.device)
                out = self.r.render(db, cfg=self.cfg, stream=s, workspace=ws)
                host = None
                if self.readback:
                    host = {k2: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k2, v in out.items()}
                    for k2 in out:
                        host[k2].copy_(out[k2], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s)
        except Exception:
            # the copy may be queued: the stage is not reused before the stream has drained
            s.synchronize()
            self._put_stage(stage)
            raise
        return {"db": db, "ws": ws, "out": out, "host": host, "event": ev, "batches": batches, "stream": s,
                "stage": stage}

    def _put_stage(self, stage: ParamStage) -> None:
        with self._stage_lock:
            self._stages.append(stage)

    def wait(self, h):
        h["event"].synchronize()
        status = self.L.orrb_read_status(self.r.ctx, h["ws"].data_ptr(), h["stream"].cuda_stream)
        if status:  # a content check or a bounded wait on the device gave up: the outputs are not trusted
            raise RuntimeError(f"device status {status:#x}")
        res, p0, s0 = [], 0, 0
        src = h["host"] if h["host"] is not None else h["out"]
        for b in h["batches"]:
            n, ns = b.total_pixels, b.n_samples
            # channels are flat over pixels; shadow maps are per sample
            res.append({k: (v[s0:s0 + ns] if k == "shadow_map" else v[p0:p0 + n]) for k, v in src.items()})
            p0 += n
            s0 += ns
        return res

    def release(self, h):
        # tensors return to torch's caching allocator once the stream's work is done; the batch has
        # finished (wait() synchronised on its event, or the launch failed and drained), so its
        # stage is free again
        h["ws"].record_stream(h["stream"])
        stage = h.get("stage")
        h.clear()
        if stage is not None:
            self._put_stage(stage)


def run_poisson(server: Server, requests, batches, duration_s: float, warmup_s: float = 0.0,
                keep_results: bool = True):
    """Submit `batches[i]` at arrival time `requests[i].arrival_s`; returns (submitted ServeRequests, wall seconds).
    With keep_results=False the client drops each request's outputs as soon as the request has
    completed (a client that consumes its results), so the device memory of finished batches
    returns to the allocator during the run; latencies and errors are kept."""
    t0 = time.perf_counter()
    subs = []
    oldest = 0  # the first request whose outputs may still be held
    for req, b in zip(requests, batches):
        delay = t0 + req.arrival_s - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        subs.append(server.submit(ServeRequest(req.rid, b)))
        if not keep_results:
            while oldest < len(subs) and subs[oldest].event.is_set():
                subs[oldest].result = None
                oldest += 1
    for s in subs:
        s.event.wait(timeout=60.0)
        if not keep_results:
            s.result = None
    return subs, time.perf_counter() - t0
