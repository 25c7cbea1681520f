"""Throughput benchmark of the batched renderer (one JSON line on rank 0).

Workload: the hand-like scene -- 24 capsule links (320 triangles each) posed by
seeded hinge angles, a 12-triangle block with 6 face materials, a 2-triangle
table; 256 samples x 3 cameras at 200x200 with camera jitter, 1-4 point lights,
random materials; all four channels (RGB u8, depth f32, normal f16x3, seg u8).
The paper's benchmark scene (Sec. 5: Shadow hand + block, 3 cameras, 200x200)
is not available; this seeded synthetic scene of the same shape stands in.

A step renders one batch.  `value` is samples/s with inputs resident in HBM,
timed per step with CUDA events on the launch stream, L2 flushed between
steps (a 256 MB write) outside the events.  `e2e` is the same metric through
the public API with host buffers: each step copies the batch parameters from
pinned host memory, renders, and copies all four channels back to pinned host
memory (the paper's capture pipeline returns the whole batch to the CPU,
Sec. 4.4).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import json
import math
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "samples/s (RGB+depth+normal+seg, 3x200² cams) at 1 B300, fused vs plain; % roofline"
UNIT = "samples/s"
N_SAMPLES = 256
N_CAMS = 3
RES = 200
SEED = 0
SHADOW_RES = 256    # side of the spot lights' shadow maps in the shadow workload
CUBE_RES = 128      # side of the point lights' cube-map faces in the cube workload
BYTES_PER_PX = 3 + 4 + 6 + 1           # rgb u8x3, depth f32, normal f16x3, seg u8
CONFIG = {"workload": "hand-like scene: 256 samples x 3 cameras x 200x200, 24 capsule links + block + table, "
                      "1-4 point lights, 4 channels", "global_batch": N_SAMPLES, "cameras": N_CAMS,
          "resolution": RES, "tris_per_sample": 24 * 320 + 14, "l2": "flushed between timed steps (256 MB write)"}


def set_samples(n: int) -> None:
    global N_SAMPLES, CONFIG
    N_SAMPLES = n
    CONFIG = dict(CONFIG, workload=CONFIG["workload"].replace("256 samples", f"{n} samples"), global_batch=n)


def parallelism(world: int) -> str:
    """How the job splits over its ranks (the same words in both arms' config)."""
    return f"replicas x{world}" if world > 1 else "single GPU"


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("orrb_render.cu", "orrb_internal.h", "orrb_shading.cuh"):
        with open(os.path.join(ROOT, "paper_1906_11633_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_value(key: str):
    """A figure (`key: value` line) of the committed ncu summary, if it was taken on this kernel source."""
    try:
        text = open(os.path.join(ROOT, "profiles", "render_fused_hand256.md")).read()
    except OSError:
        return None
    if kernel_source_hash() not in text:
        return None
    for line in text.splitlines():
        if line.startswith(key + ":"):
            return float(line.split(":")[1])
    return None


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this kernel source."""
    return profiled_value("traffic_bytes_per_launch")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0}, "fallback"


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    """Dense FP32 FMA peak: SMs x 128 lanes x 2 flop x clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


# Algorithmic FP32 operations of the per-pixel steps (G-buffer interpolation, shading, grading,
# quantisation), with the per-term counts that the oracle tallies beside its own arithmetic
# (oracle/orrb_oracle.c, render_image and shade_f32; each +, -, *, /, sqrt, pow, negation,
# comparison and clamp counts once; work that depends on the image only, such as moving the lights
# to view space, counts once per image).  tests/test_oracle_flops.py checks this function against
# the oracle's count on the same G-buffer.  Shadow-map lookups are not counted (a lower bound for
# the shadowed workloads).
FLOP_PIXEL = {False: 91, True: 74}        # per visible pixel: perspective, orthographic camera
FLOP_LIGHT = {0: 33, 1: 20, 2: 33}        # per (visible pixel, light) by light type
FLOP_SPOT_CONE, FLOP_SPOT_NULL = 16, 8    # more per (pixel, spot light): a cone, a null cone
FLOP_LIT = 21                             # more per (pixel, light) with n . L > 0
FLOP_GRADE, FLOP_GRADE_BG = 64, 64 + 18   # per graded visible pixel, per graded background pixel


def alg_flops(batch, gb_pos, gb_nrm, gb_mat) -> float:
    """The algorithmic FP32 operations of one render of `batch`, from its G-buffer (positions
    [N, 3], normals [N, 3], material words [N], -1 background)."""
    total = 0
    start = 0
    for c in range(batch.n_cams):
        n = int(batch.cam_wh[c, 0]) * int(batch.cam_wh[c, 1])
        sl = slice(start, start + n)
        start += n
        s = int(batch.cam_sample[c])
        ortho = bool(batch.cam_intr[c, 5] != 0)
        fg = gb_mat[sl] >= 0
        nv = int(fg.sum())
        count, typ = int(batch.light_meta[s, 0]), int(batch.light_meta[s, 1])
        if not (typ in (0, 1) or (typ == 2 and batch.light_spot is not None)):
            count = 0
        graded = batch.grading is not None
        total += 2 + count * (18 + (16 if typ == 2 else 0)) + 1 + (6 if graded else 0)   # per image
        total += nv * FLOP_PIXEL[ortho] + (n - nv) * (FLOP_GRADE_BG if graded else 0) + (nv * FLOP_GRADE if graded else 0)
        if nv == 0 or count == 0:
            continue
        V = batch.cam_view[c].astype(np.float64)
        P = gb_pos[sl][fg].astype(np.float64)
        nrm = gb_nrm[sl][fg].astype(np.float64)
        for l in range(count):
            total += nv * FLOP_LIGHT[typ]
            if typ == 2:
                sp = batch.light_spot[s, l]
                total += nv * (FLOP_SPOT_CONE if sp[4] > sp[3] else FLOP_SPOT_NULL)
            if typ == 1:
                Ld = np.broadcast_to(-(V[:, :3] @ batch.light[s, l, :3]), P.shape)
            else:
                Ld = V[:, :3] @ batch.light[s, l, :3] + V[:, 3] - P
            total += FLOP_LIT * int((np.einsum("ij,ij->i", nrm, Ld) > 0).sum())
    return float(total)


def measured_fp32_peak(reps: int = 3):
    """FP32 multiply-add throughput measured on this device by the probe library (scalar FFMA and
    packed FFMA2 chains, CUDA events): (best TFLOP/s, scalar, packed), or None if unavailable."""
    import ctypes
    path = os.path.join(ROOT, "paper_1906_11633_b300", "libfp32peak.so")
    try:
        lib = ctypes.CDLL(path)
    except OSError:
        return None
    a, b = ctypes.c_double(), ctypes.c_double()
    if lib.orrb_measure_fp32_peak(reps, ctypes.byref(a), ctypes.byref(b)) != 0:
        return None
    return max(a.value, b.value) / 1e12, a.value / 1e12, b.value / 1e12


class ClockSampler:
    """Samples SM clock and clock-event reasons with nvidia-smi while the timed region runs (read-only)."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id: str, period_ms: int = 20):
        self.gpu_id, self.period_ms = gpu_id, period_ms
        self.proc = None
        self.lines = []

    def __enter__(self):
        import subprocess
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.2)
        return self

    def __exit__(self, *a):
        time.sleep(0.05)
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < len(self.FIELDS):
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for name, v in zip(self.NAMES, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi during the timed fused steps"}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def shard_samples(rank: int, world: int, n: int) -> np.ndarray:
    """Sample ids of rank `rank`: every rank renders its own n samples (weak scaling, no collective)."""
    return np.arange(rank * n, (rank + 1) * n, dtype=np.int64)


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_baseline(batch, budget_s: float = 15.0):
    """Time the CPU oracle on a bounded sample of the workload on all host cores."""
    from oracle import oracle as orc
    from paper_1906_11633_b300 import scenegen as sg
    threads = orc.default_threads()
    n, passes, dt = 16, 0, 0.0
    sub = sg.select_samples(batch, list(range(n)))
    while dt < budget_s and passes < 1000:
        t0 = time.perf_counter()
        orc.render(sub, threads=threads)
        dt += time.perf_counter() - t0
        passes += 1
    # one core as well, on a smaller slice (the oracle itself is single-threaded per image)
    one = sg.select_samples(batch, [0, 1])
    p1, dt1 = 0, 0.0
    while dt1 < 3.0 and p1 < 100:
        t0 = time.perf_counter()
        orc.render(one, threads=1)
        dt1 += time.perf_counter() - t0
        p1 += 1
    return {"value": n * passes / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {n} of the {batch.n_samples} samples ({n * N_CAMS} images) x {passes} passes, "
                      f"{dt:.1f} s",
            "single_core": {"value": 2 * p1 / dt1, "unit": UNIT,
                            "sample": f"first 2 samples (6 images) x {p1} passes on 1 thread, {dt1:.1f} s"}}


def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_1906_11633_b300 import scenegen as sg
    from oracle import oracle as orc
    batch = sg.hand_batch(SEED, np.arange(N_SAMPLES), res=RES, n_cams=N_CAMS)
    threads = orc.default_threads()
    n = max(8, threads)                    # samples per step: a bounded slice of the batch, three images a thread
    per = []
    for i in range(args.warmup + args.steps):
        ids = [(i * n + k) % N_SAMPLES for k in range(n)]
        sub = sg.select_samples(batch, ids)
        t0 = time.perf_counter()
        orc.render(sub, threads=threads)
        if i >= args.warmup:
            per.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(per))
    value = n / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(CONFIG, parallelism=parallelism(args.gpus)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{n} samples ({n * N_CAMS} images) per step of the same workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    from paper_1906_11633_b300 import scenegen as sg
    from paper_1906_11633_b300 import lib as L
    from paper_1906_11633_b300.render import Renderer, config, host_arrays, DeviceBatch, batch_shape

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ids = shard_samples(rank, world, N_SAMPLES)
    batch = sg.hand_batch(SEED, ids, res=RES, n_cams=N_CAMS)
    r = Renderer(batch.meshes, device=local)
    db = r.upload(batch)
    cfg = config(mode=L.ORRB_MODE_FUSED, tile_w=args.tile_w, tile_h=args.tile_h, threads=args.threads)
    out = r.render(db, cfg=cfg, rgb_linear=False)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    N = batch.total_pixels

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        evs = []
        for _ in range(steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        barrier(world)
        return [a.elapsed_time(b) for a, b in evs]

    # -- fused (the headline) ----------------------------------------------------
    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    with ClockSampler(gpu_id) as clk:
        per = timed(lambda: r.render(db, out=out, cfg=cfg), args.steps, args.warmup)
    status = r.status()
    total_ms = max_over_ranks(float(np.sum(per)), world)
    ms = total_ms / args.steps
    value = world * N_SAMPLES * args.steps / (total_ms / 1e3)
    kernel_ms = float(np.mean(per))

    # -- plain per-sample launches (comparison) ----------------------------------
    pcfg = config(mode=L.ORRB_MODE_PLAIN, tile_w=args.tile_w, tile_h=args.tile_h, threads=args.threads)
    psteps = max(3, args.steps // 10)
    pper = timed(lambda: r.render(db, out=out, cfg=pcfg), psteps, min(args.warmup, 3))
    plain_ms = max_over_ranks(float(np.sum(pper)), world) / psteps
    plain_value = world * N_SAMPLES / (plain_ms / 1e3)

    # -- staged: the same three kernels launched once each over the whole batch (a non-fused
    # comparison without the per-sample launch overhead of the plain mode) ----------------------
    scfg = config(mode=L.ORRB_MODE_STAGED, tile_w=args.tile_w, tile_h=args.tile_h, threads=args.threads)
    ssteps = max(3, args.steps // 10)
    sper = timed(lambda: r.render(db, out=out, cfg=scfg), ssteps, min(args.warmup, 3))
    staged_ms = max_over_ranks(float(np.sum(sper)), world) / ssteps
    staged_value = world * N_SAMPLES / (staged_ms / 1e3)
    staged_ok = bool(all(torch.equal(a, b) for a, b in zip(
        r.render(db, cfg=scfg).values(), r.render(db, cfg=cfg).values())))

    # -- e2e through host buffers: the capture pipeline (Sec. 4.4) -------------------
    # every step copies its parameters from pinned host memory, renders, and reads all
    # four channels back to pinned host memory; consecutive steps overlap (render of
    # step k+1 during the readback of step k) on two slots
    from paper_1906_11633_b300.render import CapturePipeline
    arrs = host_arrays(batch)
    pipe = CapturePipeline(r, batch, depth=2, cfg=cfg)
    pinned_in = CapturePipeline.pin(batch)
    h2d = sum(v.numel() * v.element_size() for v in pinned_in.values())
    d2h = sum(v.numel() * v.element_size() for v in pipe.slots[0]["out"].values())
    esteps = max(6, args.steps // 5)
    for _ in range(min(args.warmup, 3)):
        last = pipe.submit(pinned_in)
    CapturePipeline.result(last)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(pipe.compute)
    for _ in range(esteps):
        last = pipe.submit(pinned_in)
    e1.record(pipe.copy)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world) / esteps
    e2e_value = world * N_SAMPLES / (e2e_ms / 1e3)
    ok = bool((CapturePipeline.result(last)["seg"].numpy() == out["seg"].cpu().numpy()).all())

    # -- the differentiation pattern on the same batch: forward with G-buffer + shading adjoint ---
    dfms, dbms, dbytes = time_diff(r, db, batch, reps=10, warmup=3)
    # -- the batching and serving patterns, briefly (their own workloads measure them at length) --
    uneven = serve = None
    if not args.no_patterns:
        uneven = measure_uneven(args, world, rank, local)
        serve = measure_serve(1.0, world, rank, local)

    if rank != 0:
        return
    # -- roofline -----------------------------------------------------------------
    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    param_bytes = sum(v.nbytes for k, v in arrs.items())
    mesh_bytes = int(r.arena.numel())
    alg_bytes = BYTES_PER_PX * N + param_bytes + mesh_bytes
    # algorithmic shading FLOPs from this batch's visible pixels and lights
    o = r.render(db, cfg=cfg, rgb_linear=True, gbuffer=True)
    gb = o["gbuffer"].cpu().numpy()
    flops = alg_flops(batch, gb[0:3].T, gb[3:6].T, gb[6].view(np.int32))
    props = torch.cuda.get_device_properties(dev)
    clk_sum = clk.summary()
    nominal = fp32_peak_tflops(props.multi_processor_count, float(peaks.get("sm_max_mhz", 2032.0)))
    probe = measured_fp32_peak()
    fp32_peak = probe[0] if probe is not None else nominal
    t_hbm = alg_bytes / (hbm * 1e9)
    t_fp32 = flops / (fp32_peak * 1e12)
    bound = "hbm" if t_hbm >= t_fp32 else "alu"
    achieved_gbs = alg_bytes / (kernel_ms / 1e3) / 1e9
    achieved_tf = flops / (kernel_ms / 1e3) / 1e12
    roof = {"bound": bound,
            "achieved": achieved_gbs if bound == "hbm" else achieved_tf,
            "peak": hbm if bound == "hbm" else fp32_peak,
            "unit": "GB/s" if bound == "hbm" else "TFLOP/s",
            "frac": (achieved_gbs / hbm) if bound == "hbm" else (achieved_tf / fp32_peak),
            "traffic": args.traffic if args.traffic is not None else profiled_traffic(),
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if bound == "hbm" else
                           ("measured FP32 FMA-chain probe" if probe is not None else
                            "nominal: SMs x 128 x 2 x max SM clock"),
            "fp32_peak_tflops": {"measured_scalar_ffma": probe[1] if probe else None,
                                 "measured_packed_ffma2": probe[2] if probe else None,
                                 "nominal": nominal, "used": fp32_peak},
            "alg_bytes_per_launch": alg_bytes, "alg_fp32_flop_per_launch": flops,
            "t_roof_us": 1e6 * max(t_hbm, t_fp32), "t_hbm_us": 1e6 * t_hbm, "t_fp32_us": 1e6 * t_fp32,
            "roofline_frac_of_step": 1e3 * max(t_hbm, t_fp32) / kernel_ms,
            "kernel": "render_fused_kernel"}
    # secondary (not the headline): the instruction-issue roofline, with the warp instructions
    # per pixel that ncu counted on this kernel source (rasterisation is integer/issue work
    # that the FP32 shading term does not count)
    ipp = profiled_value("warp_instructions_per_pixel")
    if ipp is not None:
        issue_peak = props.multi_processor_count * 4 * float(peaks.get("sm_max_mhz", 2032.0)) * 1e6
        inst = ipp * N
        roof["secondary_issue"] = {"warp_inst_per_launch": inst, "achieved_ginst_s": inst / (kernel_ms / 1e3) / 1e9,
                                   "peak_ginst_s": issue_peak / 1e9,
                                   "frac": inst / (kernel_ms / 1e3) / issue_peak,
                                   "source": "ncu smsp__inst_executed per pixel (profiles/render_fused_hand256.md); "
                                             "peak = SMs x 4 schedulers x max SM clock"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded procedural hand scene)",
            "config": dict(CONFIG, parallelism=parallelism(world)),
            "launch": {"tile": [min(args.tile_w or L.DEFAULT_TILE_W, RES), args.tile_h or L.DEFAULT_TILE_H],
                       "threads": args.threads or L.DEFAULT_THREADS},
            "plain": {"value": plain_value, "ms_per_step": plain_ms, "steps": psteps,
                      "launches_per_step": 3 * N_SAMPLES},
            "fused_over_plain": value / plain_value,
            "staged": {"value": staged_value, "ms_per_step": staged_ms, "steps": ssteps,
                       "launches_per_step": 3, "outputs_equal_fused": staged_ok,
                       "how": "every image's geometry, then every image's binning, then the raster: "
                              "three batch-wide launches of the plain kernels, one scratch slot per image"},
            "fused_over_staged": value / staged_value,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "ms_per_step": e2e_ms, "steps": esteps, "readback_ok": bool(ok),
                    "how": "CapturePipeline: 2 round-robin slots, H2D + render on one stream, bulk D2H of all "
                           "channels on a copy stream; D2H is capped near 57 GB/s on this host link"},
            "gpu_launches": args.steps,
            "roofline": roof,
            "uneven": None if uneven is None else {
                k: uneven[k] for k in ("value", "ms_per_step", "fused_over_plain", "plain", "fused_over_staged", "staged",
                                       "device_status")} | {
                "config": {k: uneven["config"][k] for k in ("scenes", "images", "pixels", "triangles_per_scene", "tile",
                                                             "threads")}},
            "serve": None if serve is None else {
                k: serve[k] for k in ("value", "p50_ms", "p99_ms", "max_ms", "requests", "batches",
                                      "max_concurrent_batches")} | {"seconds": 1.0, "rate_hz": 2000.0},
            "diff": {"forward_gbuffer_ms": dfms, "adjoint_ms": dbms,
                     "adjoint_achieved_gbs": dbytes / (dbms / 1e3) / 1e9,
                     "adjoint_frac_of_hbm": dbytes / (dbms / 1e3) / 1e9 / hbm,
                     "adjoint_alg_bytes": dbytes,
                     "how": "L2 loss against a target rendered with perturbed parameters; adjoint = "
                            "backward_partial_kernel + backward_reduce_kernel; 40 B per pixel read"},
            "clocks": clk_sum,
            "device_status": status}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(batch)
    print(json.dumps(line), flush=True)


def run_uneven(args, world, rank, local):
    """1024 scenes with log-uniform [1k, 50k] triangles, square resolutions U{64..512}, 1-3 cameras: one
    persistent launch replayed from a CUDA graph with the autotuned tiling, vs per-scene plain launches."""
    line = measure_uneven(args, world, rank, local)
    if line is not None:
        print(json.dumps(line), flush=True)


def measure_uneven(args, world, rank, local):
    """The uneven workload's JSON line (rank 0; None on the others)."""
    import torch
    from paper_1906_11633_b300 import scenegen as sg
    from paper_1906_11633_b300 import lib as L
    from paper_1906_11633_b300.render import GraphRender, Renderer, config
    from paper_1906_11633_b300.tune import tune
    torch.cuda.set_device(local)
    n = 1024
    batch = sg.uneven_batch(SEED, shard_samples(rank, world, n))
    r = Renderer(batch.meshes, device=local)
    db = r.upload(batch)
    cfg, timings = tune(r, db, reps=3)
    g = GraphRender(r, db, cfg=cfg)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    per = []
    for _ in range(max(5, args.steps // 10)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        per.append((e0, e1))
    torch.cuda.synchronize()
    ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in per])), world)
    out = g.out
    pcfg = config(mode=L.ORRB_MODE_PLAIN, tile_w=cfg.tile_w, tile_h=cfg.tile_h, threads=cfg.threads)
    r.render(db, out=out, cfg=pcfg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r.render(db, out=out, cfg=pcfg)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = max_over_ranks(e0.elapsed_time(e1), world)
    # staged: the plain kernels once each over chunks of the images (the slots of every image do not
    # fit the staged mode's scratch budget at 50k triangles per scene)
    scfg = config(mode=L.ORRB_MODE_STAGED, tile_w=cfg.tile_w, tile_h=cfg.tile_h, threads=cfg.threads)
    r.render(db, out=out, cfg=scfg)
    torch.cuda.synchronize()
    sper = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.render(db, out=out, cfg=scfg)
        e1.record(stream)
        sper.append((e0, e1))
    torch.cuda.synchronize()
    staged_ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in sper])), world)
    slot = (L.orrb_workspace_size(r.ctx, db.shape, pcfg) - 256) // max(1, int(db.shape.max_cams_per_sample))
    chunk = max(1, (L.orrb_workspace_size(r.ctx, db.shape, scfg) - 256) // slot)
    if rank != 0:
        return None
    peaks, _ = load_peaks()
    alg_bytes = BYTES_PER_PX * batch.total_pixels
    line = {"workload": "uneven", "metric": "samples/s, uneven batch in one persistent launch (CUDA graph)",
            "value": world * n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "n_gpus": world,
            "config": {"scenes": n, "images": batch.n_cams, "pixels": batch.total_pixels,
                       "triangles_per_scene": [int(batch.tris_per_sample().min()), int(batch.tris_per_sample().max())],
                       "tile": [cfg.tile_w, cfg.tile_h], "threads": cfg.threads, "tuner_ms": timings},
            "plain": {"value": world * n / (plain_ms / 1e3), "ms_per_step": plain_ms,
                      "launches_per_step": 3 * n},
            "fused_over_plain": plain_ms / ms,
            "staged": {"value": world * n / (staged_ms / 1e3), "ms_per_step": staged_ms,
                       "launches_per_step": 3 * -(-batch.n_cams // chunk), "images_per_chunk": int(chunk)},
            "fused_over_staged": staged_ms / ms,
            "roofline": {"bound": "hbm", "achieved": alg_bytes / (ms / 1e3) / 1e9, "peak": float(peaks["hbm_gbs"]),
                         "unit": "GB/s", "frac": alg_bytes / (ms / 1e3) / 1e9 / float(peaks["hbm_gbs"]),
                         "alg_bytes_per_launch": alg_bytes},
            "device_status": r.status()}
    return line


def time_diff(r, db, batch, reps: int, warmup: int):
    """Forward with G-buffer and shading adjoint of `db` (L2 loss against a target rendered with
    perturbed parameters): (forward ms, adjoint ms, algorithmic adjoint bytes), CUDA events."""
    import torch
    from paper_1906_11633_b300 import scenegen as sg
    mat_t, light_t, ev_t = sg.perturb_params(batch, SEED)
    dbt = db.with_params(material=torch.from_numpy(mat_t).to(r.device), light=torch.from_numpy(light_t).to(r.device),
                         exposure_ev=torch.from_numpy(ev_t).to(r.device))
    target = r.render(dbt, rgb_linear=True)["rgb_linear"].clone()
    out = r.render(db, rgb_linear=True, gbuffer=True)
    stream = torch.cuda.current_stream(r.device)
    d = 2.0 * (out["rgb_linear"] - target)
    for _ in range(warmup):
        r.render(db, out=out, rgb_linear=True, gbuffer=True)
        r.shade_backward(db, out["gbuffer"], d)
    torch.cuda.synchronize()
    fw, bw = [], []
    for _ in range(reps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        r.render(db, out=out, rgb_linear=True, gbuffer=True)
        e[1].record(stream)
        r.shade_backward(db, out["gbuffer"], d)
        e[2].record(stream)
        fw.append(e[:2])
        bw.append(e[1:])
    torch.cuda.synchronize()
    fms = float(np.mean([a.elapsed_time(b) for a, b in fw]))
    bms = float(np.mean([a.elapsed_time(b) for a, b in bw]))
    # 40 B per pixel read (G-buffer 28 B + dL/drgb 12 B), the gradient rows written
    bw_bytes = batch.total_pixels * (7 * 4 + 12) + batch.n_samples * (128 + 16 + 1) * 4
    return fms, bms, bw_bytes


def run_diff(args, world, rank, local):
    """Forward with G-buffer + shading adjoint for 256 hand samples (L2 loss against perturbed-parameter targets)."""
    import torch
    from paper_1906_11633_b300 import scenegen as sg
    from paper_1906_11633_b300.render import Renderer
    torch.cuda.set_device(local)
    batch = sg.hand_batch(SEED, shard_samples(rank, world, N_SAMPLES), res=RES, n_cams=N_CAMS)
    r = Renderer(batch.meshes, device=local)
    db = r.upload(batch)
    fms, bms, bw_bytes = time_diff(r, db, batch, max(5, args.steps // 10), args.warmup)
    if rank != 0:
        return
    peaks, _ = load_peaks()
    line = {"workload": "diff", "metric": "samples/s, forward with G-buffer + shading adjoint",
            "value": world * N_SAMPLES / ((fms + bms) / 1e3), "unit": UNIT, "n_gpus": world,
            "forward_ms": fms, "backward_ms": bms, "backward_samples_per_s": N_SAMPLES / (bms / 1e3),
            "roofline_backward": {"bound": "hbm", "achieved": bw_bytes / (bms / 1e3) / 1e9,
                                  "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                                  "frac": bw_bytes / (bms / 1e3) / 1e9 / float(peaks["hbm_gbs"]),
                                  "alg_bytes_per_launch": bw_bytes},
            "config": {"samples": N_SAMPLES, "cameras": N_CAMS, "resolution": RES}}
    print(json.dumps(line), flush=True)


def _timed_renders(r, db, args, world, **kw):
    """Mean kernel time (ms, max over ranks) of one render of `db`, L2 flushed before each timed launch."""
    import torch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=r.device)
    stream = torch.cuda.current_stream()
    out = r.render(db, **kw)
    for _ in range(args.warmup):
        r.render(db, out=out)
    torch.cuda.synchronize()
    evs = []
    for _ in range(max(10, args.steps // 10)):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.render(db, out=out)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in evs])), world)


def run_grade(args, world, rank, local):
    """The hand batch with the colour-grading epilogue of the rgb channel (per-sample hue, saturation,
    contrast, brightness, white balance and grain): kernel time against the same batch ungraded."""
    import torch
    from paper_1906_11633_b300 import scenegen as sg
    from paper_1906_11633_b300.render import Renderer
    torch.cuda.set_device(local)
    batch = sg.hand_batch(SEED, shard_samples(rank, world, N_SAMPLES), res=RES, n_cams=N_CAMS, grading=True)
    r = Renderer(batch.meshes, device=local)
    graded = r.upload(batch)
    plain = graded.with_params(grading=None)
    gms, pms = _timed_renders(r, graded, args, world), _timed_renders(r, plain, args, world)
    if rank != 0:
        return
    line = {"workload": "grade", "metric": "samples/s with the colour-grading epilogue",
            "value": world * N_SAMPLES / (gms / 1e3), "unit": UNIT, "n_gpus": world, "ms_per_step": gms,
            "ungraded_ms_per_step": pms, "overhead": gms / pms - 1.0, "device_status": r.status(),
            "config": {"samples": N_SAMPLES, "cameras": N_CAMS, "resolution": RES,
                       "grading": "hue U(+-0.1) rad, saturation and contrast U[0.8, 1.2], brightness U(+-0.05), "
                                  "temperature and tint U(+-0.1), grain U[0, 0.05]"}}
    print(json.dumps(line), flush=True)


def run_track(args, world, rank, local):
    """The hand batch with the tracker rows (screen box and projected origin of every instance in every
    image, folded in by the vertex stage): kernel time against the same batch without them."""
    import torch
    from paper_1906_11633_b300 import scenegen as sg
    from paper_1906_11633_b300.render import Renderer
    torch.cuda.set_device(local)
    batch = sg.hand_batch(SEED, shard_samples(rank, world, N_SAMPLES), res=RES, n_cams=N_CAMS)
    r = Renderer(batch.meshes, device=local)
    db = r.upload(batch)
    tms, pms = _timed_renders(r, db, args, world, tracker=True), _timed_renders(r, db, args, world)
    if rank != 0:
        return
    line = {"workload": "track", "metric": "samples/s with the tracker rows",
            "value": world * N_SAMPLES / (tms / 1e3), "unit": UNIT, "n_gpus": world, "ms_per_step": tms,
            "untracked_ms_per_step": pms, "overhead": tms / pms - 1.0, "device_status": r.status(),
            "config": {"samples": N_SAMPLES, "cameras": N_CAMS, "resolution": RES,
                       "rows": f"one per camera and instance ({batch.n_inst // batch.n_samples} instances per sample), "
                               "8 int32 each"}}
    print(json.dumps(line), flush=True)


def run_spot(args, world, rank, local):
    """The hand scene lit and coloured like the paper's benchmark scene: three spot lights (LightSetup
    placement, LightRandomizer levels and cones), FixedHue block materials with emission, jittered
    cameras and grading; kernel time against the hand batch with its 1-4 point lights."""
    import torch
    from paper_1906_11633_b300 import scenegen as sg
    from paper_1906_11633_b300.render import Renderer
    torch.cuda.set_device(local)
    ids = shard_samples(rank, world, N_SAMPLES)
    bench = sg.benchmark_batch(SEED, ids, res=RES, n_cams=N_CAMS)
    r = Renderer(bench.meshes, device=local)
    sms = _timed_renders(r, r.upload(bench), args, world)
    pms = _timed_renders(r, r.upload(sg.hand_batch(SEED, ids, res=RES, n_cams=N_CAMS)), args, world)
    if rank != 0:
        return
    line = {"workload": "spot", "metric": "samples/s, benchmark-like lighting (3 spot lights, emission, grading)",
            "value": world * N_SAMPLES / (sms / 1e3), "unit": UNIT, "n_gpus": world, "ms_per_step": sms,
            "point_lit_ms_per_step": pms, "overhead": sms / pms - 1.0, "device_status": r.status(),
            "config": {"samples": N_SAMPLES, "cameras": N_CAMS, "resolution": RES,
                       "lights": "3 spot lights, outer half-angle U[25, 45] deg, inner (0.6-0.9) x outer, "
                                 "total intensity U[0.5, 1] split by weights U[0.5, 1]",
                       "materials": "block faces FixedHue (HSV radius 0.03/0.15/0.15, emissive p = 0.15)",
                       "grading": True}}
    print(json.dumps(line), flush=True)


def run_shadow(args, world, rank, local):
    """The benchmark-like scene with its soft shadows: three shadow-casting spot lights, each with a
    256 x 256 shadow map rendered every step (its own depth-only launch over the back faces) and a
    3 x 3 percentage-closer lookup per pixel and light; kernel time of both launches against the
    same scene without shadows."""
    import torch
    from paper_1906_11633_b300 import scenegen as sg
    from paper_1906_11633_b300.render import Renderer
    torch.cuda.set_device(local)
    ids = shard_samples(rank, world, N_SAMPLES)
    bench = sg.benchmark_batch(SEED, ids, res=RES, n_cams=N_CAMS, shadow_res=SHADOW_RES)
    r = Renderer(bench.meshes, device=local)
    db = r.upload(bench)
    sms = _timed_renders(r, db, args, world)
    nms = _timed_renders(r, r.upload(bench.with_params(shadow_view=None, shadow_intr=None, shadow_res=0)), args, world)
    if rank != 0:
        return
    n_maps = int((bench.light_meta[:, 0]).sum())
    line = {"workload": "shadow", "metric": "samples/s, benchmark-like scene with shadow-casting spot lights",
            "value": world * N_SAMPLES / (sms / 1e3), "unit": UNIT, "n_gpus": world, "ms_per_step": sms,
            "unshadowed_ms_per_step": nms, "overhead": sms / nms - 1.0, "device_status": r.status(),
            "gpu_launches_per_step": 3,
            "config": {"samples": N_SAMPLES, "cameras": N_CAMS, "resolution": RES, "shadow_maps": n_maps,
                       "shadow_res": SHADOW_RES, "pcf": "3x3 taps", "lights": "3 spot lights", "grading": True}}
    print(json.dumps(line), flush=True)


def run_cube(args, world, rank, local):
    """The hand scene with its 1-4 point lights casting cube-map shadows (six 128 x 128 faces per
    light, rendered every step); kernel time against the same batch without shadows."""
    import torch
    from paper_1906_11633_b300 import scenegen as sg
    from paper_1906_11633_b300.render import Renderer
    torch.cuda.set_device(local)
    ids = shard_samples(rank, world, N_SAMPLES)
    batch = sg.hand_batch(SEED, ids, res=RES, n_cams=N_CAMS, shadow_res=CUBE_RES)
    r = Renderer(batch.meshes, device=local)
    sms = _timed_renders(r, r.upload(batch), args, world)
    nms = _timed_renders(r, r.upload(batch.with_params(shadow_view=None, shadow_intr=None, shadow_res=0)), args, world)
    if rank != 0:
        return
    n_maps = int(batch.light_meta[:, 0].sum()) * 6
    line = {"workload": "cube", "metric": "samples/s, hand scene with cube-map shadows of its point lights",
            "value": world * N_SAMPLES / (sms / 1e3), "unit": UNIT, "n_gpus": world, "ms_per_step": sms,
            "unshadowed_ms_per_step": nms, "overhead": sms / nms - 1.0, "device_status": r.status(),
            "gpu_launches_per_step": 3,
            "config": {"samples": N_SAMPLES, "cameras": N_CAMS, "resolution": RES, "shadow_maps": n_maps,
                       "shadow_res": CUBE_RES, "faces_per_light": 6, "pcf": "3x3 taps"}}
    print(json.dumps(line), flush=True)


def run_serve(args, world, rank, local):
    """Poisson arrivals at 2000 req/s of 1-64-sample hand requests at {64,128,200,256} px, 1-3 cameras."""
    line = measure_serve(args.serve_seconds, world, rank, local)
    if line is not None:
        print(json.dumps(line), flush=True)


def measure_serve(seconds, world, rank, local):
    """The serving workload's JSON line for `seconds` of arrivals (rank 0; None on the others)."""
    import torch
    from paper_1906_11633_b300 import scenegen as sg
    from paper_1906_11633_b300.serve import GpuBackend, Server, run_poisson
    torch.cuda.set_device(local)
    rate, dur = 2000.0, seconds
    reqs = sg.poisson_requests(SEED + rank, rate, dur)
    meshes = sg.hand_meshes()
    t0 = time.perf_counter()
    batches = [sg.request_batch(SEED, q, meshes=meshes) for q in reqs]
    gen_s = time.perf_counter() - t0
    be = GpuBackend(meshes, device=local, n_streams=2)
    # warm the path (workspace and output sizes in torch's allocator) with half a second of other
    # arrivals at the same rate first
    wreqs = sg.poisson_requests(SEED + 1000 + rank, rate, 0.5)
    wbatches = [sg.request_batch(SEED + 1000, q, meshes=meshes) for q in wreqs]
    warm = Server(be, n_streams=2, max_inflight=4, tick_ms=2.0)
    run_poisson(warm, wreqs, wbatches, 0.5, keep_results=False)
    warm.close()
    del wreqs, wbatches, warm
    # the requests' arrays are long-lived: move them out of the collector's generations so that a
    # full collection during the run does not scan them (the usual set-up of a Python server)
    import gc
    gc.collect()
    gc.freeze()
    try:
        srv = Server(be, n_streams=2, max_inflight=4, tick_ms=2.0)
        subs, wall = run_poisson(srv, reqs, batches, dur, keep_results=False)
        st = srv.stats(wall)
        srv.close()
    finally:
        gc.unfreeze()
    if rank != 0:
        return None
    line = {"workload": "serve", "metric": "samples/s and request latency under Poisson arrivals",
            "value": st["samples_per_s"], "unit": UNIT, "n_gpus": world,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
            "requests": st["requests"], "samples": st["samples"], "batches": st["batches"],
            "max_concurrent_batches": st["max_concurrent_batches"], "memory_waits": st["memory_waits"],
            "config": {"rate_hz": rate, "seconds": dur, "tick_ms": 2.0, "streams": 2, "max_inflight": 4,
                       "request_samples": "U{1..64}", "resolution": list(sg.SERVE_RES), "cameras": "U{1..3}",
                       "host_generation_s": gen_s, "gc": "collected and frozen before the run",
                       "client": "drops each request's outputs once it has completed"}}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tile-w", type=int, default=0)
    ap.add_argument("--tile-h", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the fused kernel from an ncu capture of the same kernel source")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-patterns", action="store_true",
                    help="headline: skip the short uneven-batch and serving measurements")
    ap.add_argument("--workload", choices=["hand", "uneven", "diff", "serve", "grade", "track", "spot", "shadow", "cube"], default="hand",
                    help="hand: the headline line; the others print supplementary lines")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--samples", type=int, default=N_SAMPLES,
                    help="hand samples per step (smaller batches for profiler captures; the headline is 256)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.samples != N_SAMPLES:
        set_samples(args.samples)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "uneven":
        run_uneven(args, world, rank, local)
    elif args.workload == "diff":
        run_diff(args, world, rank, local)
    elif args.workload == "serve":
        run_serve(args, world, rank, local)
    elif args.workload == "grade":
        run_grade(args, world, rank, local)
    elif args.workload == "track":
        run_track(args, world, rank, local)
    elif args.workload == "spot":
        run_spot(args, world, rank, local)
    elif args.workload == "shadow":
        run_shadow(args, world, rank, local)
    elif args.workload == "cube":
        run_cube(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
