"""Tile-shape autotuner for the fused render launch.

Every configuration renders bit-identical channels (each pixel's result does
not depend on how pixels are grouped into tiles or CTAs), so the tuner only
looks at time: it renders the given batch with each candidate
(tile width x tile height x CTA size), keeps the fastest, and caches the
choice in a JSON file keyed by GPU name and a coarse class of the batch shape
(largest image side, triangles per sample, image count), so a serving loop
or a training job pays the sweep once per class.
"""

from __future__ import annotations

import json
import math
import os
import threading
from typing import Dict, Iterable, Optional, Tuple

import torch

from . import lib as L
from .render import DeviceBatch, Renderer, config

DEFAULT_CANDIDATES: Tuple[Tuple[int, int, int], ...] = (
    (256, 2, 512), (256, 1, 512), (256, 2, 256), (128, 2, 512), (128, 1, 512), (64, 2, 512), (64, 4, 512),
    (32, 4, 512), (512, 1, 256), (512, 2, 256))

_lock = threading.Lock()


def default_cache_path() -> str:
    return os.environ.get("ORRB_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "orrb_tune.json"))


def shape_class(db: DeviceBatch) -> str:
    s = db.shape
    side = max(s.max_width, s.max_height)
    tris = max(1, s.max_tris_per_sample)
    return f"side{1 << math.ceil(math.log2(max(side, 1)))}-tris{1 << math.ceil(math.log2(tris))}-imgs{1 << math.ceil(math.log2(max(s.n_cams, 1)))}"


def cache_key(db: DeviceBatch, device: int) -> str:
    return f"{torch.cuda.get_device_name(device)}|{shape_class(db)}"


def _load(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, data: Dict[str, dict]) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_config(r: Renderer, db: DeviceBatch, cfg: L.orrb_config, out, reps: int = 5, warmup: int = 2) -> float:
    """Mean milliseconds per fused render of `db` under `cfg` (CUDA events on the current stream)."""
    stream = torch.cuda.current_stream(r.device)
    for _ in range(warmup):
        r.render(db, out=out, cfg=cfg)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        r.render(db, out=out, cfg=cfg)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(r: Renderer, db: DeviceBatch, candidates: Optional[Iterable[Tuple[int, int, int]]] = None, reps: int = 5,
         cache_path: Optional[str] = None, use_cache: bool = True) -> Tuple[L.orrb_config, Dict[str, float]]:
    """Fastest fused configuration for `db`; returns (config, {candidate: ms})."""
    path = cache_path or default_cache_path()
    key = cache_key(db, r.device.index or 0)
    if use_cache:
        with _lock:
            hit = _load(path).get(key)
        if hit:
            return config(tile_w=hit["tile_w"], tile_h=hit["tile_h"], threads=hit["threads"]), hit.get("timings", {})
    out = r.alloc_outputs(db.total_pixels)
    timings: Dict[str, float] = {}
    best, best_ms = None, float("inf")
    for tw, th, nt in candidates or DEFAULT_CANDIDATES:
        cfg = config(tile_w=tw, tile_h=th, threads=nt)
        try:
            ms = time_config(r, db, cfg, out, reps=reps)
        except L.OrrbError:
            continue          # does not fit in shared memory for this shape
        timings[f"{tw}x{th}x{nt}"] = ms
        if ms < best_ms:
            best, best_ms = (tw, th, nt), ms
    if best is None:
        raise RuntimeError("no candidate configuration fits this batch")
    with _lock:
        data = _load(path)
        data[key] = {"tile_w": best[0], "tile_h": best[1], "threads": best[2], "ms": best_ms, "timings": timings}
        _store(path, data)
    return config(tile_w=best[0], tile_h=best[1], threads=best[2]), timings
