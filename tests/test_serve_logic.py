"""Scheduling logic of the continuous-batching server with a fake backend (no GPU).

Checks: every request completes exactly once, in-flight batches never exceed
the slot count or the memory budget, batches overlap (more than one in flight)
when requests keep arriving, and a request larger than the budget is never
admitted alongside others that would overflow it, and a request that could never
fit the budget fails alone instead of blocking the queue behind it.
"""

import threading
import time

from paper_1906_11633_b300 import scenegen as sg
from paper_1906_11633_b300.serve import Server, ServeRequest


class FakeBackend:
    def __init__(self, gpu_ms=4.0, budget=10_000_000):
        self.gpu_ms = gpu_ms
        self.budget = budget
        self.lock = threading.Lock()
        self.active_bytes = 0
        self.peak_bytes = 0
        self.active = 0
        self.peak_active = 0

    def memory_budget(self):
        return self.budget

    def bytes_needed(self, batches):
        return sum(b.total_pixels for b in batches) * 14

    def launch(self, batches, k):
        nb = self.bytes_needed(batches)
        with self.lock:
            self.active_bytes += nb
            self.active += 1
            self.peak_bytes = max(self.peak_bytes, self.active_bytes)
            self.peak_active = max(self.peak_active, self.active)
        return {"t_end": time.perf_counter() + self.gpu_ms / 1e3, "batches": batches, "nb": nb}

    def wait(self, h):
        d = h["t_end"] - time.perf_counter()
        if d > 0:
            time.sleep(d)
        return [{"n": b.n_samples} for b in h["batches"]]

    def release(self, h):
        with self.lock:
            self.active_bytes -= h["nb"]
            self.active -= 1


def _req_batch(i, n, res):
    return sg.hand_batch(0, range(1000 * i, 1000 * i + n), res=res, n_cams=1)


def test_every_request_completes_within_budget_and_batches_overlap():
    be = FakeBackend(gpu_ms=6.0, budget=64 * 64 * 14 * 40)
    srv = Server(be, n_streams=2, max_inflight=3, tick_ms=1.0)
    batches = [_req_batch(i, 1 + i % 4, 64) for i in range(40)]
    reqs = []
    for i in range(40):
        reqs.append(srv.submit(ServeRequest(i, batches[i])))
        time.sleep(0.0015)
    for r in reqs:
        assert r.event.wait(10.0)
    st = srv.stats(1.0)
    srv.close()
    assert st["requests"] == 40 and len({rid for rid, _, _ in srv.completed}) == 40
    assert all(r.result["n"] == r.batch.n_samples for r in reqs)
    assert be.peak_bytes <= be.budget
    assert 2 <= be.peak_active <= 3
    assert st["batches"] < 40              # requests were batched together
    assert all(r.latency_ms > 0 for r in reqs)


def test_memory_budget_serialises_large_batches():
    one = 128 * 128 * 14 * 8
    be = FakeBackend(gpu_ms=3.0, budget=one)                # room for one 8-sample 128px request at a time
    srv = Server(be, n_streams=2, max_inflight=4, tick_ms=1.0)
    batches = [_req_batch(i, 8, 128) for i in range(5)]
    reqs = [srv.submit(ServeRequest(i, b)) for i, b in enumerate(batches)]
    for r in reqs:
        assert r.event.wait(10.0)
    srv.close()
    assert be.peak_bytes <= one and be.peak_active == 1


class FaultyBackend(FakeBackend):
    """Fails the launch of batch `launch_fail` and the wait of batch `wait_fail` (counting from 0),
    as a render call that returns an error code or a device status word would."""

    def __init__(self, launch_fail, wait_fail, **kw):
        super().__init__(**kw)
        self.launch_fail, self.wait_fail, self.n = launch_fail, wait_fail, 0

    def launch(self, batches, k):
        i, self.n = self.n, self.n + 1
        if i == self.launch_fail:
            raise RuntimeError("launch error code")
        h = super().launch(batches, k)
        h["i"] = i
        return h

    def wait(self, h):
        res = super().wait(h)
        if h["i"] == self.wait_fail:
            raise RuntimeError("device status 0x40")
        return res


def test_failed_batches_fail_their_requests_and_the_server_goes_on():
    be = FaultyBackend(launch_fail=1, wait_fail=3, gpu_ms=2.0)
    srv = Server(be, n_streams=2, max_inflight=2, tick_ms=1.0, max_batch_samples=4)
    reqs = []
    for i in range(24):
        reqs.append(srv.submit(ServeRequest(i, _req_batch(i, 2, 32))))
        time.sleep(0.002)
    for r in reqs:
        assert r.event.wait(10.0), f"request {r.rid} never finished"
    srv.close()
    failed = [r for r in reqs if r.error]
    ok = [r for r in reqs if not r.error]
    assert failed and any("launch" in r.error for r in failed) and any("render" in r.error for r in failed)
    assert all(r.result is None for r in failed) and all(r.result is not None for r in ok)
    assert len(ok) + len(failed) == 24 and len(ok) >= 16         # later batches still ran
    assert srv.inflight_bytes == 0 and be.active_bytes == 0
    st = srv.stats(1.0)
    assert st["failed"] == len(failed) and st["requests"] == len(ok)


def test_request_larger_than_the_whole_budget_fails_and_the_queue_moves_on():
    small = 64 * 64 * 14                      # one 64 x 64 image
    be = FakeBackend(gpu_ms=2.0, budget=4 * small)
    srv = Server(be, n_streams=2, max_inflight=2, tick_ms=1.0)
    big = srv.submit(ServeRequest(0, _req_batch(0, 8, 64)))        # 8 images: twice the budget
    rest = [srv.submit(ServeRequest(i, _req_batch(i, 1, 64))) for i in range(1, 9)]
    for r in [big] + rest:
        assert r.event.wait(10.0), f"request {r.rid} never finished"
    srv.close()
    assert big.error and "does not fit" in big.error and big.result is None
    assert all(r.error is None and r.result is not None for r in rest)
    assert be.peak_bytes <= 4 * small and srv.inflight_bytes == 0
    assert srv.stats(1.0)["failed"] == 1


class SlowLaunchBackend(FakeBackend):
    """A launch that takes long on the host (packing, copies): the request is out of the pending
    queue but not yet in flight while it runs."""

    def launch(self, batches, k):
        time.sleep(0.2)
        return super().launch(batches, k)


def test_close_waits_for_a_batch_that_is_still_launching():
    be = SlowLaunchBackend(gpu_ms=1.0)
    srv = Server(be, n_streams=2, max_inflight=2, tick_ms=1.0)
    req = srv.submit(ServeRequest(0, _req_batch(0, 2, 32)))
    deadline = time.perf_counter() + 5.0
    while srv.pending and time.perf_counter() < deadline:   # the scheduler has taken it ...
        time.sleep(0.001)
    assert not srv.pending and not req.event.is_set()        # ... and is inside the launch
    srv.close()
    assert req.event.is_set() and req.error is None and req.result == {"n": 2}
    assert be.active == 0


def test_param_stage_packs_every_array_at_aligned_offsets():
    """The serving backend's parameter stage: every array of a packed batch (optional arrays
    included) lands at a 256-byte aligned offset of one buffer and comes back as a view holding
    exactly its bytes (CPU tensors stand in for the pinned and device buffers)."""
    import numpy as np
    import torch
    from paper_1906_11633_b300.render import host_arrays
    from paper_1906_11633_b300.serve import ParamStage
    meshes = sg.hand_meshes()
    parts = [sg.hand_batch(3, np.arange(0, 2), res=64, meshes=meshes),
             sg.benchmark_batch(4, np.arange(2, 5), res=64, n_cams=2, meshes=meshes, shadow_res=32)]
    arrs = host_arrays(sg.concat_batches(parts))
    assert {"grading", "light_spot", "emission", "shadow_view", "shadow_intr"} <= set(arrs)
    offs, nbytes = ParamStage.layout(arrs)
    assert all(o % 256 == 0 for o in offs.values()) and nbytes % 256 == 0
    spans = sorted((offs[n], offs[n] + a.nbytes) for n, a in arrs.items())
    assert all(e <= b for (_, e), (b, _) in zip(spans, spans[1:]))      # no overlap
    stage = ParamStage.__new__(ParamStage)
    stage.host = torch.zeros(nbytes + 512, dtype=torch.uint8)
    stage.dev = torch.full((nbytes + 512,), 0xAB, dtype=torch.uint8)
    stage.host_np = stage.host.numpy()
    t = stage.upload(torch, arrs, offs, nbytes, None)
    for n, a in arrs.items():
        assert t[n].numel() == a.size and t[n].numpy().dtype == a.dtype, n
        assert t[n].numpy().tobytes() == a.tobytes(), n
    assert (stage.dev[nbytes:] == 0xAB).all()                            # nothing written past the layout
