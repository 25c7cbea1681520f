"""Bounded device waits made to run out on purpose (GPU).

The persistent launch has two kinds of wait between CTAs: a CTA that has no image left looks for
raster tiles of other CTAs' images to help with, and an image's owner waits for the helpers still
on its tiles.  Each gives up after orrb_config.wait_cycles SM cycles, sets ORRB_DEV_TIMEOUT in the
status word and leaves the launch.  A budget of one cycle makes them give up at once: the launch
must still return, report the timeout through the status word (the render API) and as a failed
request (the serving loop), and leave the context usable: the same batch rendered again with the
default budget matches the oracle.  No wait is left without a limit and nothing faults: the test
only shortens the limit.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_11633_b300 import lib as L
from paper_1906_11633_b300 import scenegen as sg
from paper_1906_11633_b300.render import Renderer, config, to_numpy


def _timeout_batch():
    # images of two sizes: CTAs that own a small image finish early and look for help while the
    # large images are still in their geometry phase, so a one-cycle search finds nothing
    small = sg.hand_batch(5, np.arange(6), res=32, n_cams=2)
    large = sg.hand_batch(6, np.arange(6, 8), res=256, n_cams=2)
    return sg.concat_batches([small, large])


def test_one_cycle_budget_times_out_and_the_context_stays_usable(oracle):
    b = _timeout_batch()
    r = Renderer(b.meshes)
    db = r.upload(b)
    out = r.render(db, cfg=config(wait_cycles=1))
    torch.cuda.synchronize()                       # the launch returned
    st = r.status()
    assert st & L.ORRB_DEV_TIMEOUT, f"status {st:#x}"
    assert (st & ~L.ORRB_DEV_TIMEOUT) == 0         # nothing else was flagged
    # the default budget renders the same batch in full
    good = to_numpy(r.render(db))
    torch.cuda.synchronize()
    assert r.status() == 0
    o = oracle.render(b)
    assert (good["seg"] == o["seg"]).all()
    assert (good["depth"] == o["depth"]).all()
    assert np.abs(good["rgb"].astype(int) - o["rgb"].astype(int)).max() <= 1
    del out


def test_serving_loop_fails_the_batch_whose_waits_ran_out():
    from paper_1906_11633_b300.serve import GpuBackend, Server, ServeRequest
    b = _timeout_batch()
    be = GpuBackend(b.meshes, n_streams=1, cfg=config(wait_cycles=1))
    srv = Server(be, n_streams=1, max_inflight=1, tick_ms=1.0)
    req = srv.submit(ServeRequest(0, b))
    assert req.event.wait(60.0)
    srv.close()
    assert req.result is None and req.error is not None
    assert f"device status {L.ORRB_DEV_TIMEOUT:#x}" in req.error, req.error
