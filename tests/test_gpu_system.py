"""Batched launch under a CUDA graph, the autotuner, and the continuous-batching server (GPU).

- a captured graph replays to the same channels as a direct render, and again after new
  batch contents of the same shapes are copied in;
- the uneven batch (mixed triangle counts and resolutions) renders in one persistent launch
  and matches per-scene plain launches and batch-wide staged launches (in chunks when the
  scratch slots do not all fit) bit for bit;
- the autotuner returns a configuration whose output equals the default's and caches it;
- served requests: each result equals the same request rendered alone, and batches overlap.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_11633_b300 import lib as L
from paper_1906_11633_b300 import scenegen as sg
from paper_1906_11633_b300.render import GraphRender, Renderer, config, to_numpy


@pytest.fixture(scope="module")
def renderer():
    return Renderer(sg.hand_meshes())


def _equal(a, b, batch=None):
    """Channel by channel; shadow maps only where a light casts (the others are left as they were)."""
    for k in a:
        x, y = to_numpy({k: a[k]})[k], to_numpy({k: b[k]})[k]
        if k == "shadow_map":
            cast = (np.arange(4)[None, :, None] < batch.light_meta[:, :1, None]) & (batch.shadow_intr[..., 0] != 0)
            assert cast.any()
            x, y = x[cast], y[cast]
        np.testing.assert_array_equal(x, y, err_msg=k)


def test_graph_replay_matches_direct_render_and_takes_new_contents(renderer):
    b1 = sg.hand_batch(1, np.arange(8), res=128)
    b2 = sg.hand_batch(2, np.arange(8), res=128)
    g = GraphRender(renderer, renderer.upload(b1))
    out = g.replay()
    torch.cuda.synchronize()
    _equal(out, renderer.render(renderer.upload(b1)))
    g.update(b2)
    out = g.replay()
    torch.cuda.synchronize()
    _equal(out, renderer.render(renderer.upload(b2)))


def test_graph_replay_with_shadow_maps(renderer):
    """A shadowed batch is several launches (shadow pass, the maps' neighbourhood table, cameras)
    and a queue reset; its captured graph replays them, maps included, and takes new contents."""
    b1 = sg.benchmark_batch(3, np.arange(6), res=96, shadow_res=128)
    b2 = sg.benchmark_batch(4, np.arange(6), res=96, shadow_res=128)
    g = GraphRender(renderer, renderer.upload(b1))
    assert "shadow_map" in g.out
    out = g.replay()
    torch.cuda.synchronize()
    _equal(out, renderer.render(renderer.upload(b1)), b1)
    g.update(b2)
    out = g.replay()
    torch.cuda.synchronize()
    _equal(out, renderer.render(renderer.upload(b2)), b2)


def test_uneven_batch_in_one_launch_matches_plain_launches(renderer):
    b = sg.uneven_batch(3, np.arange(48))
    db = renderer.upload(b)
    g = GraphRender(renderer, db)
    fused = g.replay()
    torch.cuda.synchronize()
    plain = renderer.render(db, cfg=config(mode=L.ORRB_MODE_PLAIN))
    torch.cuda.synchronize()
    assert renderer.status() == 0
    _equal(fused, plain)
    staged = renderer.render(db, cfg=config(mode=L.ORRB_MODE_STAGED))  # (every image in one chunk)
    torch.cuda.synchronize()
    assert renderer.status() == 0
    _equal(fused, staged)


def test_autotuner_result_is_valid_and_cached(renderer, tmp_path):
    from paper_1906_11633_b300.tune import tune
    b = sg.hand_batch(4, np.arange(16), res=200)
    db = renderer.upload(b)
    cands = [(256, 1, 512), (64, 2, 512), (32, 4, 256), (512, 64, 512)]   # the last cannot fit
    path = str(tmp_path / "tune.json")
    cfg, timings = tune(renderer, db, candidates=cands, reps=2, cache_path=path)
    assert (cfg.tile_w, cfg.tile_h, cfg.threads) in cands[:3]
    assert "512x64x512" not in timings and len(timings) == 3
    cfg2, _ = tune(renderer, db, candidates=cands, reps=2, cache_path=path)
    assert (cfg2.tile_w, cfg2.tile_h, cfg2.threads) == (cfg.tile_w, cfg.tile_h, cfg.threads)
    _equal(renderer.render(db, cfg=cfg), renderer.render(db))


@pytest.mark.parametrize("n_stages,stage_bytes", [(4, 8 << 20), (1, 16 << 10)])
def test_served_requests_equal_their_solo_render(n_stages, stage_bytes):
    """Requests batched together equal their solo renders; with one 16 KB parameter stage the
    backend makes larger stages as batches need them, and every stage is back after the run."""
    from paper_1906_11633_b300.serve import GpuBackend, Server, ServeRequest
    meshes = sg.hand_meshes()
    be = GpuBackend(meshes, n_streams=2, n_stages=n_stages, stage_bytes=stage_bytes)
    srv = Server(be, n_streams=2, max_inflight=4, tick_ms=2.0)
    rng = np.random.default_rng(0)
    batches = []
    first = 0
    for i in range(40):
        n = int(rng.integers(1, 7))
        batches.append(sg.hand_batch(7, np.arange(first, first + n), res=int(rng.choice([64, 128])),
                                     n_cams=int(rng.integers(1, 4)), meshes=meshes))
        first += n
    reqs = [srv.submit(ServeRequest(i, b)) for i, b in enumerate(batches)]
    for r in reqs:
        assert r.event.wait(60.0)
    st = srv.stats(1.0)
    srv.close()
    assert st["requests"] == 40
    assert st["batches"] < 40                       # requests were batched together
    caps = sorted(stg.capacity for stg in be._stages)
    if n_stages == 4:
        assert caps == [8 << 20] * 4                # the preallocated stages sufficed and all came back
    else:
        assert len(caps) >= 2 and caps[-1] > 16 << 10
    solo = Renderer(meshes)
    for r in reqs[::7]:
        alone = solo.render(solo.upload(r.batch))
        torch.cuda.synchronize()
        _equal(r.result, alone)


@pytest.mark.parametrize("shadows", [False, True])
def test_capture_pipeline_results_match_direct_renders(renderer, shadows):
    """Round-robin slots with bulk readback equal direct renders; with shadow maps the maps come
    back with the channels."""
    from paper_1906_11633_b300.render import CapturePipeline
    if shadows:
        batches = [sg.benchmark_batch(20 + k, np.arange(4), res=80, shadow_res=96) for k in range(3)]
    else:
        batches = [sg.hand_batch(20 + k, np.arange(6), res=96) for k in range(3)]
    pipe = CapturePipeline(renderer, batches[0], depth=2)
    handles = [pipe.submit(CapturePipeline.pin(b)) for b in batches[:2]]
    got0 = {k: v.clone() for k, v in CapturePipeline.result(handles[0]).items()}
    handles.append(pipe.submit(CapturePipeline.pin(batches[2])))     # reuses slot 0 after its readback
    got = [got0] + [{k: v.clone() for k, v in CapturePipeline.result(h).items()} for h in handles[1:]]
    for b, g in zip(batches, got):
        ref = renderer.render(renderer.upload(b))
        torch.cuda.synchronize()
        for k in ref:
            # (maps of lights that cast no shadow are left as they were: compare the casting ones)
            keep = np.arange(4)[None, :] < b.light_meta[:, :1] if k == "shadow_map" else slice(None)
            np.testing.assert_array_equal(g[k].numpy()[keep], ref[k].cpu().numpy()[keep], err_msg=k)


def test_served_shadowed_requests_equal_their_solo_render():
    """Requests with shadow maps batched together: each one's channels and the maps of its own
    samples equal its render alone."""
    from paper_1906_11633_b300.serve import GpuBackend, Server, ServeRequest
    meshes = sg.hand_meshes()
    be = GpuBackend(meshes, n_streams=2)
    srv = Server(be, n_streams=2, max_inflight=2, tick_ms=5.0)
    batches = [sg.benchmark_batch(11, np.arange(3 * i, 3 * i + 1 + i % 3), res=64, n_cams=2, meshes=meshes,
                                  shadow_res=64) for i in range(6)]
    reqs = [srv.submit(ServeRequest(i, b)) for i, b in enumerate(batches)]
    for r in reqs:
        assert r.event.wait(60.0)
    st = srv.stats(1.0)
    srv.close()
    assert st["requests"] == 6 and st["batches"] < 6
    solo = Renderer(meshes)
    for r in reqs:
        alone = solo.render(solo.upload(r.batch))
        torch.cuda.synchronize()
        cast = np.arange(4)[None, :] < r.batch.light_meta[:, :1]
        for k in alone:
            keep = cast if k == "shadow_map" else slice(None)
            np.testing.assert_array_equal(to_numpy({k: r.result[k]})[k][keep], to_numpy({k: alone[k]})[k][keep],
                                          err_msg=k)


def test_served_requests_with_bad_input_fail_alone():
    """Two bad requests among good ones, each in a batch of its own: one names a mesh that does not
    exist (the host cannot size it: it fails before launch), one has a light count beyond the
    maximum (the kernel clamps it and flags the status word, and the loop fails the batch with
    that status).  The requests around them are rendered as usual."""
    from paper_1906_11633_b300.serve import GpuBackend, Server, ServeRequest
    meshes = sg.hand_meshes()
    be = GpuBackend(meshes, n_streams=2)
    srv = Server(be, n_streams=2, max_inflight=2, tick_ms=1.0, max_batch_samples=2)
    batches = [sg.hand_batch(9, np.arange(2 * i, 2 * i + 2), res=64, n_cams=2, meshes=meshes) for i in range(6)]
    bad_mesh = batches[1].inst_mesh.copy()
    bad_mesh[5] = 999
    batches[1] = batches[1].with_params(inst_mesh=bad_mesh)
    bad_lights = batches[3].light_meta.copy()
    bad_lights[0, 0] = 9
    batches[3] = batches[3].with_params(light_meta=bad_lights)
    reqs = [srv.submit(ServeRequest(i, b)) for i, b in enumerate(batches)]
    for r in reqs:
        assert r.event.wait(60.0)
    srv.close()
    assert reqs[1].error is not None and reqs[1].error.startswith("invalid request")
    assert reqs[3].error is not None and "device status 0x10" in reqs[3].error and reqs[3].result is None
    assert all(r.error is None and r.result is not None for i, r in enumerate(reqs) if i not in (1, 3))
    solo = Renderer(meshes)
    alone = solo.render(solo.upload(batches[4]))
    torch.cuda.synchronize()
    _equal(reqs[4].result, alone)


def test_staged_chunks_match_the_fused_launch(renderer):
    """The uneven batch's 2,072 images in the staged mode: with up to 50k triangles per scene the
    scratch slots do not all fit in the staged mode's budget, so the launches run over chunks of
    the images; every channel equals the fused launch's bit for bit (compared on the device)."""
    b = sg.uneven_batch(0, np.arange(1024))
    db = renderer.upload(b)
    fused = renderer.render(db)
    staged = renderer.render(db, cfg=config(mode=L.ORRB_MODE_STAGED))
    torch.cuda.synchronize()
    assert renderer.status() == 0
    # the plain mode holds one slot per camera of a scene: its workspace gives a slot's size
    per_scene = int(db.shape.max_cams_per_sample)
    slot = (L.orrb_workspace_size(renderer.ctx, db.shape, config(mode=L.ORRB_MODE_PLAIN)) - 256) // per_scene
    chunk = (L.orrb_workspace_size(renderer.ctx, db.shape, config(mode=L.ORRB_MODE_STAGED)) - 256) // slot
    assert 0 < chunk < b.n_cams  # several chunks
    for k in fused:
        assert torch.equal(fused[k], staged[k]), k
