"""GPU parity of the forward renderer against the CPU oracle, through the C-ABI.

Workloads: the tiny cube scene, the hand-like scene (full 256-sample batch at
200x200 x 3 cameras), the uneven batch (a stratified subset covering every
resolution and both triangle-count extremes), plus ragged, orthographic,
wide (> one tile column), empty and degenerate cases; and invariances that
must hold bit for bit: fused vs plain launches, every tile shape and block
size, a sample alone vs inside a batch.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_11633_b300 import scenegen as sg
from paper_1906_11633_b300 import lib as L
from paper_1906_11633_b300.render import Renderer, config, to_numpy
from tests import scenes
from tests.parity import compare


@pytest.fixture(scope="module")
def oracle():
    from oracle import oracle as orc
    orc.build()
    return orc


@pytest.fixture(scope="module")
def hand_renderer():
    return Renderer(sg.hand_meshes())


@pytest.fixture(scope="module")
def tiny_renderer():
    return Renderer(sg.tiny_meshes())


def render_np(r, batch, cfg=None, **kw):
    out = r.render(r.upload(batch), cfg=cfg, rgb_linear=True, **kw)
    torch.cuda.synchronize()
    assert r.status() == 0, f"device status {r.status():#x}"
    return to_numpy(out)


def test_tiny_matches_oracle(tiny_renderer, oracle):
    b = sg.tiny_batch(0, n_samples=8)
    st = compare(render_np(tiny_renderer, b), oracle.render(b, debug=True), "tiny")
    assert st["depth_exact"] > 0.999


@pytest.mark.parametrize("mode", [L.ORRB_MODE_FUSED, L.ORRB_MODE_PLAIN, L.ORRB_MODE_STAGED])
def test_hand_full_batch_matches_oracle(hand_renderer, oracle, mode):
    b = sg.hand_batch(0, np.arange(256))
    st = compare(render_np(hand_renderer, b, config(mode=mode)), oracle.render(b, debug=True), "hand")
    assert st["pixels"] == 256 * 3 * 200 * 200


def test_uneven_stratified_subset_matches_oracle(hand_renderer, oracle):
    full_layout = sg.uneven_layout(0, np.arange(1024))
    n_links, res, cams = full_layout
    pick = []
    for r in sg.UNEVEN_RES:
        idx = np.nonzero(res == r)[0]
        order = idx[np.argsort(n_links[idx])]
        pick += list(order[:8]) + list(order[-8:]) + list(order[len(order) // 2 - 8:len(order) // 2 + 8])
    pick = np.unique(pick)
    assert len(pick) >= 128
    b = sg.uneven_batch(0, pick)
    assert set(np.unique(b.cam_wh[:, 0])) == set(sg.UNEVEN_RES)
    compare(render_np(hand_renderer, b), oracle.render(b, debug=True), "uneven")


def test_ragged_wide_and_orthographic(oracle):
    meshes = [sg.plane_mesh(3, 3), sg.box_mesh(0.5), sg.capsule_mesh(0.3, 0.8)]
    r = Renderer(meshes)
    poses = [scenes.identity_pose(), scenes.pose(t=(0.2, -0.1, 0.5)),
             scenes.pose(R=sg._rot("z", np.array(0.7)), t=(-0.6, 0.3, 0.9))]
    cams = [scenes.camera_look((2.0, -2.5, 1.8), (0, 0, 0.4), 67, 45, 50.0),      # ragged tiles
            scenes.camera_look((1.0, -3.0, 1.0), (0, 0, 0.4), 600, 40, 30.0),     # two tile columns
            scenes.camera_down((0.05, 0.02, 4.0), 53, 61, px_per_m=17.0),         # orthographic
            scenes.camera_look((0.3, -0.2, 0.05), (0, 0, 0.6), 31, 29, 80.0)]     # near the plane: clipping
    b = scenes.single_sample(meshes, [0, 1, 2], poses, cams, seg=[1, 2, 3], mat_base=[0, 1, 7],
                             lights=[((0.5, -1.0, 2.0), 2.0), ((-1.0, 0.5, 1.5), 1.0)], albedo=(0.6, 0.4, 0.3),
                             specular=0.5, shininess=20.0, ambient=(0.05, 0.05, 0.05), background=(0.2, 0.3, 0.4))
    for tw, th in ((256, 2), (256, 1), (64, 4), (24, 8), (512, 1), (512, 2)):
        compare(render_np(r, b, config(tile_w=tw, tile_h=th, threads=256)), oracle.render(b, debug=True),
                f"ragged tile={tw}x{th}")


def test_empty_scene_and_no_lights(tiny_renderer, oracle):
    b = sg.tiny_batch(3, n_samples=3)
    b = b.with_params(inst_offset=np.array([0, 2, 2, 4], np.int32),
                      inst_mesh=b.inst_mesh[:4], inst_pose=b.inst_pose[:4], inst_seg=b.inst_seg[:4],
                      inst_mat_base=b.inst_mat_base[:4], light_meta=np.array([[1, 1], [1, 1], [0, 1]], np.int32))
    g = render_np(tiny_renderer, b)
    o = oracle.render(b, debug=True)
    compare(g, o, "empty")
    n = 64 * 64
    assert (g["seg"][n:2 * n] == 0).all() and (g["depth"][n:2 * n] == 0).all()


@pytest.mark.parametrize("tile", [(256, 1), (200, 2), (64, 2), (32, 4), (16, 8), (8, 16), (120, 1)])
@pytest.mark.parametrize("threads", [256, 512])
def test_bit_identical_across_tilings_and_modes(hand_renderer, tile, threads):
    b = sg.hand_batch(5, np.arange(6), res=200)
    ref = render_np(hand_renderer, b, config())
    got = render_np(hand_renderer, b, config(tile_w=tile[0], tile_h=tile[1], threads=threads))
    plain = render_np(hand_renderer, b, config(mode=L.ORRB_MODE_PLAIN, tile_w=tile[0], tile_h=tile[1],
                                               threads=threads))
    staged = render_np(hand_renderer, b, config(mode=L.ORRB_MODE_STAGED, tile_w=tile[0], tile_h=tile[1],
                                                threads=threads))
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
        np.testing.assert_array_equal(plain[k], ref[k], err_msg=k)
        np.testing.assert_array_equal(staged[k], ref[k], err_msg=k)


def test_sample_alone_equals_sample_in_batch(hand_renderer):
    b = sg.hand_batch(8, np.arange(12), res=128)
    full = render_np(hand_renderer, b)
    n = 128 * 128 * 3
    for s in (0, 7, 11):
        alone = render_np(hand_renderer, sg.hand_batch(8, [s], res=128))
        for k in full:
            np.testing.assert_array_equal(alone[k], full[k][s * n:(s + 1) * n], err_msg=k)


def test_device_checks_flag_bad_input(hand_renderer):
    b = sg.hand_batch(1, np.arange(2), res=64)
    ok = hand_renderer.upload(b)
    bad_mesh = ok.tensors["inst_mesh"].clone()
    bad_mesh[3] = 999                                   # no such mesh: the kernel skips the instance
    hand_renderer.render(ok.with_params(inst_mesh=bad_mesh))
    assert hand_renderer.status() & 0x2
    bad_wh = ok.tensors["cam_wh"].clone()
    bad_wh[1, 0] = 4000                                 # wider than the declared maximum
    hand_renderer.render(ok.with_params(cam_wh=bad_wh))
    assert hand_renderer.status() & 0x1
    hand_renderer.render(ok)
    assert hand_renderer.status() == 0


def test_host_checks_reject_bad_arguments(hand_renderer):
    b = sg.hand_batch(1, np.arange(1), res=64)
    db = hand_renderer.upload(b)
    with pytest.raises(L.OrrbError):
        hand_renderer.render(db, cfg=config(tile_w=7))
    with pytest.raises(L.OrrbError):
        hand_renderer.render(db, cfg=config(threads=100))
    with pytest.raises(L.OrrbError):
        small = torch.empty(256, dtype=torch.uint8, device="cuda")
        hand_renderer.render(db, workspace=small)


def test_maximum_sizes(oracle):
    """Largest image sides (4096 wide; 4096 tall, whose 4096 row tiles keep their binning counters in
    global memory) and the largest instance count per sample (1024)."""
    meshes = [sg.plane_mesh(3, 3), sg.box_mesh(0.05), sg.capsule_mesh(0.03, 0.1)]
    r = Renderer(meshes)
    rng = np.random.default_rng(11)
    n = 1024
    inst_mesh = np.concatenate([[0], rng.integers(1, 3, n - 1)])
    poses = [scenes.identity_pose()] + [
        scenes.pose(R=sg._rot("z", np.array(rng.uniform(0, 6.28))), t=(rng.uniform(-1, 1), rng.uniform(-1, 1),
                                                                         rng.uniform(0.05, 0.6)))
        for _ in range(n - 1)]
    cams = [scenes.camera_look((0.0, -2.5, 2.0), (0, 0, 0.2), 4096, 64, 20.0),
            scenes.camera_look((0.3, -2.0, 2.5), (0, 0, 0.2), 64, 4096, 60.0)]
    b = scenes.single_sample(meshes, inst_mesh, poses, cams, seg=np.arange(n) % 250 + 1, mat_base=np.arange(n) % 26,
                             lights=[((0.5, -1.0, 2.0), 2.0)], albedo=(0.6, 0.4, 0.3), specular=0.3,
                             shininess=16.0, ambient=(0.05, 0.05, 0.05), background=(0.2, 0.3, 0.4))
    g = render_np(r, b)
    o = oracle.render(b, debug=True)
    st = compare(g, o, "max sizes")
    assert (o["seg"] > 2).sum() > 1000      # many of the 1023 small instances are visible


def _fan_mesh(rim_px, centre_px=(100.5, 100.5), W=200, H=200, px_per_m=16.0):
    """Coplanar fan (z = 0) whose vertices project exactly onto the given pixel centres of an
    orthographic W x H camera at px_per_m (x_s = W/2 + f x, y_s = H/2 - f y); each triangle is
    listed in both windings, so exactly one copy faces the camera."""
    def world(u, v):
        return ((u - 0.5 * W) / px_per_m, (0.5 * H - v) / px_per_m, 0.0)
    pos = [world(*centre_px)] + [world(u, v) for u, v in rim_px]
    tris = []
    for k in range(len(rim_px)):
        a, b = 1 + k, 1 + (k + 1) % len(rim_px)
        tris += [(0, a, b), (0, b, a)]
    return sg.Mesh(pos=np.asarray(pos, np.float32), nrm=np.tile(np.float32([0, 0, 1]), (len(pos), 1)),
                   idx=np.asarray(tris, np.uint32), tri_mat=np.zeros(len(tris), np.uint8))


@pytest.mark.parametrize("rim", [
    # 4 large triangles: 4 x 200 (triangle, row) pairs fit the shared-memory span table
    [(0.5, 0.5), (199.5, 50.5), (150.5, 199.5), (0.5, 199.5)],
    # 10 large triangles: 2000 pairs, so every pixel is tested instead
    [(0.5, 0.5), (57.5, 0.5), (199.5, 0.5), (199.5, 13.5), (199.5, 150.5), (199.5, 199.5), (120.5, 199.5),
     (0.5, 199.5), (0.5, 160.5), (0.5, 50.5)],
], ids=["span-table", "per-pixel"])
def test_large_triangles_with_edges_through_pixel_centres(oracle, rim):
    """Large (unbinned) triangles whose edges run through pixel centres at slopes 0, 1, 1/2, vertical
    and co-prime ones, so the top-left rule decides every pixel on a shared edge: coverage must
    equal the oracle's exactly with the per-row span table and with per-pixel tests."""
    meshes = [_fan_mesh(rim)]
    r = Renderer(meshes)
    cam = scenes.camera_down((0.0, 0.0, 4.0), 200, 200, px_per_m=16.0)
    b = scenes.single_sample(meshes, [0], [scenes.identity_pose()], [cam], seg=[1],
                             lights=[((0.0, 0.0, 3.0), 2.0)], background=(0.2, 0.3, 0.4))
    o = oracle.render(b, debug=True)
    assert (o["seg"] == 1).sum() > 0.4 * 200 * 200
    for cfg in (config(), config(tile_w=64, tile_h=4), config(tile_w=24, tile_h=8), config(mode=L.ORRB_MODE_PLAIN)):
        g = render_np(r, b, cfg)
        st = compare(g, o, f"fan {len(rim)} {cfg.tile_w}x{cfg.tile_h}")
        assert st["flips"] == 0
        np.testing.assert_array_equal(g["seg"], o["seg"])


def test_slivers_on_pixel_centre_rows(oracle):
    """Small binned triangles on one- and two-row tiles, where each row's candidate columns are narrowed
    to the triangle's float extent along the row: slivers (nearly horizontal and nearly
    vertical), vertices exactly on pixel-centre rows and columns, and sub-pixel triangles must
    cover exactly the oracle's pixels."""
    rng = np.random.default_rng(5)
    W = H = 96
    f = 16.0

    def world(u, v, z):
        return ((u - 0.5 * W) / f, (0.5 * H - v) / f, z)

    pos, tris = [], []
    for k in range(600):
        cu, cv = rng.uniform(2, W - 2), rng.uniform(2, H - 2)
        kind = k % 4
        if kind == 0:      # on pixel-centre rows/columns
            cu, cv = np.floor(cu) + 0.5, np.floor(cv) + 0.5
            d = rng.integers(-6, 7, size=(2, 2)) + 0.0
        elif kind == 1:    # nearly horizontal sliver
            d = np.array([[rng.uniform(-8, 8), rng.uniform(-0.05, 0.05)], [rng.uniform(-8, 8), rng.uniform(-0.6, 0.6)]])
        elif kind == 2:    # nearly vertical sliver
            d = np.array([[rng.uniform(-0.05, 0.05), rng.uniform(-8, 8)], [rng.uniform(-0.6, 0.6), rng.uniform(-8, 8)]])
        else:              # sub-pixel
            d = rng.uniform(-0.8, 0.8, size=(2, 2))
        z = -0.001 * k
        i = len(pos)
        pos += [world(cu, cv, z), world(cu + d[0, 0], cv + d[0, 1], z), world(cu + d[1, 0], cv + d[1, 1], z)]
        tris += [(i, i + 1, i + 2), (i, i + 2, i + 1)]     # one winding faces the camera
    mesh = sg.Mesh(pos=np.asarray(pos, np.float32), nrm=np.tile(np.float32([0, 0, 1]), (len(pos), 1)),
                   idx=np.asarray(tris, np.uint32), tri_mat=np.zeros(len(tris), np.uint8))
    r = Renderer([mesh])
    cam = scenes.camera_down((0.0, 0.0, 4.0), W, H, px_per_m=f)
    b = scenes.single_sample([mesh], [0], [scenes.identity_pose()], [cam], seg=[1],
                             lights=[((0.0, 0.0, 3.0), 2.0)], background=(0.2, 0.3, 0.4))
    o = oracle.render(b, debug=True)
    assert (o["seg"] == 1).sum() > 500
    for cfg in (config(), config(tile_w=256, tile_h=1), config(tile_w=64, tile_h=2), config(tile_w=32, tile_h=4)):
        g = render_np(r, b, cfg)
        compare(g, o, f"slivers {cfg.tile_w}x{cfg.tile_h}")
        np.testing.assert_array_equal(g["seg"], o["seg"])
        np.testing.assert_array_equal(g["depth"], o["depth"])


def test_hand_directional_lights_and_orthographic_cameras(hand_renderer, oracle):
    """The hand scene with directional lights (unit directions) and every second camera
    orthographic (the scene's 0.7 m span over the image), against the oracle."""
    b = sg.hand_batch(9, np.arange(24))
    light = b.light.copy()
    d = light[:, :, :3].astype(np.float64)
    d /= np.maximum(np.linalg.norm(d, axis=-1, keepdims=True), 1e-9)
    light[:, :, :3] = d.astype(np.float32)
    meta = b.light_meta.copy()
    meta[:, 1] = sg.LIGHT_DIRECTIONAL
    intr = b.cam_intr.copy()
    ortho = np.arange(len(intr)) % 2 == 1
    intr[ortho, 0] = intr[ortho, 1] = 200 / 0.7
    intr[ortho, 5] = sg.CAM_ORTHOGRAPHIC
    b = b.with_params(light=light, light_meta=meta, cam_intr=intr)
    g = render_np(hand_renderer, b)
    o = oracle.render(b, debug=True)
    compare(g, o, "hand directional/ortho")
    assert (o["seg"] >= 3).sum() > 1000          # the hand is in view


def test_bin_overflow_falls_back_to_exact_offsets(oracle):
    """Each tile's bin holds an equal share of the bin array; a stack of 300 small triangles on
    8x1 tiles of a 512x512 image overfills its tiles' shares, so phase B redoes the image with
    exact per-tile offsets.  The result must equal the oracle's."""
    rng = np.random.default_rng(3)
    W = H = 512
    f = 64.0

    def world(u, v, z):
        return ((u - 0.5 * W) / f, (0.5 * H - v) / f, z)

    pos, tris = [], []
    for k in range(300):
        cu, cv = 200.0 + rng.uniform(-3, 3), 300.0 + rng.uniform(-3, 3)
        d = rng.uniform(-6, 6, size=(3, 2))
        z = -0.002 * k
        i = len(pos)
        pos += [world(cu + d[j, 0], cv + d[j, 1], z) for j in range(3)]
        tris += [(i, i + 1, i + 2), (i, i + 2, i + 1)]
    mesh = sg.Mesh(pos=np.asarray(pos, np.float32), nrm=np.tile(np.float32([0, 0, 1]), (len(pos), 1)),
                   idx=np.asarray(tris, np.uint32), tri_mat=(np.arange(len(tris)) % 7).astype(np.uint8))
    r = Renderer([mesh])
    cam = scenes.camera_down((0.0, 0.0, 4.0), W, H, px_per_m=f)
    b = scenes.single_sample([mesh], [0], [scenes.identity_pose()], [cam], seg=[1],
                             lights=[((0.0, 0.0, 3.0), 2.0)], background=(0.2, 0.3, 0.4))
    o = oracle.render(b, debug=True)
    for cfg in (config(tile_w=8, tile_h=1), config(tile_w=8, tile_h=2), config()):
        g = render_np(r, b, cfg)
        compare(g, o, f"stack {cfg.tile_w}x{cfg.tile_h}")
        np.testing.assert_array_equal(g["seg"], o["seg"])


def test_colour_grading_matches_oracle(hand_renderer, oracle):
    """The colour-grading epilogue of the rgb channel (random hue, saturation, contrast, brightness,
    white balance and grain per sample) against the oracle, in fused and plain launches; identity
    parameters leave every channel bit-identical, and the other channels never change."""
    b = sg.hand_batch(13, np.arange(12), res=96, grading=True)
    plain_b = b.with_params(grading=None)
    o = oracle.render(b, debug=True)
    ref = render_np(hand_renderer, plain_b)
    for cfg in (config(), config(mode=L.ORRB_MODE_PLAIN)):
        g = render_np(hand_renderer, b, cfg)
        compare(g, o, "graded")
        for k in ("depth", "normal", "seg", "rgb_linear"):
            np.testing.assert_array_equal(g[k], ref[k], err_msg=k)
    assert np.abs(g["rgb"].astype(int) - ref["rgb"].astype(int)).max() > 5     # the grading did something
    ident = render_np(hand_renderer, b.with_params(grading=sg.identity_grading(b.n_samples)))
    for k in ref:
        np.testing.assert_array_equal(ident[k], ref[k], err_msg=k)


def test_tracker_rows_match_oracle(hand_renderer, oracle):
    """Per (camera, instance) screen boxes and projected origins: integers from the bit-exact vertex
    projection, so they must equal the oracle's exactly, in fused and plain launches and with the
    near plane cutting instances (the camera near the table) and an instance behind the camera."""
    b = sg.hand_batch(17, np.arange(10), res=128)
    meshes = [sg.plane_mesh(3, 3), sg.box_mesh(0.5), sg.capsule_mesh(0.3, 0.8)]
    near = scenes.single_sample(meshes, [0, 1, 2, 2],
                                [scenes.identity_pose(), scenes.pose(t=(0.2, -0.1, 0.5)),
                                 scenes.pose(R=sg._rot("z", np.array(0.7)), t=(-0.6, 0.3, 0.9)),
                                 scenes.pose(t=(0.6, -0.4, -0.5))],                  # behind the first camera
                                [scenes.camera_look((0.3, -0.2, 0.05), (0, 0, 0.6), 31, 29, 80.0),
                                 scenes.camera_down((0.05, 0.02, 4.0), 53, 61, px_per_m=17.0)],
                                lights=[((0.5, -1.0, 2.0), 2.0)])
    for r, batch in ((hand_renderer, b), (Renderer(meshes), near)):
        o = oracle.render(batch, tracker=True)["tracker"]
        for cfg in (config(), config(mode=L.ORRB_MODE_PLAIN)):
            db = r.upload(batch)
            out = r.render(db, cfg=cfg, tracker=True)
            out["tracker"].fill_(7)
            out = r.render(db, cfg=cfg, out=out)
            torch.cuda.synchronize()
            assert r.status() == 0
            g = out["tracker"].cpu().numpy()
            np.testing.assert_array_equal(g, o)
    assert (o[..., 6] & 1).any() and o[0, 3, 6] == 0 and o[1, 3, 6] == 3


def test_spot_lights_and_emission_match_oracle(hand_renderer, oracle):
    """The benchmark-like scene (three spot lights with random cones aimed at the block, emissive
    block faces, orbit cameras, grading) in fused and plain launches, and mixed in one batch with
    point-lit samples (which pass a zero cone table and no emission)."""
    spot = sg.benchmark_batch(21, np.arange(10), res=96, orbit=True)
    spot = spot.with_params(emission=spot.emission + np.float32(0.02) * (np.arange(32) % 3 == 0))
    point = sg.hand_batch(22, np.arange(10, 16), res=96, grading=True)
    mixed = sg.concat_batches([sg.select_samples(spot, range(5)), point, sg.select_samples(spot, range(5, 10))])
    for b in (spot, mixed):
        o = oracle.render(b, debug=True)
        for cfg in (config(), config(mode=L.ORRB_MODE_PLAIN)):
            compare(render_np(hand_renderer, b, cfg), o, "spot")
    lin = o["rgb_linear"].reshape(-1, 96 * 96, 3)
    assert (lin[:5].max(axis=(1, 2)) > 0.2).all()           # the spots light the scene


def test_lights_that_light_nothing_are_flagged(hand_renderer, oracle):
    """A spot type without its cone table and an unknown type light nothing and set the light flag;
    a null cone (cos_inner <= cos_outer) lights nothing and is valid input."""
    b = sg.benchmark_batch(3, np.arange(3), res=64, grading=False)
    null_cone = b.light_spot.copy()
    null_cone[1, :, 4] = null_cone[1, :, 3]
    meta = b.light_meta.copy()
    meta[2, 1] = 7
    for bad, flagged in ((b.with_params(light_spot=null_cone), False), (b.with_params(light_spot=None), True),
                         (b.with_params(light_meta=meta), True)):
        out = hand_renderer.render(hand_renderer.upload(bad), rgb_linear=True)
        torch.cuda.synchronize()
        assert bool(hand_renderer.status() & 0x10) == flagged
        compare(to_numpy(out), oracle.render(bad, debug=True), "dark lights")


@pytest.mark.parametrize("mode,kind", [(L.ORRB_MODE_FUSED, "spot"), (L.ORRB_MODE_PLAIN, "spot"),
                                       (L.ORRB_MODE_STAGED, "spot"), (L.ORRB_MODE_FUSED, "cube"),
                                       (L.ORRB_MODE_PLAIN, "cube"), (L.ORRB_MODE_STAGED, "cube")])
def test_shadow_maps_and_lookups_match_oracle(hand_renderer, oracle, mode, kind):
    """Shadow maps of the benchmark-like scene's spot lights (one face each) and of the hand scene's
    point lights (six cube faces each): every map of a casting face bit-identical to the oracle's
    (the same rasterisation, back faces), every G-buffer material word (slot and shadowed taps per
    light) identical, and the channels within the contract; maps of lights that cast none are
    left untouched."""
    if kind == "spot":
        b = sg.benchmark_batch(31, np.arange(8), res=96, shadow_res=128)
    else:
        b = sg.hand_batch(32, np.arange(8), res=96, shadow_res=64)
    b = b.with_params(light_meta=b.light_meta.copy())
    b.light_meta[5, 0] = max(1, b.light_meta[5, 0] - 1)   # a sample with one light fewer
    o = oracle.render(b, debug=True, gbuffer=True)
    r = hand_renderer
    db = r.upload(b)
    out = r.render(db, cfg=config(mode=mode), rgb_linear=True, gbuffer=True)
    out["shadow_map"].fill_(-1.0)
    out = r.render(db, cfg=config(mode=mode), out=out)
    torch.cuda.synchronize()
    assert r.status() == 0
    g = to_numpy(out)
    cast = np.arange(4)[None, :] < b.light_meta[:, :1]
    np.testing.assert_array_equal(g["shadow_map"][cast], o["shadow_map"][cast])
    assert (g["shadow_map"][~cast] == -1.0).all()
    assert (o["shadow_map"][cast] > 0).mean() > 0.001
    np.testing.assert_array_equal(g["gbuffer"][6].view(np.int32), o["gb_mat"])
    same = g["depth"] == o["depth"]                     # the lookup's input: the G-buffer position, bit for bit
    np.testing.assert_array_equal(g["gbuffer"][0:3].T[same], o["gb_pos"][same])
    k = (o["gb_mat"][o["gb_mat"] >= 0] >> 8) & 0xfff
    assert (k > 0).mean() > 0.01                        # shadows fall on a share of the pixels
    compare(g, o, "shadows")


@pytest.mark.parametrize("grading", [True, False])
@pytest.mark.parametrize("shadows", [True, False])
def test_option_combinations_with_tracker_rows_match_oracle(hand_renderer, oracle, grading, shadows):
    """Tracker rows together with spot lights, emission, colour grading and shadow maps, each
    combination its own kernel instance, fused, plain and staged: channels, G-buffer words, maps and
    tracker rows against the oracle."""
    b = sg.benchmark_batch(41, np.arange(6), res=80, grading=grading, shadow_res=96 if shadows else 0)
    o = oracle.render(b, debug=True, gbuffer=True, tracker=True)
    cast = np.arange(4)[None, :] < b.light_meta[:, :1]
    for cfg in (config(), config(mode=L.ORRB_MODE_PLAIN), config(mode=L.ORRB_MODE_STAGED)):
        g = render_np(hand_renderer, b, cfg, gbuffer=True, tracker=True)
        compare(g, o, "options")
        np.testing.assert_array_equal(g["tracker"], o["tracker"])
        np.testing.assert_array_equal(g["gbuffer"][6].view(np.int32), o["gb_mat"])
        if shadows:
            np.testing.assert_array_equal(g["shadow_map"][cast], o["shadow_map"][cast])


def test_graded_tracked_point_lit_batch_matches_oracle(hand_renderer, oracle):
    """Colour grading with tracker rows and plain point lights (the grading-and-tracker instance)."""
    b = sg.hand_batch(43, np.arange(4), res=80, grading=True)
    o = oracle.render(b, debug=True, tracker=True)
    g = render_np(hand_renderer, b, tracker=True)
    compare(g, o, "graded and tracked")
    np.testing.assert_array_equal(g["tracker"], o["tracker"])


@pytest.mark.parametrize("mode", [L.ORRB_MODE_FUSED, L.ORRB_MODE_PLAIN])
def test_ragged_shadow_maps_match_oracle(hand_renderer, oracle, mode):
    """Shadow maps of a ragged side (257: a partial tile column in the shadow pass, and a one-column
    block and a one-row walk in the neighbourhood table) with camera images of a ragged width,
    against the oracle."""
    b = sg.benchmark_batch(47, np.arange(3), res=72, grading=False, shadow_res=257)
    o = oracle.render(b, debug=True, gbuffer=True)
    g = render_np(hand_renderer, b, config(mode=mode, tile_w=64, tile_h=2), gbuffer=True)
    cast = np.arange(4)[None, :] < b.light_meta[:, :1]
    np.testing.assert_array_equal(g["shadow_map"][cast], o["shadow_map"][cast])
    np.testing.assert_array_equal(g["gbuffer"][6].view(np.int32), o["gb_mat"])
    k = (o["gb_mat"][o["gb_mat"] >= 0] >> 8) & 0xfff
    assert ((k & 15) % 9 != 0).any()                   # partly shadowed points: the taps were counted
    compare(g, o, "ragged shadows")


@pytest.mark.parametrize("mode", [L.ORRB_MODE_FUSED, L.ORRB_MODE_PLAIN])
def test_directional_light_shadows_match_oracle(tiny_renderer, oracle, mode):
    """The tiny scene's directional light casting the cube's shadow from an orthographic map: maps,
    G-buffer words and channels against the oracle."""
    b = sg.tiny_batch(5, n_samples=8, shadow_res=128)
    o = oracle.render(b, debug=True, gbuffer=True)
    g = render_np(tiny_renderer, b, config(mode=mode), gbuffer=True)
    cast = np.arange(4)[None, :] < b.light_meta[:, :1]
    np.testing.assert_array_equal(g["shadow_map"][cast], o["shadow_map"][cast])
    np.testing.assert_array_equal(g["gbuffer"][6].view(np.int32), o["gb_mat"])
    k = (o["gb_mat"][o["gb_mat"] >= 0] >> 8) & 15
    assert (k == 9).mean() > 0.02 and ((k > 0) & (k < 9)).any()
    compare(g, o, "directional shadows")
