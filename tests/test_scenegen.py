"""The seeded input generator: a sample's parameters do not depend on its batch (Sec. 4.3 seeding)."""

from pathlib import Path

import numpy as np

from paper_1906_11633_b300 import scenegen as sg

GOLDEN = Path(__file__).parent / "golden"


def test_philox_matches_the_published_known_answer_vectors():
    """The block function every draw comes from, against the Philox4x32-10 vectors published with
    the generator (Salmon et al., SC 2011): all-zero, all-one and pi-digit counters and keys."""
    rows = [ln.split() for ln in (GOLDEN / "philox4x32_10_kat.txt").read_text().splitlines()
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        c, k, want = [int(v, 16) for v in row[:4]], [int(v, 16) for v in row[4:6]], [int(v, 16) for v in row[6:]]
        got = sg.philox4x32_10(*[np.uint32(v) for v in c], *k)
        assert [int(v) for v in got] == want, row
    # broadcast over a counter array gives the same words as one call per counter
    ctr = np.array([0, 0xFFFFFFFF], np.uint32)
    many = sg.philox4x32_10(ctr, ctr, ctr, ctr, 0, 0)
    for i, v in enumerate(ctr):
        one = sg.philox4x32_10(v, v, v, v, 0, 0)
        assert [int(w[i]) for w in many] == [int(w) for w in one]


def test_sample_identical_alone_and_in_batch():
    full = sg.hand_batch(9, np.arange(6))
    for s in (0, 3, 5):
        alone = sg.hand_batch(9, [s])
        sub = sg.select_samples(full, [s])
        for name in ("inst_pose", "cam_view", "cam_intr", "light", "light_meta", "material", "exposure_ev",
                     "ambient", "background"):
            np.testing.assert_array_equal(getattr(alone, name), getattr(sub, name), err_msg=name)


def test_streams_are_independent():
    a = sg.uniform(1, sg.STREAM_LIGHTS, [0, 1, 2], 5)
    b = sg.uniform(1, sg.STREAM_LIGHTS, [0, 1, 2], 40)
    np.testing.assert_array_equal(a, b[:, :5])
    c = sg.uniform(1, sg.STREAM_CAMERA, [0, 1, 2], 5)
    assert not np.array_equal(a, c)
    u = sg.uniform(3, 1, np.arange(20000), 4).ravel()
    assert 0.0 < u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def test_poses_are_rigid_and_counts_match_the_workloads():
    b = sg.hand_batch(0, np.arange(4))
    R = b.inst_pose[:, :, :3].astype(np.float64)
    err = np.abs(np.einsum("nij,nik->njk", R, R) - np.eye(3)).max()
    assert err < 1e-6
    assert b.tris_per_sample()[0] == 24 * 320 + 12 + 2
    u = sg.uneven_batch(0, np.arange(64))
    tps = u.tris_per_sample()
    assert tps.min() >= 320 + 14 and tps.max() <= 50000 + 320
    assert set(np.unique(u.cam_wh[:, 0])) <= set(sg.UNEVEN_RES)


def test_hsv_to_rgb_matches_colorsys():
    import colorsys
    rng = np.random.default_rng(1)
    hsv = rng.uniform(0, 1, (500, 3))
    hsv[:5] = [[0, 0, 0], [0.5, 0, 1], [1 / 6, 1, 1], [2 / 3, 1, 0.5], [0.999999, 0.3, 0.7]]
    want = np.array([colorsys.hsv_to_rgb(*v) for v in hsv])
    np.testing.assert_allclose(sg.hsv_to_rgb(hsv), want, atol=1e-12)


def test_fixed_hue_materials_stay_near_their_calibrated_colours():
    import colorsys
    ids = np.arange(4000)
    hsv = sg.BLOCK_HSV
    albedo, ks, alpha, em = sg.fixed_hue_materials(3, ids, hsv, radius=(0.03, 0.15, 0.15),
                                                   clamp=((0, 1), (0.2, 1.0), (0.2, 1.0)), specular=(0.0, 0.6),
                                                   glossiness=(0.3, 0.9), emissive_prob=0.15,
                                                   emissive_power=(0.1, 0.6))
    back = np.array([colorsys.rgb_to_hsv(*c) for c in albedo.reshape(-1, 3)]).reshape(albedo.shape)
    dh = (back[..., 0] - hsv[:, 0] + 0.5) % 1.0 - 0.5
    assert np.abs(dh).max() <= 0.03 + 1e-9
    assert (np.abs(back[..., 1:] - hsv[:, 1:]) <= 0.15 + 1e-9).all() and back[..., 1:].min() >= 0.2 - 1e-9
    assert 0.0 <= ks.min() and ks.max() <= 0.6
    assert 128 ** 0.3 - 1e-9 <= alpha.min() and alpha.max() <= 128 ** 0.9 + 1e-9
    on = em > 0
    assert abs(on.mean() - 0.15) < 0.01 and em[on].min() >= 0.1 and em.max() <= 0.6
    a1, _, _, e1 = sg.fixed_hue_materials(3, [17], hsv)
    np.testing.assert_array_equal(a1[0], albedo[17])
    np.testing.assert_array_equal(e1[0], em[17])


def test_light_setup_points_every_light_at_the_target():
    target = np.array([0.02, 0.0, 0.16])
    pos, axis = sg.light_setup(2, np.arange(300), 3, target, distance=(0.35, 0.6), height=(0.4, 0.7))
    off = pos - target
    d, h = np.hypot(off[..., 0], off[..., 1]), off[..., 2]
    assert d.min() >= 0.35 and d.max() <= 0.6 and h.min() >= 0.4 and h.max() <= 0.7
    np.testing.assert_allclose(np.linalg.norm(axis, axis=-1), 1.0, atol=1e-12)
    np.testing.assert_allclose(np.cross(axis, -off), 0.0, atol=1e-12)    # the axis lies on the line to the target
    assert ((axis * -off).sum(-1) > 0).all()
    az = np.arctan2(off[..., 1], off[..., 0])
    gap = (np.diff(np.sort(az, axis=1), axis=1) + 2 * np.pi) % (2 * np.pi)
    np.testing.assert_allclose(gap, 2 * np.pi / 3, atol=1e-9)            # spread evenly in azimuth


def test_light_levels_split_the_total_and_order_the_cones():
    inten, cos_o, cos_i = sg.light_levels(4, np.arange(2000), 3, total=(0.5, 1.0), weight=(0.5, 1.0),
                                          outer_deg=(25, 45), softness=(0.1, 0.4))
    T = inten.sum(1)
    assert T.min() >= 0.5 and T.max() <= 1.0
    share = inten / T[:, None]
    assert share.min() >= 0.5 / (0.5 + 2 * 1.0) - 1e-12 and share.max() <= 1.0 / (1.0 + 2 * 0.5) + 1e-12
    outer = np.degrees(np.arccos(cos_o))
    assert outer.min() >= 25 - 1e-9 and outer.max() <= 45 + 1e-9
    ratio = np.arccos(cos_i) / np.arccos(cos_o)
    assert ratio.min() >= 0.6 - 1e-9 and ratio.max() <= 0.9 + 1e-9 and (cos_i > cos_o).all()


def test_orbit_cameras_look_at_the_point_of_interest():
    poi = np.array([0.02, 0.0, 0.16])
    views, owner = sg.orbit_views(6, np.arange(100), 3, poi, radius=(0.4, 0.6), elevation_deg=(20, 70))
    assert views.shape == (300, 3, 4) and (owner == np.repeat(np.arange(100), 3)).all()
    R, t = views[:, :, :3], views[:, :, 3]
    p = np.einsum("cij,j->ci", R, poi) + t                   # the point of interest in view space
    np.testing.assert_allclose(p[:, :2], 0.0, atol=1e-12)
    r = -p[:, 2]
    assert r.min() >= 0.4 - 1e-12 and r.max() <= 0.6 + 1e-12
    eye = -np.einsum("cji,cj->ci", R, t)
    el = np.degrees(np.arcsin((eye[:, 2] - poi[2]) / r))
    assert el.min() >= 20 - 1e-9 and el.max() <= 70 + 1e-9


def test_benchmark_sample_identical_alone_and_in_batch():
    full = sg.benchmark_batch(9, np.arange(5), res=32, orbit=True)
    for s in (0, 4):
        alone = sg.benchmark_batch(9, [s], res=32, orbit=True)
        sub = sg.select_samples(full, [s])
        for name in ("cam_view", "light", "light_meta", "light_spot", "material", "emission", "grading"):
            np.testing.assert_array_equal(getattr(alone, name), getattr(sub, name), err_msg=name)
    assert (full.light_meta[:, 1] == sg.LIGHT_SPOT).all() and (full.light_meta[:, 0] == 3).all()
