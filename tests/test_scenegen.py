"""The seeded input generator: a sample's parameters do not depend on its batch (Sec. 4.3 seeding)."""

import numpy as np

from paper_1906_11633_b300 import scenegen as sg


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
