"""Pins of the oracle's tracker rows (per camera and instance: the 8.8 fixed-point screen box of the
instance's vertices in front of the near plane, the projected origin and flags):

  a quad whose corners project exactly onto known pixel positions (orthographic camera) has exactly
  those corners as its box, and its pose translation as its keypoint; an instance behind the camera
  has an empty row; an instance cut by the near plane boxes only its vertices in front; and every
  pixel an unclipped instance covers has its centre inside that instance's box.
"""

import numpy as np
import pytest

from paper_1906_11633_b300 import scenegen as sg
from tests import scenes

INT_MAX, INT_MIN = 2**31 - 1, -2**31


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as o
    o.build()
    return o


def _quad(u0, v0, u1, v1, W=64, H=48, f=16.0):
    """Quad with corners projecting onto (u, v) pixel coordinates of an orthographic W x H camera at f px/m."""
    def world(u, v):
        return ((u - 0.5 * W) / f, (0.5 * H - v) / f, 0.0)
    corners = [world(u0, v1), world(u1, v1), world(u1, v0), world(u0, v0)]
    return sg.quad_mesh(corners, (0.0, 0.0, 1.0))


def test_box_and_keypoint_of_a_quad_are_exact(orc):
    W, H, f = 64, 48, 16.0
    mesh = _quad(10.25, 7.5, 41.75, 30.0)
    t = (0.3125, -0.25, 0.0)                    # a translation exact in 8.8 at 16 px/m
    cam = scenes.camera_down((0.0, 0.0, 4.0), W, H, px_per_m=f)
    b = scenes.single_sample([mesh], [0], [scenes.pose(t=t)], [cam], seg=[1], lights=[((0, 0, 3), 1.0)])
    row = orc.render(b, tracker=True)["tracker"][0, 0]
    du, dv = t[0] * f, -t[1] * f                 # the translation in pixels (screen y points down)
    want = [round(256 * (10.25 + du)), round(256 * (7.5 + dv)), round(256 * (41.75 + du)), round(256 * (30.0 + dv))]
    assert list(row[:4]) == want
    assert list(row[4:6]) == [round(256 * (0.5 * W + du)), round(256 * (0.5 * H + dv))]
    assert row[6] == 3 and row[7] == 0


def test_instance_behind_the_camera_has_an_empty_row(orc):
    cam = scenes.camera_look((0.0, -2.0, 1.0), (0.0, 0.0, 1.0), 64, 64, 60.0)
    mesh = sg.box_mesh(0.2)
    b = scenes.single_sample([mesh], [0, 0], [scenes.pose(t=(0.0, 0.5, 1.0)), scenes.pose(t=(0.0, -3.0, 1.0))],
                             [cam], seg=[1, 2], lights=[((0, 0, 3), 1.0)])
    rows = orc.render(b, tracker=True)["tracker"][0]
    assert rows[0, 6] == 3 and rows[0, 0] <= rows[0, 2] and rows[0, 1] <= rows[0, 3]
    assert list(rows[1]) == [INT_MAX, INT_MAX, INT_MIN, INT_MIN, 0, 0, 0, 0]


def _project(cam, pts):
    """fp64 screen coordinates (8.8 units) and view depth of world points."""
    view, intr, _ = cam
    v = pts @ view[:, :3].T + view[:, 3]
    fx, fy, cx, cy = intr[:4]
    return 256 * (cx + fx * v[:, 0] / -v[:, 2]), 256 * (cy - fy * v[:, 1] / -v[:, 2]), -v[:, 2]


def test_near_plane_cut_boxes_only_vertices_in_front(orc):
    cam = scenes.camera_look((0.0, -2.0, 1.0), (0.3, 0.0, 1.2), 64, 64, 60.0)
    mesh = sg.box_mesh(0.6)
    t = np.array([0.1, -1.9, 1.05])              # the box straddles the camera plane
    b = scenes.single_sample([mesh], [0], [scenes.pose(t=t)], [cam], seg=[1], lights=[((0, 0, 3), 1.0)])
    row = orc.render(b, tracker=True)["tracker"][0, 0]
    xs, ys, z = _project(cam, mesh.pos.astype(np.float64) + t)
    front = z > 0.01 + 1e-6
    assert 0 < front.sum() < len(z) and row[6] & 1
    assert abs(row[0] - xs[front].min()) <= 2 and abs(row[2] - xs[front].max()) <= 2
    assert abs(row[1] - ys[front].min()) <= 2 and abs(row[3] - ys[front].max()) <= 2
    assert row[6] & 2 == 0 or _project(cam, t[None])[2][0] > 0.01


def test_covered_pixels_lie_inside_the_box(orc):
    b = sg.hand_batch(2, np.arange(3), res=96)
    o = orc.render(b, tracker=True)
    seg = o["seg"].reshape(b.n_cams, 96, 96)
    n = 0
    for c in range(b.n_cams):
        s = int(b.cam_sample[c])
        for i in range(int(b.inst_offset[s + 1] - b.inst_offset[s])):
            row = o["tracker"][c, i]
            sid = int(b.inst_seg[b.inst_offset[s] + i])
            ys, xs = np.nonzero(seg[c] == sid)
            mesh = b.meshes[int(b.inst_mesh[b.inst_offset[s] + i])]
            pose = b.inst_pose[b.inst_offset[s] + i].astype(np.float64)
            world = mesh.pos.astype(np.float64) @ pose[:, :3].T + pose[:, 3]
            view = world @ b.cam_view[c, :, :3].astype(np.float64).T + b.cam_view[c, :, 3]
            if len(xs) == 0 or not (view[:, 2] < -0.011).all():   # unseen, or cut by the near plane
                continue
            cx, cy = 256 * xs + 128, 256 * ys + 128
            assert (cx >= row[0]).all() and (cx <= row[2]).all() and (cy >= row[1]).all() and (cy <= row[3]).all()
            n += 1
    assert n > 40
