"""Hand-built scenes for closed-form tests (test helper; builds inputs only)."""

import numpy as np

from paper_1906_11633_b300 import scenegen as sg


def camera_down(eye, W, H, fovy_deg=None, px_per_m=None, near=0.01):
    """Camera at `eye` looking straight down -z_world, image +y = world +y (R = identity)."""
    R = np.eye(3)
    view = sg.view_matrix(R, np.asarray(eye, np.float64))
    if px_per_m is not None:
        intr = sg.orthographic_intrinsics(W, H, px_per_m, near)
    else:
        intr = sg.perspective_intrinsics(W, H, fovy_deg, near)
    return view, intr, (W, H)


def camera_look(eye, target, W, H, fovy_deg, near=0.01):
    R = sg.look_at(eye, target)
    return sg.view_matrix(R, np.asarray(eye, np.float64)), sg.perspective_intrinsics(W, H, fovy_deg, near), (W, H)


def identity_pose():
    return np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)


def pose(R=None, t=(0, 0, 0)):
    R = np.eye(3) if R is None else np.asarray(R)
    return np.concatenate([R, np.asarray(t, np.float64).reshape(3, 1)], axis=1)


def single_sample(meshes, inst_mesh, poses, cams, seg=None, mat_base=None, lights=(), light_type=sg.LIGHT_POINT,
                  albedo=None, specular=0.0, shininess=1.0, ev=0.0, ambient=(0, 0, 0), background=(0, 0, 0),
                  spots=None, emission=None):
    """One sample.  `spots`: per light (axis xyz, cos outer, cos inner) for spot lights;
    `emission`: a scalar or [32] per-slot material emission."""
    n = len(inst_mesh)
    seg = np.arange(1, n + 1) if seg is None else np.asarray(seg)
    mat_base = np.zeros(n) if mat_base is None else np.asarray(mat_base)
    mat = np.zeros((1, sg.MAX_MATERIALS, 5))
    mat[0, :, :3] = 0.5 if albedo is None else np.asarray(albedo)
    mat[0, :, 3] = specular
    mat[0, :, 4] = shininess
    light = np.zeros((1, sg.MAX_LIGHTS, 4))
    for i, (p, I) in enumerate(lights):
        light[0, i, :3] = p
        light[0, i, 3] = I
    wh = np.array([c[2] for c in cams], np.int32).reshape(-1, 2)
    return sg.Batch(
        meshes=list(meshes),
        inst_offset=np.array([0, n], np.int32),
        inst_mesh=np.asarray(inst_mesh, np.uint32),
        inst_pose=np.asarray(poses, np.float64).reshape(n, 3, 4).astype(np.float32),
        inst_seg=seg.astype(np.uint8),
        inst_mat_base=mat_base.astype(np.int16),
        cam_offset=np.array([0, len(cams)], np.int32),
        cam_sample=np.zeros(len(cams), np.int32),
        cam_view=np.stack([c[0] for c in cams]).astype(np.float32),
        cam_intr=np.stack([c[1] for c in cams]).astype(np.float32),
        cam_wh=wh,
        img_offset=sg._img_offsets(wh),
        light=light.astype(np.float32),
        light_meta=np.array([[len(lights), light_type]], np.int32),
        material=mat.astype(np.float32),
        exposure_ev=np.array([ev], np.float32),
        ambient=np.asarray(ambient, np.float32).reshape(1, 3),
        background=np.asarray(background, np.float32).reshape(1, 3),
        sample_ids=np.zeros(1, np.int64),
        light_spot=None if spots is None else _spot_table(spots),
        emission=None if emission is None else np.broadcast_to(np.asarray(emission, np.float32),
                                                               (1, sg.MAX_MATERIALS)).copy(),
    )


def _spot_table(spots):
    t = np.zeros((1, sg.MAX_LIGHTS, 5), np.float32)
    for i, (axis, cos_o, cos_i) in enumerate(spots):
        t[0, i, :3] = axis
        t[0, i, 3] = cos_o
        t[0, i, 4] = cos_i
    return t
