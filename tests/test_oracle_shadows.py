"""Pins of the oracle's shadows (the benchmark scene's shadow-casting spot lights, Sec. 5): the
shadow pass (steps 2-8 from the light's shadow camera, back faces only) and the 3 x 3
percentage-closer lookup, against closed forms of box geometry:

  a box seen from straight above has its bottom face at the bottom face's depth in the middle of
  its map and its side faces, at the depth where the pixel ray meets them, in the ring out to the
  top face's outline, and nothing outside (a front-face pass would show the top face instead);
  the shadow of a floating box under a light straight above is the box's central projection from
  the light, so plane pixels well inside it have all 9 taps shadowed and pixels well outside none;
  lights without a shadow camera render exactly as without shadows.
"""

import math

import numpy as np

from paper_1906_11633_b300 import scenegen as sg
from tests import scenes


def _down_camera(eye, R, half_deg, bias=0.0, near=0.05):
    view = sg.view_matrix(np.eye(3), np.asarray(eye, np.float64))
    f = 0.5 * R / math.tan(math.radians(half_deg))
    return view, np.array([f, f, 0.5 * R, 0.5 * R, near, bias, 0.0])


def _shadowed(batch, views, intrs, R):
    sv = np.zeros((batch.n_samples, 4, 1, 3, 4), np.float32)
    si = np.zeros((batch.n_samples, 4, 1, 7), np.float32)
    for l, (v, i) in enumerate(zip(views, intrs)):
        sv[:, l, 0], si[:, l, 0] = v, i
    return batch.with_params(shadow_view=sv, shadow_intr=si, shadow_res=R, shadow_faces=1)


def test_shadow_map_holds_the_nearest_back_faces(oracle):
    a, zc, H, R, half = 0.1, 0.3, 1.0, 96, 20.0            # box half-size and centre height, camera height
    b = scenes.single_sample([sg.box_mesh(a, per_face_material=False)], [0], [scenes.pose(t=(0.0, 0.0, zc))],
                             [scenes.camera_down((0.0, 0.0, 3.0), 8, 8, fovy_deg=40)], lights=[((0, 0, H), 1.0)])
    view, intr = _down_camera((0.0, 0.0, H), R, half)
    m = oracle.render(_shadowed(b, [view], [intr], R))["shadow_map"][0, 0, 0].astype(np.float64)
    f = intr[0]
    u = (np.arange(R) + 0.5 - 0.5 * R) / f                  # pixel-centre ray slopes
    ux, uy = np.meshgrid(u, -u)
    reach = np.maximum(np.abs(ux), np.abs(uy))
    d_bottom, d_top = H - (zc - a), H - (zc + a)
    px = 1.0 / f                                            # one pixel, in slope units
    inner = reach < a / d_bottom - px
    ring = (reach > a / d_bottom + px) & (reach < a / d_top - px)
    outside = reach > a / d_top + px
    assert inner.sum() > 100 and ring.sum() > 100 and outside.sum() > 100
    np.testing.assert_allclose(m[inner], d_bottom, rtol=1e-6)
    np.testing.assert_allclose(m[ring], a / reach[ring], rtol=2e-5)   # the side face x = a (or y = a)
    assert (m[outside] == 0).all()


def test_box_shadow_is_its_central_projection_from_the_light(oracle):
    a, z0, z1, H, R = 0.15, 0.1, 0.4, 1.2, 256              # floating box [z0, z1], light height H
    plane, box = sg.plane_mesh(2.0, 2.0), sg.box_mesh(a, per_face_material=False)
    cam = scenes.camera_down((0.0, 0.0, 4.0), 240, 240, fovy_deg=12)
    b = scenes.single_sample([plane, box], [0, 1], [scenes.identity_pose(), scenes.pose(t=(0, 0, 0.5 * (z0 + z1)))],
                             [cam], seg=[1, 2], lights=[((0.0, 0.0, H), 1.0)], light_type=sg.LIGHT_SPOT,
                             spots=[((0.0, 0.0, -1.0), math.cos(math.radians(40)), math.cos(math.radians(30)))])
    view, intr = _down_camera((0.0, 0.0, H), R, 44.0, bias=0.004)
    o = oracle.render(_shadowed(b, [view], [intr], R), gbuffer=True)
    k = (o["gb_mat"] >> 8) & 15
    on_plane = o["seg"] == 1
    fx, fy, cx, cy = b.cam_intr[0, :4].astype(np.float64)
    xs, ys = np.meshgrid(np.arange(240) + 0.5, np.arange(240) + 0.5)
    reach = np.maximum(np.abs(4.0 * (xs - cx) / fx), np.abs(4.0 * (ys - cy) / fy)).ravel()
    edge = a * H / (H - z1)                                 # the shadow's half-size on the plane
    margin = 2.5 * H / intr[0] + 0.004                      # PCF reach (1.5 texels) + a texel + the bias
    inside = on_plane & (reach < edge - margin)
    outside = on_plane & (reach > edge + margin) & (reach < 0.6)
    assert inside.sum() > 200 and outside.sum() > 200
    assert (k[inside] == 9).all()
    assert (k[outside] == 0).all()
    assert ((k[on_plane] > 0) & (k[on_plane] < 9)).any()   # a penumbra between
    lit = oracle.render(b)["rgb_linear"]
    np.testing.assert_array_equal(o["rgb_linear"][inside], 0 * lit[inside])     # no ambient: black
    np.testing.assert_array_equal(o["rgb_linear"][outside], lit[outside])


def test_lights_without_a_shadow_camera_are_unshadowed(oracle):
    b = sg.benchmark_batch(2, np.arange(2), res=48, shadow_res=64, grading=False)
    plain = oracle.render(b.with_params(shadow_view=None, shadow_intr=None, shadow_res=0), gbuffer=True)
    off = b.shadow_intr.copy()
    off[..., 0] = 0.0                                       # fx = 0: no shadow camera
    got = oracle.render(b.with_params(shadow_intr=off), gbuffer=True)
    for k in ("rgb", "rgb_linear", "depth", "normal", "seg", "gb_mat"):
        np.testing.assert_array_equal(got[k], plain[k], err_msg=k)
    shadowed = oracle.render(b, gbuffer=True)
    assert (shadowed["gb_mat"] > 0xff).any() and (shadowed["rgb_linear"] != plain["rgb_linear"]).any()
    np.testing.assert_array_equal(shadowed["gb_mat"] & 0xff | (shadowed["gb_mat"] < 0) * -1,
                                  plain["gb_mat"])          # the slot bits are unchanged


def _floating_box(bias, R=256, a=0.15, z0=0.1, z1=0.4, H=1.2):
    """A box floating over [z0, z1] above a plane, a spot light straight above at height H with a
    straight-down shadow camera (R x R, 44 deg half-angle), and a camera straight down from 4 m."""
    plane, box = sg.plane_mesh(2.0, 2.0), sg.box_mesh(a, per_face_material=False)
    cam = scenes.camera_down((0.0, 0.0, 4.0), 240, 240, fovy_deg=12)
    b = scenes.single_sample([plane, box], [0, 1], [scenes.identity_pose(), scenes.pose(t=(0, 0, 0.5 * (z0 + z1)))],
                             [cam], seg=[1, 2], lights=[((0.0, 0.0, H), 1.0)], light_type=sg.LIGHT_SPOT,
                             spots=[((0.0, 0.0, -1.0), math.cos(math.radians(40)), math.cos(math.radians(30)))])
    view, intr = _down_camera((0.0, 0.0, H), R, 44.0, bias=bias)
    return _shadowed(b, [view], [intr], R), intr


def test_depth_bias_is_subtracted_from_the_receiver_depth(oracle):
    """Seen from the light the plane lies at depth H and the box's back faces at H - z for exit
    heights z in [z0, z1]: a bias just below z0 leaves the shadow's core fully shadowed, a bias just
    above z1 lifts every shadow."""
    a, z0, z1, H = 0.15, 0.1, 0.4, 1.2
    for bias, core in ((z0 - 0.002, 9), (z1 + 0.002, 0)):
        b, intr = _floating_box(bias)
        o = oracle.render(b, gbuffer=True)
        k = (o["gb_mat"] >> 8) & 15
        on_plane = o["seg"] == 1
        P = o["gb_pos"].astype(np.float64)                  # camera R = identity: view x, y = world x, y
        reach = np.maximum(np.abs(P[:, 0]), np.abs(P[:, 1]))
        inside = on_plane & (reach < a * H / (H - z1) - 2.5 * H / intr[0])
        assert inside.sum() > 200
        assert (k[inside] == core).all(), (bias, np.bincount(k[inside]))
        if core == 0:
            assert (k[on_plane] == 0).all()


def test_pcf_taps_match_the_plane_geometry(oracle):
    """For plane pixels the receiver's texel position has a closed form (u = cx + f x / H, v = cy -
    f y / H under the straight-down shadow camera): counting the 3 x 3 taps of the oracle's own map
    (pinned above) around it gives the oracle's counts, except where u or v falls within 1e-3 texel
    of a texel edge (fp32 rounding)."""
    H, bias, R = 1.2, 0.004, 96
    b, intr = _floating_box(bias, R=R)
    o = oracle.render(b, gbuffer=True)
    m = o["shadow_map"][0, 0, 0].astype(np.float64)
    k = (o["gb_mat"] >> 8) & 15
    P = o["gb_pos"].astype(np.float64)
    sel = np.nonzero(o["seg"] == 1)[0]
    f, c = intr[0], intr[2]
    u, v = c + f * P[sel, 0] / H, c - f * P[sel, 1] / H
    i0, j0 = np.floor(u).astype(int), np.floor(v).astype(int)
    inside = (i0 >= 0) & (j0 >= 0) & (i0 < R) & (j0 < R)       # else no face contains the point: lit
    want = np.zeros(len(sel), int)
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            i, j = i0 + di, j0 + dj
            ok = (i >= 0) & (j >= 0) & (i < R) & (j < R)
            d = np.where(ok, m[np.clip(j, 0, R - 1), np.clip(i, 0, R - 1)], 0.0)
            want += ((d > 0) & (H - bias > d) & inside).astype(int)
    safe = (np.abs(u - np.round(u)) > 1e-3) & (np.abs(v - np.round(v)) > 1e-3)
    assert safe.mean() > 0.99 and (want[safe] == 9).sum() > 50 and ((want[safe] > 0) & (want[safe] < 9)).sum() > 20
    np.testing.assert_array_equal(k[sel][safe], want[safe])


def _ray_hits_box(L, p, c, half, grow):
    """Does the segment L -> p (rows of p) pass through the box centred at c (half-sizes `half` grown
    by `grow`)?  Slab test in fp64."""
    d = p - L
    lo, hi = c - half - grow, c + half + grow
    with np.errstate(divide="ignore", invalid="ignore"):
        t1, t2 = (lo - L) / d, (hi - L) / d
    tmin = np.nanmax(np.minimum(t1, t2), axis=1)
    tmax = np.nanmin(np.maximum(t1, t2), axis=1)
    return (tmax >= np.maximum(tmin, 0.0)) & (tmin <= 1.0)


def test_cube_faces_shadow_a_point_light_in_every_direction(oracle):
    """A point light with six 90-degree cube-face cameras over a plane with boxes below it and to
    its sides: every plane point whose ray to the light passes well inside a box is fully shadowed
    (whichever face sees it), every point whose ray misses all boxes by a margin is lit."""
    H, R, a = 0.5, 128, 0.06
    boxes = [np.array([0.0, 0.0, 0.25]), np.array([0.55, 0.0, 0.2]), np.array([0.0, -0.6, 0.2])]
    plane, box = sg.plane_mesh(2.0, 2.0), sg.box_mesh(a, per_face_material=False)
    cam = scenes.camera_down((0.0, 0.0, 4.0), 240, 240, fovy_deg=40)
    b = scenes.single_sample([plane, box], [0, 1, 1, 1], [scenes.identity_pose()] + [scenes.pose(t=c) for c in boxes],
                             [cam], seg=[1, 2, 3, 4], lights=[((0.0, 0.0, H), 1.0)])
    sv, si = sg.point_shadow_cameras(np.array([[0.0, 0.0, H]]), R, near=0.02, bias=0.004)
    b = b.with_params(shadow_view=np.pad(sv[None], ((0, 0), (0, 3), (0, 0), (0, 0), (0, 0))).astype(np.float32),
                      shadow_intr=np.pad(si[None], ((0, 0), (0, 3), (0, 0), (0, 0))).astype(np.float32),
                      shadow_res=R, shadow_faces=6)
    o = oracle.render(b, gbuffer=True)
    assert (o["shadow_map"][0, 0] > 0).any(axis=(1, 2)).sum() >= 3       # boxes seen by three faces
    k = (o["gb_mat"] >> 8) & 15
    on_plane = np.nonzero(o["seg"] == 1)[0]
    P = o["gb_pos"][on_plane].astype(np.float64)
    world = np.stack([P[:, 0], P[:, 1], np.zeros(len(P))], 1)            # camera R = identity, plane z = 0
    L = np.array([0.0, 0.0, H])
    margin = 3 * 2.0 / R * 0.7                                           # three texels at 0.7 m
    hit = np.zeros(len(P), bool)
    miss = np.ones(len(P), bool)
    for c in boxes:
        hit |= _ray_hits_box(L, world, c, a, -margin)
        miss &= ~_ray_hits_box(L, world, c, a, margin)
    faces = np.argmax(np.abs(world - L) * np.array([1, 1, 1]), axis=1)
    assert hit.sum() > 300 and miss.sum() > 1000
    assert len(np.unique(faces[hit])) >= 2                              # shadows through different faces
    assert (k[on_plane][hit] == 9).all(), np.bincount(k[on_plane][hit])
    assert (k[on_plane][miss] == 0).all(), np.bincount(k[on_plane][miss])


def test_directional_light_shadows_by_parallel_projection(oracle):
    """A directional light 30 degrees off vertical with an orthographic shadow camera: a floating
    box shadows exactly the plane points whose ray towards the light passes through it (all nine
    taps well inside, none well outside)."""
    th = math.radians(30.0)
    d = np.array([math.sin(th), 0.0, -math.cos(th)])        # the direction the light travels
    a, c, R, half = 0.15, np.array([0.0, 0.0, 0.3]), 192, 1.0
    plane, box = sg.plane_mesh(2.0, 2.0), sg.box_mesh(a, per_face_material=False)
    cam = scenes.camera_down((0.0, 0.0, 4.0), 200, 200, fovy_deg=25)
    b = scenes.single_sample([plane, box], [0, 1], [scenes.identity_pose(), scenes.pose(t=c)], [cam], seg=[1, 2],
                             lights=[(d, 1.0)], light_type=sg.LIGHT_DIRECTIONAL)
    view, intr = sg.directional_shadow_camera(d, (0.0, 0.0, 0.3), half, R, bias=0.004)
    o = oracle.render(_shadowed(b, [view], [intr], R), gbuffer=True)
    k = (o["gb_mat"] >> 8) & 15
    sel = np.nonzero(o["seg"] == 1)[0]
    P = o["gb_pos"][sel].astype(np.float64)
    world = np.stack([P[:, 0], P[:, 1], np.zeros(len(P))], 1)
    far = world - 10.0 * d                                   # a point far along the ray towards the light
    margin = 3 * half / (0.5 * R)                            # three texels
    hit = _ray_hits_box(far, world, c, a, -margin)
    miss = ~_ray_hits_box(far, world, c, a, margin)
    assert hit.sum() > 200 and miss.sum() > 1000
    assert (k[sel][hit] == 9).all(), np.bincount(k[sel][hit])
    assert (k[sel][miss] == 0).all(), np.bincount(k[sel][miss])
    assert (world[hit, 0] > 0.2).mean() > 0.5                 # cast away from the light, along +x
