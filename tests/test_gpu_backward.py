"""GPU shading adjoint (gradients w.r.t. randomized material / light / exposure parameters at fixed
visibility) against the oracle's fp64 adjoint and fp64 central differences, to 1e-3 relative."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_11633_b300 import scenegen as sg
from paper_1906_11633_b300.render import Renderer, ShadeFn, to_numpy

REL = 1e-3


@pytest.fixture(scope="module")
def oracle():
    from oracle import oracle as orc
    orc.build()
    return orc


@pytest.fixture(scope="module")
def renderer():
    return Renderer(sg.hand_meshes())


def rel_err(g, ref):
    scale = max(float(np.abs(ref).max()), 1e-30)
    return np.abs(g - ref) / np.maximum(np.abs(ref), 1e-3 * scale)


def setup(renderer, oracle, batch, seed=0):
    db = renderer.upload(batch)
    out = renderer.render(db, rgb_linear=True, gbuffer=True)
    o = to_numpy(out)
    gb = o["gbuffer"]
    gpos = np.ascontiguousarray(gb[0:3].T)
    gnrm = np.ascontiguousarray(gb[3:6].T)
    gmat = gb[6].view(np.int32).copy()
    mat_t, light_t, ev_t = sg.perturb_params(batch, seed)
    target = oracle.shade_f64(batch, gpos, gnrm, gmat, material=mat_t, light=light_t, exposure_ev=ev_t)
    d_rgb = (2.0 * (o["rgb_linear"].astype(np.float64) - target)).astype(np.float32)
    d_rgb[gmat < 0] = 0.0
    return db, out, (gpos, gnrm, gmat), target, d_rgb


@pytest.mark.parametrize("res", [64, 200])
def test_adjoint_matches_oracle(renderer, oracle, res):
    """At 200 px the full differentiation batch: 256 hand samples x 3 cameras."""
    b = sg.hand_batch(4, np.arange(8 if res == 64 else 256), res=res)
    db, out, gb, target, d_rgb = setup(renderer, oracle, b)
    dm, dl, de = renderer.shade_backward(db, out["gbuffer"], torch.from_numpy(d_rgb).cuda())
    rdm, rdl, rde = oracle.shade_backward_f64(b, *gb, d_rgb.astype(np.float64))
    assert rel_err(dm.cpu().numpy(), rdm).max() < REL
    act = np.arange(4)[None, :] < b.light_meta[:, :1]
    assert rel_err(dl.cpu().numpy()[act], rdl[act]).max() < REL
    assert rel_err(de.cpu().numpy(), rde).max() < REL


def test_adjoint_matches_central_differences(renderer, oracle):
    b = sg.hand_batch(6, np.arange(2), res=48)
    db, out, gb, target, d_rgb = setup(renderer, oracle, b, seed=3)
    dm, dl, de = [t.cpu().numpy() for t in renderer.shade_backward(db, out["gbuffer"], torch.from_numpy(d_rgb).cuda())]
    m, l, e = b.material.astype(np.float64), b.light.astype(np.float64), b.exposure_ev.astype(np.float64)
    fg = gb[2] >= 0

    def loss(mm, ll, ee):
        rgb = oracle.shade_f64(b, *gb, material=mm, light=ll, exposure_ev=ee)
        return ((rgb[fg] - target[fg]) ** 2).sum()

    h = 1e-4
    fd, an = [], []
    used = np.unique(gb[2][fg & (np.arange(len(fg)) < 48 * 48 * 3)])
    checks = [("m", (0, int(k), c)) for k in used[:5] for c in range(4)]
    checks += [("l", (0, li, c)) for li in range(b.light_meta[0, 0]) for c in range(4)] + [("e", (0,))]
    for kind, idx in checks:
        vals = []
        for sgn in (1, -1):
            mm, ll, ee = m.copy(), l.copy(), e.copy()
            {"m": mm, "l": ll, "e": ee}[kind][idx] += sgn * h
            vals.append(loss(mm, ll, ee))
        fd.append((vals[0] - vals[1]) / (2 * h))
        an.append({"m": dm, "l": dl, "e": de}[kind][idx])
    assert rel_err(np.array(an), np.array(fd)).max() < REL


def test_backward_is_bit_identical_run_to_run(renderer, oracle):
    b = sg.hand_batch(9, np.arange(8), res=96)
    db, out, gb, target, d_rgb = setup(renderer, oracle, b)
    g = torch.from_numpy(d_rgb).cuda()
    r1 = [t.clone() for t in renderer.shade_backward(db, out["gbuffer"], g)]
    r2 = [t.clone() for t in renderer.shade_backward(db, out["gbuffer"], g)]
    for a, c in zip(r1, r2):
        assert torch.equal(a, c)


def test_shadefn_autograd(renderer, oracle):
    b = sg.hand_batch(2, np.arange(3), res=64)
    db = renderer.upload(b)
    mat = db.tensors["material"].clone().requires_grad_(True)
    light = db.tensors["light"].clone().requires_grad_(True)
    ev = db.tensors["exposure_ev"].clone().requires_grad_(True)
    rgb = ShadeFn.apply(mat, light, ev, renderer, db)
    tgt = torch.full_like(rgb, 0.25)
    loss = ((rgb - tgt) ** 2).sum()
    loss.backward()
    out = renderer.render(db, rgb_linear=True, gbuffer=True)
    d_rgb = 2.0 * (out["rgb_linear"] - 0.25)
    d_rgb[out["gbuffer"][6].view(torch.int32) < 0] = 0.0
    dm, dl, de = renderer.shade_backward(db, out["gbuffer"], d_rgb)
    assert torch.allclose(mat.grad[..., :4], dm, rtol=1e-5, atol=1e-6)
    assert torch.allclose(light.grad, dl, rtol=1e-5, atol=1e-6)
    assert torch.allclose(ev.grad, de, rtol=1e-5, atol=1e-6)
    assert (mat.grad[..., 4] == 0).all()


def test_spot_and_emission_adjoint_matches_oracle(renderer, oracle):
    """Three spot lights (the cone factor's dependence on the light position) and emissive
    materials: every gradient, d emission included, against the oracle's fp64 adjoint; ShadeFn
    returns d emission when given the emission tensor."""
    b = sg.benchmark_batch(7, np.arange(12), res=96, grading=False)
    b = b.with_params(emission=b.emission + np.float32(0.03))
    db, out, gb, target, d_rgb = setup(renderer, oracle, b)
    dm, dl, de, dem = [t.cpu().numpy() for t in
                       renderer.shade_backward(db, out["gbuffer"], torch.from_numpy(d_rgb).cuda(), emission=True)]
    rdm, rdl, rde, rdem = oracle.shade_backward_f64(b, *gb, d_rgb.astype(np.float64), return_emission=True)
    assert rel_err(dm, rdm).max() < REL
    assert rel_err(dl[:, :3], rdl[:, :3]).max() < REL
    assert rel_err(de, rde).max() < REL
    assert rel_err(dem, rdem).max() < REL
    assert np.abs(rdem).max() > 0
    emission = db.tensors["emission"].clone().requires_grad_(True)
    mat = db.tensors["material"].clone().requires_grad_(True)
    rgb = ShadeFn.apply(mat, db.tensors["light"], db.tensors["exposure_ev"], renderer, db, emission)
    ((rgb - torch.from_numpy(target).float().cuda()) ** 2)[out["gbuffer"][6].view(torch.int32) >= 0].sum().backward()
    assert torch.allclose(emission.grad.cpu(), torch.from_numpy(dem), rtol=1e-4, atol=1e-6)


def test_shadowed_adjoint_matches_oracle(renderer, oracle):
    """With shadow maps the G-buffer's material words carry the shadowed taps, which the adjoint
    holds fixed: every gradient against the oracle's fp64 adjoint of the same G-buffer."""
    b = sg.benchmark_batch(8, np.arange(8), res=96, grading=False, shadow_res=128)
    db, out, gb, target, d_rgb = setup(renderer, oracle, b)
    assert (gb[2][gb[2] >= 0] > 0xff).any()
    dm, dl, de, dem = [t.cpu().numpy() for t in
                       renderer.shade_backward(db, out["gbuffer"], torch.from_numpy(d_rgb).cuda(), emission=True)]
    rdm, rdl, rde, rdem = oracle.shade_backward_f64(b, *gb, d_rgb.astype(np.float64), return_emission=True)
    assert rel_err(dm, rdm).max() < REL
    assert rel_err(dl[:, :3], rdl[:, :3]).max() < REL
    assert rel_err(de, rde).max() < REL
    assert rel_err(dem, rdem).max() < REL


def test_graded_loss_adjoint_matches_oracle(renderer, oracle):
    """A loss on the graded colour (colour grading, Sec. 4.3.1 post-processing randomizer): the
    GPU's rgb_graded equals the oracle's fp64 grading of its linear colour, and the adjoint through
    the grading (material, light, exposure and the seven grading parameters) matches the oracle's
    fp64 adjoint of its step-by-step grading."""
    b = sg.benchmark_batch(8, np.arange(6), res=64)
    assert b.grading is not None
    db = renderer.upload(b)
    out = renderer.render(db, rgb_linear=True, gbuffer=True, rgb_graded=True)
    o = to_numpy(out)
    gb = o["gbuffer"]
    gpos, gnrm = np.ascontiguousarray(gb[0:3].T), np.ascontiguousarray(gb[3:6].T)
    gmat = gb[6].view(np.int32).copy()
    graded = oracle.grade_f64(b, o["rgb_linear"].astype(np.float64))
    assert np.abs(o["rgb_graded"] - graded).max() < 1e-4
    rng = np.random.default_rng(8)
    target = graded + rng.normal(0.0, 0.05, graded.shape)
    d = (2.0 * (o["rgb_graded"].astype(np.float64) - target)).astype(np.float32)
    dm, dl, de, dg = renderer.shade_backward(db, out["gbuffer"], torch.from_numpy(d).cuda(), grading=True)
    rdm, rdl, rde, rdg = oracle.graded_backward_f64(b, gpos, gnrm, gmat, d.astype(np.float64))
    assert rel_err(dm.cpu().numpy(), rdm).max() < REL
    act = np.arange(4)[None, :] < b.light_meta[:, :1]
    assert rel_err(dl.cpu().numpy()[act], rdl[act]).max() < REL
    assert rel_err(de.cpu().numpy(), rde).max() < REL
    got = dg.cpu().numpy()
    for j in range(7):   # per parameter kind, relative to that kind's largest gradient
        assert rel_err(got[:, j], rdg[:, j]).max() < REL, (j, got[:, j], rdg[:, j])
    assert np.all(got[:, 7] == 0.0)
    # ShadeFn with a grading tensor returns rgb_graded and back-propagates into it
    grading = db.tensors["grading"].clone().requires_grad_(True)
    ev = db.tensors["exposure_ev"].clone().requires_grad_(True)
    c = ShadeFn.apply(db.tensors["material"], db.tensors["light"], ev, renderer, db, None, grading)
    assert torch.equal(c, out["rgb_graded"])
    ((c.double() - torch.from_numpy(target).cuda()) ** 2).sum().backward()
    assert torch.allclose(grading.grad, dg, rtol=1e-5, atol=1e-6)
    assert torch.allclose(ev.grad, de, rtol=1e-5, atol=1e-6)
