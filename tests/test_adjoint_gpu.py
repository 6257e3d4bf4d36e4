"""GPU adjoints against the oracle's hand-derived (explicit-Jacobian) adjoint.

Per kernel: the same upstream gradients on the same state; per window: the
gradients of L = mean |x_K - target|^2 w.r.t. the initial velocities, c_drag
and mu from GicWindow (checkpoints every `ckpt` substeps, recompute) against
oracle.run_adjoint and against central finite differences of the FP64 GPU
forward.  Every array is compared element by element,
|g_i - g_o,i| <= tol * max(|g_o,i|, floor), never through a norm:

* kernel adjoints (random upstream gradients): tol * floor = 2e-6 max_k
  |g_o,k| (FP32; 1e-14 FP64).  An element is a sum of terms of the size of
  the largest elements (the eight tent-weighted samples of an interpolation,
  the pair terms of a contact); FP32 evaluates each to an ulp or so, so an
  element that cancels to near zero keeps an absolute error of ~1e-7 of the
  largest terms: the floor allows twenty such ulps and nothing larger;
* window gradients of L = mean |x_K - target|^2 w.r.t. v0:
  floor = 10 (2 / N) K dt' eps_x / tol, the change of an element when x_K
  moves by the position tolerance eps_x of the precision (1e-5 dx FP32,
  1e-12 dx FP64) with a contact amplification of 10: dL/dv0_i =
  (2 / N) (x_K,i - target_i) dx_K,i/dv0_i and dx_K/dv0 = K dt' for a free
  granule.  Scalars (c_drag, mu) are compared relatively, with no floor.
Tolerance: 1e-3 (FP32), 1e-8 (FP64) for windows.
"""
import dataclasses

import numpy as np
import pytest
import torch

import gic_inputs as gi
import oracle
from gpu_util import FP32, FP64, assert_elementwise, by_id, oracle_inputs, shuffled, sim_for
from paper_2504_00745_gb300 import gic
from paper_2504_00745_gb300.window import Simulator, window_loss_and_grads

pytestmark = pytest.mark.gpu
PRECS = [FP32, FP64]


def _kernel_ok(got, want, tol, what):
    """A kernel adjoint, element by element (absolute floor: twenty FP32 ulps,
    or 1e-14 in FP64, of the largest element; the FP32 tolerances are >= 1e-6)."""
    want = np.asarray(want, float)
    floor_abs = (2e-6 if tol >= 1e-7 else 1e-14) * np.abs(want).max()
    assert_elementwise(got, want, tol, floor_abs / tol, what)


def _gv0_ok(got, want, prob, prec, tol, what="g_v0"):
    """A window's dL/dv0, element by element (floor from the position tolerance)."""
    eps_x = (1e-5 if prec == FP32 else 1e-12) * prob.grid.dx
    floor = 10.0 * (2.0 / prob.n) * prob.K * prob.params.dt_sub * eps_x / tol
    assert_elementwise(got, want, tol, floor, what)


def _t4(a, prec):
    real = np.float32 if prec == FP32 else np.float64
    a = np.asarray(a, real)
    return torch.from_numpy(np.concatenate([a, np.zeros((a.shape[0], 1), real)], 1)).cuda()


@pytest.mark.parametrize("name", ["dense_block", "random_cloud"])
@pytest.mark.parametrize("prec", PRECS)
def test_contact_adjoint_kernel(name, prec):
    prob = shuffled(gi.make(name))
    sim = sim_for(prob, prec)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    rng = np.random.default_rng(1)
    lam = rng.normal(size=(prob.n, 3))
    ids = sim.B.id.cpu().numpy()
    lam_sorted = lam[ids]
    gpos = gic.vec4(prob.n, prec)
    gvel = gic.vec4(prob.n, prec)
    gmu = torch.zeros(1, dtype=torch.float64, device="cuda")
    gic.gic_contact_adj(sim.grid, sim.params, sim.B, sim.table, _t4(lam_sorted, prec), gpos, gvel, gmu)
    torch.cuda.synchronize()
    x, v, r = oracle_inputs(prob)
    gx_o, gv_o, gmu_o = oracle.contact_adj(prob.grid, prob.params, x, v, r, lam)
    tol = 2e-4 if prec == FP32 else 1e-9
    _kernel_ok(by_id(gpos, sim.B.id)[:, :3], gx_o, tol, "contact g_x")
    _kernel_ok(by_id(gvel, sim.B.id)[:, :3], gv_o, tol, "contact g_v")
    assert abs(float(gmu.item()) - gmu_o) <= tol * abs(gmu_o)


@pytest.mark.parametrize("prec", PRECS)
def test_g2p_adjoint_kernel(prec):
    prob = gi.make("random_cloud")
    sim = sim_for(prob, prec)
    rng = np.random.default_rng(2)
    lF, la, lal = rng.normal(size=(prob.n, 3)), rng.normal(size=(prob.n, 3)), rng.normal(size=prob.n)
    gpos = gic.vec4(prob.n, prec)
    gvel = gic.vec4(prob.n, prec)
    gc = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = sim.fluid
    real = torch.float32 if prec == FP32 else torch.float64
    gic.gic_g2p_couple_adj(sim.grid, sim.params, sim.A, F.u, F.v, F.w, F.p, F.alpha_f, _t4(lF, prec), _t4(la, prec),
                           torch.tensor(lal, dtype=real, device="cuda"), gpos, gvel, gc)
    torch.cuda.synchronize()
    x, v, r = oracle_inputs(prob)
    gx_o, gv_o, gc_o = oracle.g2p_adj(prob.grid, prob.params, x, v, r, prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f,
                                      lF, la, lal)
    tol = 1e-5 if prec == FP32 else 1e-11
    _kernel_ok(gpos.cpu().numpy()[:, :3], gx_o, tol, "g2p g_x")
    _kernel_ok(gvel.cpu().numpy()[:, :3], gv_o, tol, "g2p g_v")
    assert abs(float(gc.item()) - gc_o) <= tol * abs(gc_o)


@pytest.mark.parametrize("prec", PRECS)
def test_integrate_adjoint_kernel(prec):
    prob = gi.make("random_cloud")
    sim = sim_for(prob, prec)
    rng = np.random.default_rng(3)
    gX, gV, gF = (rng.normal(size=(prob.n, 3)) for _ in range(3))
    outs = [gic.vec4(prob.n, prec) for _ in range(5)]
    gic.gic_integrate_adj(sim.grid, sim.params, sim.A, _t4(gX, prec), _t4(gV, prec), _t4(gF, prec), *outs)
    torch.cuda.synchronize()
    want = oracle.integrate_adj(prob.grid, prob.params, prob.r.astype(float), gX, gV, gF)
    tol = 1e-6 if prec == FP32 else 1e-13
    for k, (got, w) in enumerate(zip(outs, want)):
        _kernel_ok(got.cpu().numpy()[:, :3], w, tol, f"integrate output {k}")


@pytest.mark.parametrize("prec", PRECS)
def test_p2g_adjoint_kernel(prec):
    prob = gi.make("random_cloud")
    sim = sim_for(prob, prec)
    rng = np.random.default_rng(4)
    # moved copy of the state
    x, v, r = oracle_inputs(prob)
    m = prob.params.rho_s * 4 / 3 * np.pi * r ** 3
    Fc = rng.normal(size=(prob.n, 3)) * 3000 * 9.8 * m[:, None]
    z = np.zeros((prob.n, 3))
    gic.gic_integrate(sim.grid, sim.params, sim.A, _t4(Fc, prec), _t4(z, prec), _t4(z, prec), sim.B, sim.f_ex)
    fex = rng.normal(size=(prob.n, 3))
    sim.f_ex.copy_(_t4(fex, prec))
    g = prob.grid
    real = torch.float32 if prec == FP32 else torch.float64
    ga = rng.normal(size=g.nx * g.ny * g.nz)
    gFs = [rng.normal(size=k) for k in ((g.nx + 1) * g.ny * g.nz, g.nx * (g.ny + 1) * g.nz, g.nx * g.ny * (g.nz + 1))]
    gxo = gic.vec4(prob.n, prec)
    gxn = gic.vec4(prob.n, prec)
    gfe = gic.vec4(prob.n, prec)
    gic.gic_p2g_adj(sim.grid, sim.params, sim.A, sim.B, sim.f_ex, torch.tensor(ga, device="cuda"),
                    [torch.tensor(a, dtype=real, device="cuda") for a in gFs], gxo, gxn, gfe)
    torch.cuda.synchronize()
    xa, _ = sim.positions(sim.A)
    xb, _ = sim.positions(sim.B)
    wo, wn, wf = oracle.p2g_adj(g, prob.params, xa.cpu().numpy(), xb.cpu().numpy(), r, fex, ga, gFs)
    tol = 1e-5 if prec == FP32 else 1e-11
    _kernel_ok(gxo.cpu().numpy()[:, :3], wo, tol, "p2g g_x_old")
    _kernel_ok(gxn.cpu().numpy()[:, :3], wn, tol, "p2g g_x_new")
    _kernel_ok(gfe.cpu().numpy()[:, :3], wf, tol, "p2g g_f_ex")


@pytest.mark.parametrize("name", ["dense_block", "random_cloud"])
@pytest.mark.parametrize("prec", PRECS)
def test_substep_adjoint_matches_oracle(name, prec):
    """gic_substep_adj (the integrate, G2P and contact adjoints in one pass,
    scattered through the sort's permutation) against the oracle's
    integrate_adj, g2p_adj and contact_adj composed by hand, on a call that
    builds the Verlet lists and on one that walks them."""
    prob = shuffled(gi.make(name))
    sim = sim_for(prob, prec)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    rng = np.random.default_rng(6)
    gX, gV, gFe = (rng.normal(size=(prob.n, 3)) for _ in range(3))
    ids = sim.B.id.cpu().numpy()  # sorted index -> id
    x, v, r = oracle_inputs(prob)
    gxi, gvi, gFc, gFfl, gaf = oracle.integrate_adj(prob.grid, prob.params, r, gX, gV, gFe)
    gxo, gvo, gc_o = oracle.g2p_adj(prob.grid, prob.params, x, v, r, prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f,
                                    gFfl, gaf, np.zeros(prob.n))
    gxc, gvc, gmu_o = oracle.contact_adj(prob.grid, prob.params, x, v, r, gFc)
    want_x, want_v = gxi + gxo + gxc, gvi + gvo + gvc
    F = sim.fluid
    tol = 2e-4 if prec == FP32 else 1e-9
    for _ in range(2):
        gp, gv = gic.vec4(prob.n, prec), gic.vec4(prob.n, prec)
        gs = torch.zeros(2, dtype=torch.float64, device="cuda")
        gic.gic_substep_adj(sim.grid, sim.params, sim.B, sim.perm, sim.table, sim.nb, F.u, F.v, F.w, F.p, F.alpha_f,
                            _t4(gX[ids], prec), _t4(gV[ids], prec), _t4(gFe[ids], prec), gp, gv, gs[0:1], gs[1:2])
        torch.cuda.synchronize()
        assert gic.gic_check_status() == 0
        _kernel_ok(by_id(gp, sim.A.id)[:, :3], want_x, tol, "substep g_x")
        _kernel_ok(by_id(gv, sim.A.id)[:, :3], want_v, tol, "substep g_v")
        assert abs(float(gs[0]) - gc_o) <= tol * abs(gc_o)
        assert abs(float(gs[1]) - gmu_o) <= tol * abs(gmu_o)
    assert sim.nb.builds() == 1


def test_substep_adjoint_argument_errors():
    prob = gi.make("dense_block")
    sim = sim_for(prob, FP32)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    F = sim.fluid
    g = [gic.vec4(prob.n, FP32) for _ in range(4)]

    def call(u, gpo, gvo, gpi, gvi):
        gic.gic_substep_adj(sim.grid, sim.params, sim.B, sim.perm, sim.table, sim.nb, u, F.v, F.w, F.p, F.alpha_f,
                            gpo, gvo, None, gpi, gvi)

    with pytest.raises(gic.GicError, match="aliases an input"):
        call(F.u, g[0], g[1], g[0], g[3])
    with pytest.raises(gic.GicError, match="g_pos_in aliases g_vel_in"):
        call(F.u, g[0], g[1], g[2], g[2])
    with pytest.raises(gic.GicError, match="null gradient"):
        call(F.u, g[0], None, g[2], g[3])
    with pytest.raises(gic.GicError, match="null fluid"):
        call(None, g[0], g[1], g[2], g[3])


def _window_case(kind):
    if kind == "contacts":
        prob = gi.make("dense_block", n_side=(4, 4, 4))
        prob.K = 10
        rng = np.random.default_rng(9)
        prob.target = prob.positions() + rng.normal(size=(prob.n, 3)) * 1e-4
        return prob
    return gi.make("diff_window_100k", n=1000, grid_n=16)


@pytest.mark.parametrize("kind,ckpt", [("contacts", 10), ("contacts", 3), ("loose", 10)])
@pytest.mark.parametrize("prec", PRECS)
def test_window_gradients_match_oracle_adjoint(kind, ckpt, prec):
    prob = _window_case(kind)
    loss, gv0, gc, gmu, sim = window_loss_and_grads(prob, prec, ckpt=ckpt)
    torch.cuda.synchronize()
    assert gic.gic_check_status() == 0
    out = oracle.run(prob)
    gxK = 2 * (out["x"] - prob.target) / prob.n
    adj = oracle.run_adjoint(prob, gxK)
    L_o = np.mean(np.sum((out["x"] - prob.target) ** 2, axis=1))
    tol = 1e-3 if prec == FP32 else 1e-8
    assert abs(float(loss) - L_o) <= (1e-6 if prec == FP32 else 1e-12) * L_o
    _gv0_ok(gv0.cpu().numpy(), adj["g_v0"], prob, prec, tol)
    assert abs(float(gc) - adj["g_c"]) <= tol * abs(adj["g_c"])
    assert abs(float(gmu) - adj["g_mu"]) <= tol * abs(adj["g_mu"])
    if kind == "contacts":
        assert abs(adj["g_mu"]) > 0.0


@pytest.mark.parametrize("path", ["rebuild_every_substep", "rebuild_inside_segments", "sorted_every_substep"])
@pytest.mark.parametrize("prec", PRECS)
def test_window_gradient_paths(path, prec):
    """The window's backward passes against the oracle's adjoint: with a skin
    so thin that every substep rebuilds the Verlet lists (going back restores
    another build's lists before every substep), with one that rebuilds in
    the middle of checkpoint segments (the substeps before it walk the lists
    kept with the checkpoint; the granules fall about 5e-5 m in the first
    five substeps), and without the fused path (every substep sorted,
    separate adjoint kernels)."""
    prob = _window_case("contacts")
    kw = {"rebuild_every_substep": dict(skin=1e-12), "rebuild_inside_segments": dict(skin=8e-5),
          "sorted_every_substep": dict(fused=False)}[path]
    if path != "sorted_every_substep":
        sim = Simulator.from_problem(prob, prec, **kw)
        sim.run(prob.K)
        # builds at every substep; or at substeps 0 and 5 (and maybe 8 or 9)
        assert sim.nb.builds() == prob.K if path == "rebuild_every_substep" else sim.nb.builds() in (2, 3)
    loss, gv0, gc, gmu, _ = window_loss_and_grads(prob, prec, ckpt=4, **kw)
    torch.cuda.synchronize()
    assert gic.gic_check_status() == 0
    out = oracle.run(prob)
    adj = oracle.run_adjoint(prob, 2 * (out["x"] - prob.target) / prob.n)
    tol = 1e-3 if prec == FP32 else 1e-8
    _gv0_ok(gv0.cpu().numpy(), adj["g_v0"], prob, prec, tol)
    assert abs(float(gc) - adj["g_c"]) <= tol * abs(adj["g_c"])
    assert abs(float(gmu) - adj["g_mu"]) <= tol * abs(adj["g_mu"])


def test_window_gradients_match_gpu_fd():
    """FP32 adjoint against central FD (h = 1e-4 relative) of the FP64 GPU
    forward, on the contact window (contact-stable: checked with the oracle's
    signature)."""
    prob = _window_case("contacts")
    loss, gv0, gc, gmu, _ = window_loss_and_grads(prob, FP32)

    def L(v=None, P=None):
        p = dataclasses.replace(prob, v=(prob.v if v is None else v).astype(np.float32),
                                params=prob.params if P is None else P)
        sim = Simulator.from_problem(p, FP64)
        if v is not None:
            sim.A.vel[:, :3] = torch.tensor(v, dtype=torch.float64, device="cuda")
        sim.run(prob.K, alpha_every=False)
        x, _ = sim.positions()
        return float(((x.cpu().numpy() - prob.target) ** 2).sum(1).mean())

    P = prob.params
    hm = 1e-4 * P.mu_fric
    fd_mu = (L(P=dataclasses.replace(P, mu_fric=P.mu_fric + hm)) - L(P=dataclasses.replace(P, mu_fric=P.mu_fric - hm))) / (2 * hm)
    assert abs(float(gmu) - fd_mu) <= 1e-3 * abs(fd_mu)
    hc = 1e-4 * P.c_drag
    fd_c = (L(P=dataclasses.replace(P, c_drag=P.c_drag + hc)) - L(P=dataclasses.replace(P, c_drag=P.c_drag - hc))) / (2 * hc)
    assert abs(float(gc) - fd_c) <= 1e-3 * abs(fd_c)
    rng = np.random.default_rng(5)
    w = rng.normal(size=(prob.n, 3))
    v0 = prob.v.astype(np.float64)
    h = 1e-4 * np.abs(v0).max()
    fd_v = (L(v=v0 + h * w) - L(v=v0 - h * w)) / (2 * h)
    assert abs(float((gv0.cpu().numpy() * w).sum()) - fd_v) <= 1e-3 * abs(fd_v)


def _window_loss_fp64(prob, v=None, P=None, count_contacts=False):
    """L = mean |x_K - target|^2 from the FP64 GPU forward (v: initial
    velocities, P: parameters), and with count_contacts the number of contact
    pairs before each substep (the window's contact signature)."""
    p = dataclasses.replace(prob, v=(prob.v if v is None else v).astype(np.float32),
                            params=prob.params if P is None else P)
    sim = Simulator.from_problem(p, FP64)
    if v is not None:
        sim.A.vel[:, :3] = torch.tensor(v, dtype=torch.float64, device="cuda")
    counts = []
    partners = torch.zeros(prob.n, dtype=torch.int32, device="cuda")
    for _ in range(prob.K):
        if count_contacts:
            gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
            gic.gic_contact_pairs(sim.grid, sim.B, sim.table, counts=partners)
            counts.append(int(partners.sum().item()) // 2)
        sim.substep(alpha=False, transfer=False, sums=False)
    x, _ = sim.positions()
    return float(((x.cpu().numpy() - prob.target) ** 2).sum(1).mean()), counts


@pytest.mark.slow
def test_differentiable_window_full_size():
    """100,000 granules, 64^3, 50 substeps, checkpoints every 10: FP32 GPU
    gradients against the FP64 oracle's adjoint, element by element, and
    against central finite differences (h = 1e-4 relative) of the FP64 GPU
    forward on this configuration itself: dL/dv0 . w for a seeded direction
    w, dL/dc_drag and dL/dmu.  The loose packing (volume fraction 0.3,
    smallest initial gap 0.01 r) stays contact-free for the whole window in
    all these runs (asserted: that makes every finite difference
    contact-stable), so dL/dmu is exactly zero here on both sides; the mu
    gradient is compared against the oracle and finite differences on the
    contact windows above."""
    prob = gi.make("diff_window_100k")
    loss, gv0, gc, gmu, _ = window_loss_and_grads(prob, FP32, ckpt=10)
    out = oracle.run(prob)
    adj = oracle.run_adjoint(prob, 2 * (out["x"] - prob.target) / prob.n)
    _gv0_ok(gv0.cpu().numpy(), adj["g_v0"], prob, FP32, 1e-3)
    assert abs(float(gc) - adj["g_c"]) <= 1e-3 * abs(adj["g_c"])
    assert float(gmu) == 0.0 and adj["g_mu"] == 0.0
    # central differences of the FP64 GPU forward, h = 1e-4 relative
    P = prob.params
    L0, c0 = _window_loss_fp64(prob, count_contacts=True)
    assert abs(L0 - float(loss)) <= 1e-6 * L0
    hc = 1e-4 * P.c_drag
    Lp, cp = _window_loss_fp64(prob, P=dataclasses.replace(P, c_drag=P.c_drag + hc), count_contacts=True)
    Lm, cm = _window_loss_fp64(prob, P=dataclasses.replace(P, c_drag=P.c_drag - hc), count_contacts=True)
    fd_c = (Lp - Lm) / (2 * hc)
    assert abs(float(gc) - fd_c) <= 1e-3 * abs(fd_c)
    hm = 1e-4 * P.mu_fric
    Lp_mu, _ = _window_loss_fp64(prob, P=dataclasses.replace(P, mu_fric=P.mu_fric + hm))
    Lm_mu, _ = _window_loss_fp64(prob, P=dataclasses.replace(P, mu_fric=P.mu_fric - hm))
    assert (Lp_mu - Lm_mu) / (2 * hm) == 0.0
    rng = np.random.default_rng(7)
    w = rng.normal(size=(prob.n, 3))
    v0 = prob.v.astype(np.float64)
    h = 1e-4 * np.abs(v0).max()
    Lvp, cvp = _window_loss_fp64(prob, v=v0 + h * w, count_contacts=True)
    Lvm, cvm = _window_loss_fp64(prob, v=v0 - h * w, count_contacts=True)
    fd_v = (Lvp - Lvm) / (2 * h)
    assert abs(float((gv0.cpu().numpy() * w).sum()) - fd_v) <= 1e-3 * abs(fd_v)
    for counts in (c0, cp, cm, cvp, cvm):
        assert len(counts) == prob.K and max(counts) == 0
