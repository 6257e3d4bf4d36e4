"""GPU adjoints against the oracle's hand-derived (explicit-Jacobian) adjoint.

Per kernel: the same upstream gradients on the same state; per window: the
gradients of L = mean |x_K - target|^2 w.r.t. the initial velocities, c_drag
and mu from GicWindow (checkpoints every `ckpt` substeps, recompute) against
oracle.run_adjoint and against central finite differences of the FP64 GPU
forward.  Tolerance: relative 1e-3 (FP32), 1e-8 (FP64).
"""
import dataclasses

import numpy as np
import pytest
import torch

import gic_inputs as gi
import oracle
from gpu_util import FP32, FP64, by_id, oracle_inputs, shuffled, sim_for
from paper_2504_00745_gb300 import gic
from paper_2504_00745_gb300.window import Simulator, window_loss_and_grads

pytestmark = pytest.mark.gpu
PRECS = [FP32, FP64]


def _rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


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
    assert _rel(by_id(gpos, sim.B.id)[:, :3], gx_o) < tol
    assert _rel(by_id(gvel, sim.B.id)[:, :3], gv_o) < tol
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
    assert _rel(gpos.cpu().numpy()[:, :3], gx_o) < tol
    assert _rel(gvel.cpu().numpy()[:, :3], gv_o) < tol
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
    for got, w in zip(outs, want):
        assert _rel(got.cpu().numpy()[:, :3], w) < tol


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
    assert _rel(gxo.cpu().numpy()[:, :3], wo) < tol
    assert _rel(gxn.cpu().numpy()[:, :3], wn) < tol
    assert _rel(gfe.cpu().numpy()[:, :3], wf) < tol


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
        assert _rel(by_id(gp, sim.A.id)[:, :3], want_x) < tol
        assert _rel(by_id(gv, sim.A.id)[:, :3], want_v) < tol
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
    assert _rel(gv0.cpu().numpy(), adj["g_v0"]) < tol
    assert abs(float(gc) - adj["g_c"]) <= tol * abs(adj["g_c"]) + 1e-30
    if kind == "contacts":
        assert abs(float(gmu) - adj["g_mu"]) <= tol * abs(adj["g_mu"])
    else:
        assert abs(float(gmu) - adj["g_mu"]) <= tol * max(abs(adj["g_mu"]), 1e-3 * abs(adj["g_c"]))


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
    assert _rel(gv0.cpu().numpy(), adj["g_v0"]) < tol
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


@pytest.mark.slow
def test_differentiable_window_full_size():
    """100,000 granules, 64^3, 50 substeps, checkpoints every 10: FP32 GPU
    gradients against the FP64 oracle's adjoint."""
    prob = gi.make("diff_window_100k")
    loss, gv0, gc, gmu, _ = window_loss_and_grads(prob, FP32, ckpt=10)
    out = oracle.run(prob)
    adj = oracle.run_adjoint(prob, 2 * (out["x"] - prob.target) / prob.n)
    assert _rel(gv0.cpu().numpy(), adj["g_v0"]) < 1e-3
    assert abs(float(gc) - adj["g_c"]) <= 1e-3 * abs(adj["g_c"])
    assert abs(float(gmu) - adj["g_mu"]) <= 1e-3 * max(abs(adj["g_mu"]), 1e-3 * abs(adj["g_c"]))
