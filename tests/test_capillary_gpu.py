"""GPU parity of the concentration-gradient (capillary) pair force of Sec. 5.4
inside the fused substep, and of its adjoint, against the FP64 oracle.

The wet block puts most nearest neighbours 1-3% of r apart (inside the
liquid-bridge range, d_r = 0.075 r), a few in contact, under a fluid
fraction that rises in z so that the moisture ratio varies across the
capillary factor's peak.  The bridges' share of a substep is isolated by
running each problem with and without surface tension on both sides.
"""
import dataclasses

import numpy as np
import pytest
import torch

import gic_inputs as gi
import oracle
from gpu_util import FP32, FP64, assert_elementwise, by_id, onset_taint, oracle_inputs, shuffled, sim_for
from paper_2504_00745_gb300 import gic
from paper_2504_00745_gb300.window import Simulator, window_loss_and_grads

pytestmark = pytest.mark.gpu
PRECS = [FP32, FP64]


def _dry(prob):
    return dataclasses.replace(prob, params=dataclasses.replace(prob.params, sigma=0.0))


def _t4(a, prec):
    real = np.float32 if prec == FP32 else np.float64
    a = np.asarray(a, real)
    return torch.from_numpy(np.concatenate([a, np.zeros((a.shape[0], 1), real)], 1)).cuda()


@pytest.mark.parametrize("prec", PRECS)
def test_bridge_forces_of_one_substep_match_oracle(prec):
    """One fused substep (the list build with the bridge reach): the change of
    every granule's velocity that the bridges make (wet minus dry run), per
    element, against the oracle's; and the full state."""
    prob = shuffled(gi.make("wet_block"))
    got, want = {}, {}
    for name, p in (("wet", prob), ("dry", _dry(prob))):
        sim = sim_for(p, prec)
        sim.run(1)
        x, v = sim.positions()
        torch.cuda.synchronize()
        assert gic.gic_check_status() == 0
        got[name] = (x.cpu().numpy(), v.cpu().numpy())
        ref = oracle.run(p, K=1)
        assert ref["status"] == 0
        want[name] = (ref["x"], ref["v"])
    dv_o = want["wet"][1] - want["dry"][1]
    dv_g = got["wet"][1] - got["dry"][1]
    scale = np.abs(dv_o).max()
    assert scale > 1e-6  # the bridges act: ~dt' 2 pi sigma r / m per bridge
    # FP32: velocities of ~0.05 m/s carry ~3e-9 of rounding, 1e-4 of this scale
    tol = 2e-3 if prec == FP32 else 1e-9
    assert np.abs(dv_g - dv_o).max() <= tol * scale
    vref = np.linalg.norm(want["wet"][1], axis=1).max()
    assert np.abs(got["wet"][1] - want["wet"][1]).max() <= (1e-4 if prec == FP32 else 1e-10) * vref
    assert np.abs(got["wet"][0] - want["wet"][0]).max() <= (1e-5 if prec == FP32 else 1e-12) * prob.grid.dx


@pytest.mark.parametrize("prec", PRECS)
def test_window_with_bridges_matches_oracle(prec):
    """Ten substeps with bridges (lists kept between builds): positions,
    velocities, alpha_s and F_s against the oracle's window, on the granules
    whose trajectories do not hang on a contact within rounding of onset."""
    prob = gi.make("wet_block")
    K = 10
    sim = sim_for(prob, prec)
    sim.run(K)
    x, v = sim.positions()
    torch.cuda.synchronize()
    assert gic.gic_check_status() == 0
    ref, taint = onset_taint(prob, K)
    keep = ~taint
    assert keep.sum() > 0.9 * prob.n
    dx = prob.grid.dx
    vref = np.linalg.norm(ref["v"], axis=1).max()
    x, v = x.cpu().numpy(), v.cpu().numpy()
    assert np.abs(x - ref["x"])[keep].max() <= (1e-5 if prec == FP32 else 1e-12) * dx
    assert np.linalg.norm(v - ref["v"], axis=1)[keep].max() <= (1e-4 if prec == FP32 else 1e-10) * vref
    if not taint.any():
        assert np.abs(sim.alpha_s.cpu().numpy() - ref["alpha_s"]).max() <= (1e-9 if prec == FP32 else 1e-12)


@pytest.mark.parametrize("prec", PRECS)
def test_substep_adjoint_with_bridges_matches_oracle(prec):
    """gic_substep_adj with bridges (their position gradient, through the
    pair geometry and through the moisture ratio at the granule) against the
    oracle's integrate, G2P and contact adjoints composed by hand, element by
    element, on a call that builds the lists and on one that walks them."""
    prob = shuffled(gi.make("wet_block"))
    sim = sim_for(prob, prec)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    rng = np.random.default_rng(16)
    gX, gV, gFe = (rng.normal(size=(prob.n, 3)) for _ in range(3))
    ids = sim.B.id.cpu().numpy()
    x, v, r = oracle_inputs(prob)
    gxi, gvi, gFc, gFfl, gaf = oracle.integrate_adj(prob.grid, prob.params, r, gX, gV, gFe)
    gxo, gvo, gc_o = oracle.g2p_adj(prob.grid, prob.params, x, v, r, prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f,
                                    gFfl, gaf, np.zeros(prob.n))
    gxc, gvc, gmu_o = oracle.contact_adj(prob.grid, prob.params, x, v, r, gFc, alpha_f=prob.alpha_f)
    gxc0, _, _ = oracle.contact_adj(prob.grid, _dry(prob).params, x, v, r, gFc)
    assert np.abs(gxc - gxc0).max() > 0.0  # the bridges' share is in the comparison
    want_x, want_v = gxi + gxo + gxc, gvi + gvo + gvc
    F = sim.fluid
    tol = 2e-4 if prec == FP32 else 1e-9
    floor_abs = (2e-6 if prec == FP32 else 1e-14)
    for _ in range(2):
        gp, gv = gic.vec4(prob.n, prec), gic.vec4(prob.n, prec)
        gs = torch.zeros(2, dtype=torch.float64, device="cuda")
        gic.gic_substep_adj(sim.grid, sim.params, sim.B, sim.perm, sim.table, sim.nb, F.u, F.v, F.w, F.p, F.alpha_f,
                            _t4(gX[ids], prec), _t4(gV[ids], prec), _t4(gFe[ids], prec), gp, gv, gs[0:1], gs[1:2])
        torch.cuda.synchronize()
        assert gic.gic_check_status() == 0
        assert_elementwise(by_id(gp, sim.A.id)[:, :3], want_x, tol, floor_abs * np.abs(want_x).max() / tol, "g_x")
        assert_elementwise(by_id(gv, sim.A.id)[:, :3], want_v, tol, floor_abs * np.abs(want_v).max() / tol, "g_v")
        assert abs(float(gs[0]) - gc_o) <= tol * abs(gc_o)
        assert abs(float(gs[1]) - gmu_o) <= tol * abs(gmu_o)


@pytest.mark.parametrize("prec", PRECS)
def test_window_gradients_with_bridges_match_oracle(prec):
    """A 10-substep differentiable window of a small wet block (checkpoints
    every 4 substeps): dL/dv0 element by element, dL/dc_drag and dL/dmu
    against the oracle's adjoint of the same window."""
    prob = gi.make("wet_block", n_side=(3, 3, 3), K=10)
    rng = np.random.default_rng(17)
    prob.target = prob.positions() + rng.normal(size=(prob.n, 3)) * 1e-4
    loss, gv0, gc, gmu, _ = window_loss_and_grads(prob, prec, ckpt=4)
    torch.cuda.synchronize()
    assert gic.gic_check_status() == 0
    out = oracle.run(prob)
    adj = oracle.run_adjoint(prob, 2 * (out["x"] - prob.target) / prob.n)
    tol = 1e-3 if prec == FP32 else 1e-8
    eps_x = (1e-5 if prec == FP32 else 1e-12) * prob.grid.dx
    floor = 10.0 * (2.0 / prob.n) * prob.K * prob.params.dt_sub * eps_x / tol
    assert_elementwise(gv0.cpu().numpy(), adj["g_v0"], tol, floor, "g_v0")
    assert abs(float(gc) - adj["g_c"]) <= tol * abs(adj["g_c"])
    assert abs(float(gmu) - adj["g_mu"]) <= tol * abs(adj["g_mu"])


def test_bridges_need_the_fused_path():
    """The separate contact entry points refuse sigma > 0 with a clear error."""
    prob = gi.make("wet_block")
    sim = Simulator.from_problem(prob, FP32, fused=False)
    with pytest.raises(gic.GicError, match="capillary"):
        sim.run(1)


@pytest.mark.slow
def test_full_size_bridges_one_substep():
    """The 16M-granule sweep (384^3, FCC neighbours 0.145 r apart before the
    jitter, so a fraction of the pairs sit inside d_r = 0.075 r) with
    surface tension 0.07 N/m: one gic_step in the benchmark's launch
    configuration, wet and dry, and the velocity change the bridges make,
    per granule, against the oracle's on a 100k-granule box run with a halo
    wide enough that the box's interior is exact (2 r_max + d_r + 2 dx)."""
    import math

    base = gi.make("scale_sweep_16m")
    wet = dataclasses.replace(base, params=dataclasses.replace(base.params, sigma=0.07))
    got = {}
    for name, p in (("wet", wet), ("dry", base)):
        sim = sim_for(p, FP32)
        sim.run(1)
        x, v = sim.positions()
        torch.cuda.synchronize()
        assert gic.gic_check_status() == 0
        got[name] = v.cpu().numpy()
        del sim
        torch.cuda.empty_cache()
    x0 = base.positions()
    r_max = float(base.r.max())
    d_r = oracle.rupture(r_max, 1e-4 * 4.0 / 3.0 * math.pi * r_max ** 3)
    halo = 2 * r_max + d_r + 2 * base.grid.dx
    lo_all, hi_all = x0.min(0), x0.max(0)
    w = np.sqrt((hi_all[0] - lo_all[0]) * (hi_all[1] - lo_all[1]) * 100_000 / base.n)
    c = 0.5 * (lo_all[:2] + hi_all[:2])
    lo = np.array([c[0] - w / 2, c[1] - w / 2, -1.0])
    hi = np.array([c[0] + w / 2, c[1] + w / 2, 2.0])
    inside = lambda pad: np.all((x0 >= lo - pad) & (x0 < hi + pad), axis=1)
    box, core = np.nonzero(inside(halo))[0], np.nonzero(inside(0.0))[0]
    assert len(core) > 50_000
    sub = lambda p: dataclasses.replace(p, cell=p.cell[box], q=p.q[box], r=p.r[box], v=p.v[box])
    ref_w = oracle.run(sub(wet), K=1)
    ref_d = oracle.run(sub(base), K=1)
    in_core = np.isin(box, core)
    dv_o = (ref_w["v"] - ref_d["v"])[in_core]
    dv_g = (got["wet"] - got["dry"])[box][in_core]
    scale = np.abs(dv_o).max()
    assert scale > 0.0 and np.count_nonzero(np.abs(dv_o).max(axis=1) > 0) > 100  # bridges act on many granules
    assert np.abs(dv_g - dv_o).max() <= 2e-3 * scale
