"""Verlet-list contact (gic_contact_verlet) against the cell-table walk
(gic_contact) and the oracle: same forces (the pair sums in another order),
rebuilds exactly when a granule has moved more than skin / 2, and a list
overflow that falls back to rebuilding every call."""
import numpy as np
import pytest
import torch

import gic_inputs as gi
import oracle
from gpu_util import FP32, FP64, FS_TOL_FP32, by_id, oracle_inputs, shuffled, tol_force
from paper_2504_00745_gb300 import gic
from paper_2504_00745_gb300.window import Simulator

pytestmark = pytest.mark.gpu
PRECS = [FP32, FP64]


def _forces(sim, verlet):
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    if verlet:
        gic.gic_contact_verlet(sim.grid, sim.params, sim.B, sim.table, sim.nb, sim.F_c)
    else:
        gic.gic_contact(sim.grid, sim.params, sim.B, sim.table, sim.F_c)
    torch.cuda.synchronize()
    return by_id(sim.F_c, sim.B.id)[:, :3].astype(np.float64)


def _tol(prob, prec, F):
    return (tol_force(prob, FP32) + 1e-5 * np.abs(F).max()) if prec == FP32 else 1e-12 * np.abs(F).max()


@pytest.mark.parametrize("name", ["dense_block", "random_cloud"])
@pytest.mark.parametrize("prec", PRECS)
def test_verlet_forces_match_cell_walk_and_oracle(name, prec):
    prob = shuffled(gi.make(name))
    sim = Simulator.from_problem(prob, prec)
    assert sim.nb is not None
    Fv = _forces(sim, True)  # first call builds
    Fv2 = _forces(sim, True)  # second call walks the lists
    Fc = _forces(sim, False)
    assert sim.nb.builds() == 1
    x, v, r = oracle_inputs(prob)
    Fo, _ = oracle.contact(prob.grid, prob.params, x, v, r)
    for F in (Fv, Fv2, Fc):
        assert np.abs(F - Fo).max() <= _tol(prob, prec, Fo)
    assert gic.gic_check_status() == 0


@pytest.mark.parametrize("prec", PRECS)
def test_verlet_rebuilds_only_past_half_skin(prec):
    prob = gi.make("dense_block")
    skin = 0.2 * float(prob.r.max())
    sim = Simulator(prob.grid, prob.params, prob.n, prec, verlet_skin=skin)
    sim.set_fluid(prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)
    sim.set_state(prob.cell, prob.q, prob.r, prob.v)
    _forces(sim, True)
    assert sim.nb.builds() == 1
    # move every granule by 0.4 skin (< skin / 2): the lists stay
    x0 = prob.positions()
    rng = np.random.default_rng(3)
    d = rng.normal(size=x0.shape)
    d *= (0.4 * skin / np.linalg.norm(d, axis=1))[:, None]
    for frac, builds in ((1.0, 1), (1.3, 2)):  # 0.4 skin, then 0.52 skin
        cell, q = gi.encode_positions(x0 + frac * d, prob.grid)
        # repack A directly: set_state would request a rebuild
        dev = lambda a, dt: torch.as_tensor(a).to(device="cuda", dtype=dt).contiguous()
        gic.gic_pack(sim.grid, dev(cell, torch.int32), dev(q.astype(np.int64), torch.int32),
                     dev(prob.r, torch.float32), dev(prob.v, torch.float32), sim.A)
        F = _forces(sim, True)
        assert sim.nb.builds() == builds
        Fo, _ = oracle.contact(prob.grid, prob.params, gi.decode_positions(cell, q, prob.grid), prob.v, prob.r)
        assert np.abs(F - Fo).max() <= _tol(prob, prec, Fo)


@pytest.mark.parametrize("prec", PRECS)
def test_verlet_overflow_rebuilds_every_call(prec):
    prob = shuffled(gi.make("dense_block"))
    sim = Simulator(prob.grid, prob.params, prob.n, prec, verlet_skin=0.15 * float(prob.r.max()), verlet_cap=2)
    sim.set_fluid(prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)
    sim.set_state(prob.cell, prob.q, prob.r, prob.v)
    x, v, r = oracle_inputs(prob)
    Fo, _ = oracle.contact(prob.grid, prob.params, x, v, r)
    for k in range(3):
        F = _forces(sim, True)
        assert sim.nb.overflowed()
        assert sim.nb.builds() == k + 1
        assert np.abs(F - Fo).max() <= _tol(prob, prec, Fo)


@pytest.mark.parametrize("prec", PRECS)
def test_verlet_window_matches_cell_walk_window(prec):
    """20 substeps of the dense block (contacts form and break): the Verlet
    path and the cell walk agree to the rounding of the pair-sum order."""
    prob = shuffled(gi.make("dense_block"))
    out = []
    for verlet in (True, False):
        sim = Simulator.from_problem(prob, prec, verlet=verlet)
        sim.run(20)
        x, v = sim.positions()
        out.append((x.cpu().numpy(), v.cpu().numpy(), sim.alpha_s.cpu().numpy()))
        if verlet:
            assert sim.nb.builds() >= 1
    (xa, va, aa), (xb, vb, ab) = out
    dx = prob.grid.dx
    assert np.abs(xa - xb).max() <= (1e-6 if prec == FP32 else 1e-13) * dx
    vs = np.linalg.norm(vb, axis=1).max()
    assert np.linalg.norm(va - vb, axis=1).max() <= (1e-5 if prec == FP32 else 1e-11) * vs
    assert np.abs(aa - ab).max() <= 1e-10


def test_verlet_argument_errors():
    prob = gi.make("dense_block")
    sim = Simulator.from_problem(prob, FP32)
    nb = gic.Neighbors(prob.n + 1, FP32, cap=8, skin=1e-4)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    with pytest.raises(gic.GicError, match="granules"):
        gic.gic_contact_verlet(sim.grid, sim.params, sim.B, sim.table, nb, sim.F_c)
    bad = gic.Neighbors(prob.n, FP32, cap=0, skin=1e-4)
    with pytest.raises(gic.GicError, match="cap"):
        gic.gic_contact_verlet(sim.grid, sim.params, sim.B, sim.table, bad, sim.F_c)
    neg = gic.Neighbors(prob.n, FP32, cap=8, skin=-1.0)
    with pytest.raises(gic.GicError, match="skin"):
        gic.gic_contact_verlet(sim.grid, sim.params, sim.B, sim.table, neg, sim.F_c)


@pytest.mark.parametrize("name", ["dense_block", "random_cloud"])
@pytest.mark.parametrize("prec", PRECS)
def test_fused_substep_matches_separate_calls(name, prec):
    """gic_substep (contact + G2P + integrate + P2G in one pass) against the
    separate entry points on the same Verlet lists: the same state after 20
    substeps (the same arithmetic in the same order: bit-identical positions
    and velocities), alpha_s identical, F_s to the rounding of its
    fixed-point tile (FP32) or of the atomics' order (FP64)."""
    prob = shuffled(gi.make(name))
    out = []
    # a skin that keeps the window's first lists to its end: a rebuild inside
    # the window orders the granules of a cell by the last sort, which the
    # sort-every-substep path does every substep and the fused path only at
    # rebuilds -- both correct, but the rows (and the force sums) would then
    # run in different orders
    skin = 0.15 * float(prob.r.max())
    for fused in (True, False):
        sim = Simulator.from_problem(prob, prec, fused=fused, skin=skin)
        sim.run(20)
        torch.cuda.synchronize()
        assert gic.gic_check_status() == 0
        x, v = sim.positions()
        out.append((x.cpu().numpy(), v.cpu().numpy(), sim.alpha_s.cpu().numpy(), [f.cpu().numpy() for f in sim.Fs],
                    sim.sums.cpu().numpy()))
    (xa, va, aa, Fa, sa), (xb, vb, ab, Fb, sb) = out
    assert np.array_equal(xa, xb)
    assert np.array_equal(va, vb)
    # FP32: exact integer accumulation; FP64: double atomics in another order (<= ~200 terms of <= 0.3)
    assert np.array_equal(aa, ab) if prec == FP32 else np.abs(aa - ab).max() <= 1e-13
    for fa, fb in zip(Fa, Fb):
        assert np.abs(fa - fb).max() <= (FS_TOL_FP32 if prec == FP32 else 1e-12) * max(np.abs(fb).max(), 1e-300)
    assert np.allclose(sa, sb, rtol=1e-12, atol=0)


def test_fused_substep_argument_errors():
    prob = gi.make("dense_block")
    sim = Simulator.from_problem(prob, FP32)
    F = sim.fluid
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    with pytest.raises(gic.GicError, match="null fluid"):
        gic.gic_substep(sim.grid, sim.params, sim.B, sim.table, sim.nb, None, F.v, F.w, F.p, F.alpha_f, sim.A)
    with pytest.raises(gic.GicError, match="all three"):
        gic.gic_substep(sim.grid, sim.params, sim.B, sim.table, sim.nb, F.u, F.v, F.w, F.p, F.alpha_f, sim.A,
                        Fs=(sim.Fs[0], None, None))
    with pytest.raises(gic.GicError, match="sums2 needs alpha_s"):
        gic.gic_substep(sim.grid, sim.params, sim.B, sim.table, sim.nb, F.u, F.v, F.w, F.p, F.alpha_f, sim.A,
                        sums2=sim.sums)


@pytest.mark.parametrize("name", ["dense_block", "random_cloud"])
@pytest.mark.parametrize("prec", PRECS)
def test_verlet_adjoint_matches_cell_walk(name, prec):
    """gic_contact_verlet_adj against gic_contact_adj on the same state and
    upstream gradient: first call builds the lists, second walks them."""
    prob = shuffled(gi.make(name))
    sim = Simulator.from_problem(prob, prec)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    rng = np.random.default_rng(11)
    real = np.float32 if prec == FP32 else np.float64
    lam = np.concatenate([rng.normal(size=(prob.n, 3)), np.zeros((prob.n, 1))], 1).astype(real)
    gF = torch.from_numpy(lam).cuda()
    out = []
    for verlet in (True, True, False):
        gp, gv = gic.vec4(prob.n, prec), gic.vec4(prob.n, prec)
        gmu = torch.zeros(1, dtype=torch.float64, device="cuda")
        if verlet:
            gic.gic_contact_verlet_adj(sim.grid, sim.params, sim.B, sim.table, sim.nb, sim.F_c, gF, gp, gv, gmu)
        else:
            gic.gic_contact_adj(sim.grid, sim.params, sim.B, sim.table, gF, gp, gv, gmu)
        torch.cuda.synchronize()
        out.append((gp.cpu().numpy()[:, :3], gv.cpu().numpy()[:, :3], float(gmu.item())))
    assert sim.nb.builds() == 1
    ref = out[2]
    tol = 1e-5 if prec == FP32 else 1e-12
    for gp, gv, gm in out[:2]:
        assert np.abs(gp - ref[0]).max() <= tol * np.abs(ref[0]).max()
        assert np.abs(gv - ref[1]).max() <= tol * np.abs(ref[1]).max()
        assert abs(gm - ref[2]) <= tol * abs(ref[2]) + 1e-30


def test_step_graphs_per_configuration():
    """gic_step caches one graph per configuration: two simulators (and a
    change of a parameter) interleaved give the same states as each run
    alone."""
    pa = shuffled(gi.make("dense_block"))
    pb = gi.make("random_cloud")
    alone = []
    for prob in (pa, pb):
        sim = Simulator.from_problem(prob, FP32)
        sim.run(12)
        alone.append(sim.positions()[0].cpu().numpy())
    sa = Simulator.from_problem(pa, FP32)
    sb = Simulator.from_problem(pb, FP32)
    for k in range(12):
        sa.substep(alpha=(k == 11), sums=(k == 11))
        sb.substep(alpha=(k == 11), sums=(k == 11))
    torch.cuda.synchronize()
    assert np.array_equal(sa.positions()[0].cpu().numpy(), alone[0])
    assert np.array_equal(sb.positions()[0].cpu().numpy(), alone[1])
    # a different drag coefficient is a different configuration
    sc = Simulator.from_problem(pa, FP32)
    sc.params.c_drag = 2 * float(pa.params.c_drag)
    sc.run(12)
    assert not np.array_equal(sc.positions()[0].cpu().numpy(), alone[0])
    assert gic.gic_check_status() == 0


@pytest.mark.parametrize("name", ["dense_block", "random_cloud", "plain_fp64_8k"])
def test_staged_build_gives_the_substeps_own_rows(name):
    """gic_step builds the lists of its rebuilding substep on the CTA's staged
    neighbourhood (FP32): the rows, counts and reference entries equal, bit
    for bit, those of the build inside the fused substep (gic_substep on the
    same sorted state), and the build is counted once."""
    prob = shuffled(gi.make(name))
    a = Simulator.from_problem(prob, FP32)
    a.substep(alpha=False, transfer=False, sums=False)  # gic_step: sort + staged build + list walk
    b = Simulator.from_problem(prob, FP32)
    gic.gic_sort(b.grid, b.A, b.B, b.perm, b.table, b.ws)
    b.fused_rest(alpha=False, transfer=False, sums=False)  # gic_substep: the build inside the substep
    torch.cuda.synchronize()
    assert gic.gic_check_status() == 0
    assert a.nb.builds() == 1 and b.nb.builds() == 1
    cnt = a.nb.count.cpu().numpy()
    assert np.array_equal(cnt, b.nb.count.cpu().numpy())
    la, lb = a.nb.list.view(prob.n, -1).cpu().numpy(), b.nb.list.view(prob.n, -1).cpu().numpy()
    for k in range(prob.n):
        assert np.array_equal(la[k, :cnt[k]], lb[k, :cnt[k]])
    assert np.array_equal(a.nb.ref_cell.cpu().numpy(), b.nb.ref_cell.cpu().numpy())
    assert np.array_equal(a.nb.ref_pos.cpu().numpy(), b.nb.ref_pos.cpu().numpy())
    # and the substeps that follow agree with the separate entry points' result state
    xa, va = a.positions()
    xb, vb = b.positions()
    assert np.array_equal(xa.cpu().numpy(), xb.cpu().numpy()) and np.array_equal(va.cpu().numpy(), vb.cpu().numpy())


@pytest.mark.parametrize("name", ["dense_block", "random_cloud"])
def test_neighbors_build_gives_the_rebuilding_substeps_rows(name):
    """gic_neighbors_build on a sorted state writes the rows, counts and
    reference entries that the build inside the fused substep writes for the
    same sorted state (gic_substep after gic_sort), bit for bit, and records
    one build; an FP64 state is refused."""
    prob = shuffled(gi.make(name))
    a = Simulator.from_problem(prob, FP32)
    gic.gic_sort(a.grid, a.A, a.B, a.perm, a.table, a.ws)
    gic.gic_neighbors_reset(a.nb)
    gic.gic_neighbors_build(a.grid, a.B, a.table, a.nb)
    b = Simulator.from_problem(prob, FP32)
    gic.gic_sort(b.grid, b.A, b.B, b.perm, b.table, b.ws)
    b.fused_rest(alpha=False, transfer=False, sums=False)  # gic_substep: the build inside the substep
    torch.cuda.synchronize()
    assert gic.gic_check_status() == 0
    assert a.nb.builds() == 1 and b.nb.builds() == 1
    cnt = a.nb.count.cpu().numpy()
    assert np.array_equal(cnt, b.nb.count.cpu().numpy())
    la, lb = a.nb.list.view(prob.n, -1).cpu().numpy(), b.nb.list.view(prob.n, -1).cpu().numpy()
    for k in range(prob.n):
        assert np.array_equal(la[k, :cnt[k]], lb[k, :cnt[k]])
    assert np.array_equal(a.nb.ref_cell.cpu().numpy(), b.nb.ref_cell.cpu().numpy())
    assert np.array_equal(a.nb.ref_pos.cpu().numpy(), b.nb.ref_pos.cpu().numpy())
    c = Simulator.from_problem(prob, FP64)
    gic.gic_sort(c.grid, c.A, c.B, c.perm, c.table, c.ws)
    with pytest.raises(gic.GicError, match="FP32"):
        gic.gic_neighbors_build(c.grid, c.B, c.table, c.nb)


def test_neighbors_build_overflow_leaves_the_rebuild_to_the_next_call():
    """A list build whose rows would exceed cap records no build and keeps
    the rebuild request: a gic_step that then starts from the sorted state
    rebuilds (in its own 27-cell walk) and gives the same state as a
    simulator whose first gic_step built the lists itself."""
    prob = shuffled(gi.make("dense_block"))
    K = 5
    sims = []
    for prebuilt in (True, False):
        sim = Simulator(prob.grid, prob.params, prob.n, FP32, verlet_skin=0.15 * float(prob.r.max()), verlet_cap=2)
        sim.set_fluid(prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)
        sim.set_state(prob.cell, prob.q, prob.r, prob.v)
        if prebuilt:
            gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
            gic.gic_neighbors_reset(sim.nb)
            gic.gic_neighbors_build(sim.grid, sim.B, sim.table, sim.nb)
            torch.cuda.synchronize()
            assert sim.nb.builds() == 0 and (int(sim.nb.flags[1].item()) & 1)  # overflowed: still requested
            sim.A, sim.B = sim.B, sim.A  # start from the sorted state with these lists
            sim.lists_current = True
        sim.run(K)
        torch.cuda.synchronize()
        assert gic.gic_check_status() == 0
        sims.append(sim)
    xa, va = sims[0].positions()
    xb, vb = sims[1].positions()
    assert np.array_equal(xa.cpu().numpy(), xb.cpu().numpy()) and np.array_equal(va.cpu().numpy(), vb.cpu().numpy())
