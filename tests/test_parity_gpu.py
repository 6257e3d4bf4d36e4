"""GPU parity: every step of the substep through the C ABI against the FP64
oracle, element by element, on seeded inputs.

Tolerances (stated by the workload definition for the FP32 path, derived from
the arithmetic where it states none):
  * sort permutation, cell table and contact-pair sets: bit-exact;
  * after 10 substeps: positions <= 1e-5 dx, velocities <= 1e-4 v_ref
    (v_ref = largest oracle speed), alpha_s <= 1e-9 absolute;
  * single kernels: see each test.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

import gic_inputs as gi
import oracle
from gpu_util import (FP32, FP64, FS_TOL_FP32, by_id, onset_taint, oracle_inputs, shuffled, sim_for, subset,
                      tol_force)
from paper_2504_00745_gb300 import gic
from paper_2504_00745_gb300.window import Simulator

pytestmark = pytest.mark.gpu

SMALL = ["plain_fp64_8k", "dense_block", "random_cloud"]
PRECS = [FP32, FP64]


@pytest.fixture(autouse=True)
def _clear_status():
    torch.cuda.synchronize()
    gic.gic_check_status(clear=True)
    yield


def _problem(name, shuffle=True):
    p = gi.make(name)
    return shuffled(p) if shuffle else p


# ----------------------------------------------------------------------------- a1 sort

@pytest.mark.parametrize("name", SMALL + ["ragged_2049", "ragged_6145"])
@pytest.mark.parametrize("prec", PRECS)
def test_sort_bit_exact(name, prec):
    if name.startswith("ragged"):
        base = shuffled(gi.make("dense_block", n_side=(10, 10, 10)))
        prob = subset(base, int(name.split("_")[1]))
    else:
        prob = _problem(name)
    sim = sim_for(prob, prec)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    torch.cuda.synchronize()
    x, _, _ = oracle_inputs(prob)
    c = oracle.cells(prob.grid, x)
    assert np.array_equal(c, prob.cell)
    perm_o, keys_o = oracle.sort(c)
    perm_g = sim.perm.cpu().numpy()
    assert np.array_equal(perm_g, perm_o)
    # the state moved with the permutation, ids included
    assert np.array_equal(sim.B.id.cpu().numpy(), perm_o)
    assert torch.equal(sim.B.pos.cpu(), sim.A.pos.cpu()[perm_o])
    assert torch.equal(sim.B.vel.cpu(), sim.A.vel.cpu()[perm_o])
    assert torch.equal(sim.B.cell.cpu(), sim.A.cell.cpu()[perm_o])
    # cell table: exactly the occupied cells carry the current epoch, with the
    # oracle's (start, count)
    ck, st, ct = oracle.cell_table(keys_o)
    tab = sim.table.view(-1, 4).cpu().numpy().astype(np.int64)
    epoch = tab[0, 0]
    assert epoch >= 1
    nc = prob.grid.nc
    cs = c[perm_o[st]]
    lin = 1 + cs[:, 0] + nc[0] * (cs[:, 1] + nc[1] * cs[:, 2])
    assert np.array_equal(tab[lin, 0], st)
    assert np.array_equal(tab[lin, 1], ct)
    assert np.all(tab[lin, 2] == epoch)
    assert int((tab[1:, 2] == epoch).sum()) == len(ck)


def test_sort_epochs_do_not_leak_between_calls():
    """A second sort of a different state must not see cells occupied only in
    the first one (the epoch tag retires them without a clear)."""
    prob = _problem("dense_block")
    sim = sim_for(prob, FP32)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    prob2 = subset(prob, 100)
    sim2 = Simulator(prob2.grid, prob2.params, prob2.n)
    sim2.table = sim.table  # reuse the table
    sim2.set_fluid(prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)
    sim2.set_state(prob2.cell, prob2.q, prob2.r, prob2.v)
    gic.gic_sort(sim2.grid, sim2.A, sim2.B, sim2.perm, sim2.table, sim2.ws)
    torch.cuda.synchronize()
    tab = sim.table.view(-1, 4).cpu().numpy()
    epoch = tab[0, 0]
    occupied = len(np.unique(prob2.cell, axis=0))
    assert int((tab[1:, 2] == epoch).sum()) == occupied


# ----------------------------------------------------------------------------- a2 contact

@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("prec", PRECS)
def test_contact_pairs_bit_exact(name, prec):
    prob = _problem(name)
    sim = sim_for(prob, prec)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    counts = torch.zeros(prob.n, dtype=torch.int32, device="cuda")
    cap = 20 * prob.n
    pairs = torch.zeros((cap, 2), dtype=torch.int32, device="cuda")
    npairs = torch.zeros(1, dtype=torch.int64, device="cuda")
    gic.gic_contact_pairs(sim.grid, sim.B, sim.table, counts, pairs, npairs)
    torch.cuda.synchronize()
    m = int(npairs.item())
    assert m <= cap
    got = set(map(tuple, pairs[:m].cpu().numpy().tolist()))
    x, v, r = oracle_inputs(prob)
    want = oracle.contact_pairs(prob.grid, x, r, brute=prob.n <= 3000)
    want = set(map(tuple, np.sort(want, axis=1).tolist()))
    assert got == want
    per = np.zeros(prob.n, np.int64)
    for a, b in want:
        per[a] += 1
        per[b] += 1
    assert np.array_equal(by_id(counts, sim.B.id), per)


@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("walls", [1, 0])
def test_contact_force_parity(name, prec, walls):
    prob = _problem(name)
    prob.params.walls = walls
    sim = sim_for(prob, prec)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    gic.gic_contact(sim.grid, sim.params, sim.B, sim.table, sim.F_c)
    torch.cuda.synchronize()
    assert gic.gic_check_status() == 0
    F = by_id(sim.F_c, sim.B.id)[:, :3].astype(np.float64)
    x, v, r = oracle_inputs(prob)
    Fo, st = oracle.contact(prob.grid, prob.params, x, v, r)
    assert st == 0
    scale = max(np.abs(Fo).max(), 1e-30)
    atol = tol_force(prob, prec) + (1e-5 if prec == FP32 else 1e-11) * scale
    assert np.abs(F - Fo).max() <= atol, (np.abs(F - Fo).max(), atol, scale)


# ----------------------------------------------------------------------------- a3 G2P

@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("prec", PRECS)
def test_g2p_parity(name, prec):
    prob = _problem(name)
    sim = sim_for(prob, prec)
    F = sim.fluid
    gic.gic_g2p_couple(sim.grid, sim.params, sim.A, F.u, F.v, F.w, F.p, F.alpha_f, sim.F_fl, sim.a_f, sim.alpha_f_p)
    torch.cuda.synchronize()
    x, v, r = oracle_inputs(prob)
    Ffl_o, af_o, alp_o = oracle.g2p(prob.grid, prob.params, x, v, r, prob.u, prob.vf, prob.wf, prob.p,
                                     prob.alpha_f)
    rtol = 2e-6 if prec == FP32 else 1e-12
    Ffl = sim.F_fl.cpu().numpy()[:, :3]
    af = sim.a_f.cpu().numpy()[:, :3]
    alp = sim.alpha_f_p.cpu().numpy()
    e = np.abs(Ffl - Ffl_o)
    k = np.unravel_index(np.argmax(e), e.shape)
    assert e.max() <= rtol * np.abs(Ffl_o).max(), (e.max(), np.abs(Ffl_o).max(), k, Ffl[k[0]], Ffl_o[k[0]],
                                                    x[k[0]], v[k[0]])
    # a_f = g - grad p / rho_f cancels to ~0 in hydrostatic fluid: the scale is |g|
    ascale = max(np.abs(af_o).max(), np.linalg.norm(prob.params.g))
    assert np.abs(af - af_o).max() <= rtol * ascale, (np.abs(af - af_o).max(), ascale)
    assert np.abs(alp - alp_o).max() <= rtol, np.abs(alp - alp_o).max()


# ----------------------------------------------------------------------------- a4 integrate

@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("prec", PRECS)
def test_integrate_parity(name, prec):
    prob = _problem(name)
    sim = sim_for(prob, prec)
    x, v, r = oracle_inputs(prob)
    rng = np.random.default_rng(3)
    m = prob.params.rho_s * 4 / 3 * np.pi * r ** 3
    # forces of a few hundred g, rounded to the GPU's precision so both sides read the same numbers
    real = np.float32 if prec == FP32 else np.float64
    Fc = (rng.normal(size=(prob.n, 3)) * 300 * 9.8 * m[:, None]).astype(real)
    Ffl = (rng.normal(size=(prob.n, 3)) * 3 * 9.8 * m[:, None]).astype(real)
    af = rng.normal(size=(prob.n, 3)).astype(real) * real(5)
    to4 = lambda a: torch.from_numpy(np.concatenate([a, np.zeros((prob.n, 1), real)], 1)).cuda()
    gic.gic_integrate(sim.grid, sim.params, sim.A, to4(Fc), to4(Ffl), to4(af), sim.B, sim.f_ex)
    torch.cuda.synchronize()
    xg, vg = sim.positions(sim.B)
    xo, vo, fo, st = oracle.integrate(prob.grid, prob.params, x, v, r, Fc, Ffl, af)
    unit = prob.grid.h_c * 2.0 ** -30
    xtol = 2 * unit if prec == FP32 else 1e-15
    assert np.abs(xg.cpu().numpy() - xo).max() <= xtol
    vtol = 2e-6 if prec == FP32 else 1e-13
    assert np.abs(vg.cpu().numpy() - vo).max() <= vtol * np.abs(vo).max()
    fg = sim.f_ex.cpu().numpy()[:, :3]
    assert np.abs(fg - fo).max() <= vtol * np.abs(fo).max()
    assert np.array_equal(sim.B.id.cpu().numpy(), np.arange(prob.n))


# ----------------------------------------------------------------------------- a5 P2G

def _conserved(sums, prec):
    """sums = [sum_c alpha_s dx^3, sum_i V_i].  FP32 path: both are exact
    128-bit integer totals in 2^-53 units (the cells' alpha_s and the
    granules' S_i = V_i / dx^3, which every granule deposits in full), each
    rounded once to a double, so exact conservation makes them bitwise
    equal.  FP64 path: FP64 atomics, equal to 1e-12 (the rounding of the
    ~8n-term sums)."""
    if prec == FP32:
        assert sums[0] == sums[1], (sums[0], sums[1])
    else:
        assert abs(sums[0] - sums[1]) <= 1e-12 * sums[1]



@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("prec", PRECS)
def test_p2g_parity(name, prec):
    prob = _problem(name)
    sim = sim_for(prob, prec)
    real = np.float32 if prec == FP32 else np.float64
    rng = np.random.default_rng(5)
    # a moved copy of the state: one substep with arbitrary forces
    x, v, r = oracle_inputs(prob)
    m = prob.params.rho_s * 4 / 3 * np.pi * r ** 3
    Fc = (rng.normal(size=(prob.n, 3)) * 3000 * 9.8 * m[:, None]).astype(real)
    z = np.zeros((prob.n, 3), real)
    to4 = lambda a: torch.from_numpy(np.concatenate([a, np.zeros((prob.n, 1), real)], 1)).cuda()
    gic.gic_integrate(sim.grid, sim.params, sim.A, to4(Fc), to4(z), to4(z), sim.B, sim.f_ex)
    fex = (rng.normal(size=(prob.n, 3)) * 9.8 * m[:, None]).astype(real)
    sim.f_ex.copy_(to4(fex))
    sim.zero_transfer()
    gic.gic_p2g(sim.grid, sim.params, sim.A, sim.B, sim.f_ex, sim.alpha_s, sim.Fs, sim.sums)
    torch.cuda.synchronize()
    xa, _ = sim.positions(sim.A)
    xb, _ = sim.positions(sim.B)
    a_o, Fs_o, sums_o = oracle.p2g(prob.grid, prob.params, xa.cpu().numpy(), xb.cpu().numpy(), r, fex)
    ag = sim.alpha_s.cpu().numpy()
    assert np.abs(ag - a_o).max() <= 1e-9, np.abs(ag - a_o).max()
    sums = sim.sums.cpu().numpy()
    assert abs(sums[1] - sums_o[1]) <= 1e-12 * sums_o[1]  # n-term FP64 sums in different orders
    _conserved(sums, prec)
    ftol = FS_TOL_FP32 if prec == FP32 else 1e-12
    for c in range(3):
        fg = sim.Fs[c].cpu().numpy()
        assert np.abs(fg - Fs_o[c]).max() <= ftol * np.abs(Fs_o[c]).max(), (c, np.abs(fg - Fs_o[c]).max(),
                                                                            np.abs(Fs_o[c]).max())


def test_alpha_s_integer_totals_are_equal():
    """FP32 path, exact conservation as integers: on a 1/32 grid (dx^3 =
    2^-15, so the scaling by dx^3 is exact) with a total volume fraction
    below 1 (so every conversion of a 2^-53 integer to a double is exact),
    the cells' integers summed in Python, the cell total and the granule
    total of gic_p2g are one and the same integer."""
    prob = subset(gi.make("dense_block"), 100)
    assert prob.grid.dx == 1.0 / 32
    sim = sim_for(prob, FP32)
    gic.gic_p2g(sim.grid, sim.params, sim.A, sim.A, None, sim.alpha_s, (None, None, None), sim.sums)
    torch.cuda.synchronize()
    a = sim.alpha_s.cpu().numpy()
    assert a.sum() < 1.0
    cells = sum(int(np.ldexp(val, 53)) for val in a if val != 0.0)
    assert all(np.ldexp(val, 53) == int(np.ldexp(val, 53)) for val in a)
    s0, s1 = (int(np.ldexp(float(t), 68)) for t in sim.sums.cpu().numpy())
    assert cells == s0 == s1
    V = 4.0 / 3.0 * np.pi * prob.r.astype(np.float64) ** 3
    assert abs(cells - np.ldexp(V.sum() / prob.grid.dx ** 3, 53)) <= 1e-12 * cells


@pytest.mark.parametrize("name", ["plain_fp64_8k", "diff_window_100k"])
def test_alpha_s_is_independent_of_granule_order(name):
    """FP32 path: alpha_s and the conservation totals of one state are
    bitwise identical whatever the order of the granules (integer deposits
    and integer atomics: the order in which they arrive cannot matter).
    The same state in its own order and in two shuffled orders."""
    base = gi.make(name)
    out = []
    for seed in (None, 1, 2):
        prob = base if seed is None else shuffled(base, seed)
        sim = sim_for(prob, FP32)
        gic.gic_p2g(sim.grid, sim.params, sim.A, sim.A, None, sim.alpha_s, (None, None, None), sim.sums)
        torch.cuda.synchronize()
        out.append((sim.alpha_s.cpu().numpy(), sim.sums.cpu().numpy()))
    for a, sums in out[1:]:
        assert np.array_equal(a.view(np.uint64), out[0][0].view(np.uint64))
        assert np.array_equal(sums.view(np.uint64), out[0][1].view(np.uint64))
    _conserved(out[0][1], FP32)


# ----------------------------------------------------------------------------- windows

@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("prec", PRECS)
def test_window_10_substeps(name, prec):
    prob = _problem(name)
    K = 10
    sim = sim_for(prob, prec)
    sim.run(K)
    x, v = sim.positions()
    torch.cuda.synchronize()
    st = gic.gic_check_status()
    ref = oracle.run(prob, K=K)
    assert st == ref["status"] == 0
    dx = prob.grid.dx
    ex = np.abs(x.cpu().numpy() - ref["x"]).max()
    vref = np.linalg.norm(ref["v"], axis=1).max()
    ev = np.linalg.norm(v.cpu().numpy() - ref["v"], axis=1).max()
    ea = np.abs(sim.alpha_s.cpu().numpy() - ref["alpha_s"]).max()
    print(f"window {name} prec={prec}: |dx|={ex:.3e} ({ex / dx:.2e} dx) |dv|={ev:.3e} (vref {vref:.3e}) |dalpha|={ea:.3e}")
    # per granule too: |dv_i| <= 1e-4 max(|v_i|, 1e-2 v_ref) -- relative to the
    # granule's own speed, floored at 1% of the largest (the granules start
    # at rest, so a few still move far slower than the rest)
    vo = np.linalg.norm(ref["v"], axis=1)
    er = np.linalg.norm(v.cpu().numpy() - ref["v"], axis=1) / np.maximum(vo, 1e-2 * vref)
    print(f"  worst per-granule relative velocity error {er.max():.3e}")
    if prec == FP32:
        assert ex <= 1e-5 * dx, ex
        assert ev <= 1e-4 * vref, (ev, vref)
        assert er.max() <= 1e-4, er.max()
        assert ea <= 1e-9, ea
    else:
        assert ex <= 1e-12 * dx, ex
        assert ev <= 1e-10 * vref, (ev, vref)
        assert er.max() <= 1e-10, er.max()
        assert ea <= 1e-12, ea
    sums = sim.sums.cpu().numpy()
    _conserved(sums, prec)
    assert abs(sums[1] - ref["sums"][1]) <= 1e-12 * sums[1]
    for c in range(3):
        fo = ref["Fs"][c]
        fg = sim.Fs[c].cpu().numpy()
        assert np.abs(fg - fo).max() <= (1e-4 if prec == FP32 else 1e-10) * np.abs(fo).max()


# ----------------------------------------------------------------------------- edge cases

@pytest.mark.parametrize("prec", PRECS)
def test_empty_problem(prec):
    prob = subset(gi.make("dense_block"), 0)
    sim = Simulator(prob.grid, prob.params, 0, prec)
    sim.set_fluid(prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)
    sim.alpha_s.fill_(7.0)
    sim.sums.fill_(7.0)
    sim.run(3)
    torch.cuda.synchronize()
    assert float(sim.alpha_s.abs().max()) == 0.0
    assert sim.sums.cpu().tolist() == [0.0, 0.0]
    assert gic.gic_check_status() == 0


@pytest.mark.parametrize("prec", PRECS)
def test_single_granule_matches_oracle(prec):
    prob = subset(gi.make("random_cloud"), 1)
    sim = sim_for(prob, prec)
    sim.run(10)
    x, v = sim.positions()
    ref = oracle.run(prob, K=10)
    assert np.abs(x.cpu().numpy() - ref["x"]).max() <= 1e-5 * prob.grid.dx
    assert np.abs(v.cpu().numpy() - ref["v"]).max() <= 1e-4 * np.abs(ref["v"]).max()


@pytest.mark.parametrize("prec", PRECS)
def test_out_of_domain_is_flagged_not_faulted(prec):
    prob = subset(gi.make("dense_block"), 64)
    prob.v = prob.v.copy()
    prob.v[3] = [-1e4, 0, 0]  # crosses the x = 0 wall in one substep
    prob.params.c_drag = 0.0  # (quadratic drag at 1e4 m/s would reverse the granule within the substep)
    sim = sim_for(prob, prec)
    sim.run(1)
    torch.cuda.synchronize()
    st = gic.gic_check_status()
    assert st & gic.STATUS_OUT_OF_DOMAIN
    assert st & gic.STATUS_FAST
    ref = oracle.run(prob, K=1)
    assert ref["status"] & oracle.OUT_OF_DOMAIN
    x, v = sim.positions()
    x, v = x.cpu().numpy(), v.cpu().numpy()
    assert np.all(np.isfinite(x))
    # both sides put the granule back on the x = 0 plane it crossed (and keep
    # its velocity); every other granule moves as usual
    assert x[3, 0] == prob.grid.origin[0] == ref["x"][3, 0]
    assert np.abs(x - ref["x"]).max() <= 1e-5 * prob.grid.dx
    assert np.abs(v - ref["v"]).max() <= 1e-4 * np.abs(ref["v"]).max()
    others = np.arange(prob.n) != 3
    assert np.abs(v[others] - ref["v"][others]).max() <= 1e-4 * np.abs(ref["v"][others]).max()


@pytest.mark.parametrize("prec", PRECS)
def test_coincident_pair_is_skipped_and_flagged(prec):
    prob = subset(gi.make("random_cloud"), 50)
    prob.cell = prob.cell.copy()
    prob.q = prob.q.copy()
    prob.cell[1] = prob.cell[0]
    prob.q[1] = prob.q[0]
    sim = sim_for(prob, prec)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    gic.gic_contact(sim.grid, sim.params, sim.B, sim.table, sim.F_c)
    torch.cuda.synchronize()
    assert gic.gic_check_status() & gic.STATUS_COINCIDENT
    x, v, r = oracle_inputs(prob)
    Fo, st = oracle.contact(prob.grid, prob.params, x, v, r)
    assert st & oracle.COINCIDENT
    F = by_id(sim.F_c, sim.B.id)[:, :3]
    assert np.abs(F - Fo).max() <= tol_force(prob, prec) + 1e-5 * max(np.abs(Fo).max(), 1.0)


def test_nonfinite_velocity_is_flagged():
    prob = subset(gi.make("random_cloud"), 40)
    prob.v = prob.v.copy()
    prob.v[5] = [np.nan, 0, 0]
    sim = sim_for(prob, FP32)
    sim.run(1)
    torch.cuda.synchronize()
    assert gic.gic_check_status() & gic.STATUS_NONFINITE


def test_host_errors_with_device_buffers():
    prob = gi.make("dense_block")
    sim = sim_for(prob, FP32)
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(gic.GicError, match="workspace"):
        gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, small)
    with pytest.raises(gic.GicError, match="alias"):
        gic.gic_sort(sim.grid, sim.A, sim.A, sim.perm, sim.table, sim.ws)
    s = sim.A.struct()
    s.pos = s.pos + 4  # misaligned by 4 bytes
    rc = gic.lib().gic_contact(gic.C.byref(sim.grid), gic.C.byref(sim.params), gic.C.byref(s),
                               gic.C.c_void_p(sim.table.data_ptr()), gic.C.c_void_p(sim.F_c.data_ptr()), None)
    assert rc == -4


# ----------------------------------------------------------------------------- full size (sampled)

@pytest.mark.slow
def test_dam_break_full_size_one_substep():
    """1M granules, 128^3: one substep in the launch configuration the
    benchmark uses, every output compared with the oracle (sort bit-exact)."""
    prob = gi.make("dam_break_1m")
    sim = sim_for(prob, FP32)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    gic.gic_contact(sim.grid, sim.params, sim.B, sim.table, sim.F_c)
    F = sim.fluid
    gic.gic_g2p_couple(sim.grid, sim.params, sim.B, F.u, F.v, F.w, F.p, F.alpha_f, sim.F_fl, sim.a_f, sim.alpha_f_p)
    torch.cuda.synchronize()
    x, v, r = oracle_inputs(prob)
    perm_o, _ = oracle.sort(prob.cell)
    assert np.array_equal(sim.perm.cpu().numpy(), perm_o)
    Fo, st = oracle.contact(prob.grid, prob.params, x, v, r)
    Fg = by_id(sim.F_c, sim.B.id)[:, :3]
    assert np.abs(Fg - Fo).max() <= tol_force(prob, FP32) + 1e-5 * np.abs(Fo).max()
    Ffl_o, af_o, _ = oracle.g2p(prob.grid, prob.params, x, v, r, prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)
    Ffl = by_id(sim.F_fl, sim.B.id)[:, :3]
    assert np.abs(Ffl - Ffl_o).max() <= 2e-6 * np.abs(Ffl_o).max()
    # the rest of the substep, then alpha_s against the oracle at the GPU's new positions
    gic.gic_integrate(sim.grid, sim.params, sim.B, sim.F_c, sim.F_fl, sim.a_f, sim.A, sim.f_ex)
    sim.zero_transfer()
    gic.gic_p2g(sim.grid, sim.params, sim.B, sim.A, sim.f_ex, sim.alpha_s, sim.Fs, sim.sums)
    xb, _ = sim.positions(sim.B)
    xa, _ = sim.positions(sim.A)
    fex = by_id(sim.f_ex, sim.A.id)[:, :3].astype(np.float64)
    a_o, Fs_o, sums_o = oracle.p2g(prob.grid, prob.params, xb.cpu().numpy(), xa.cpu().numpy(), r, fex)
    assert np.abs(sim.alpha_s.cpu().numpy() - a_o).max() <= 1e-9
    for c in range(3):
        assert np.abs(sim.Fs[c].cpu().numpy() - Fs_o[c]).max() <= FS_TOL_FP32 * np.abs(Fs_o[c]).max()
    # volume conservation at full size: sum_i V_i / dx^3 is ~3e4 here, far beyond
    # what a 64-bit accumulator of 2^-53 units holds
    # (against the correctly rounded sum of the FP64 volumes: a running FP64
    # sum of 1M equal terms, as the oracle's, drifts by ~1e-11)
    sums = sim.sums.cpu().numpy()
    _conserved(sums, FP32)
    vol = math.fsum(4.0 / 3.0 * math.pi * float(ri) ** 3 for ri in prob.r.astype(np.float64))
    assert abs(sums[1] - vol) <= 1e-12 * vol
    assert abs(sums_o[1] - vol) <= 1e-10 * vol
    assert abs(sums[0] - math.fsum(sim.alpha_s.cpu().numpy().tolist()) * prob.grid.dx ** 3) <= 1e-12 * sums[0]
    assert gic.gic_check_status() == 0


@pytest.mark.slow
def test_dam_break_full_size_window():
    """1M granules, 10 substeps, against the oracle's 10 substeps."""
    prob = gi.make("dam_break_1m")
    K = 10
    sim = sim_for(prob, FP32)
    sim.run(K)
    x, v = sim.positions()
    ref = oracle.run(prob, K=K)
    dx = prob.grid.dx
    assert np.abs(x.cpu().numpy() - ref["x"]).max() <= 1e-5 * dx
    vref = np.linalg.norm(ref["v"], axis=1).max()
    assert np.linalg.norm(v.cpu().numpy() - ref["v"], axis=1).max() <= 1e-4 * vref
    assert np.abs(sim.alpha_s.cpu().numpy() - ref["alpha_s"]).max() <= 1e-9


def _sub_box(prob, x, n_target, halo):
    """A box over the full bed height, centred in x, y, holding about
    n_target granules: (granules within the box grown by `halo`, granules in
    the box itself, box low corner, box high corner)."""
    lo_all, hi_all = x.min(0), x.max(0)
    area = (hi_all[0] - lo_all[0]) * (hi_all[1] - lo_all[1])
    w = np.sqrt(area * n_target / prob.n)
    c = 0.5 * (lo_all[:2] + hi_all[:2])
    lo = np.array([c[0] - w / 2, c[1] - w / 2, -1.0])
    hi = np.array([c[0] + w / 2, c[1] + w / 2, 2.0])
    inside = lambda pad: np.all((x >= lo - pad) & (x < hi + pad), axis=1)
    return np.nonzero(inside(halo))[0], np.nonzero(inside(0.0))[0], lo, hi


@pytest.mark.slow
@pytest.mark.parametrize("name", ["polydisperse_bed_8m", "scale_sweep_16m"])
@pytest.mark.parametrize("prec", PRECS)
def test_full_size_sampled_one_substep(name, prec):
    """8M granules on 256^3 (lognormal radii) and 16M on 384^3: one substep
    in the benchmark's launch configuration.  The permutation is compared in
    full (bit-exact) and the cell table on every occupied cell; contact, G2P,
    alpha_s and F_s on a 100k-granule box, against the oracle run on the box
    grown by a halo: a granule's force depends only on granules within
    2 r_max, and a cell's alpha_s and F_s only on granules within
    r_max + 2 dx of it, so the box's interior is exact."""
    prob = gi.make(name)
    sim = sim_for(prob, prec)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    gic.gic_contact(sim.grid, sim.params, sim.B, sim.table, sim.F_c)
    F = sim.fluid
    gic.gic_g2p_couple(sim.grid, sim.params, sim.B, F.u, F.v, F.w, F.p, F.alpha_f, sim.F_fl, sim.a_f, sim.alpha_f_p)
    torch.cuda.synchronize()
    assert gic.gic_check_status() == 0
    perm_o, keys_o = oracle.sort(prob.cell)
    assert np.array_equal(sim.perm.cpu().numpy(), perm_o)
    ck, st, ct = oracle.cell_table(keys_o)
    tab = sim.table.view(-1, 4)
    epoch = int(tab[0, 0].item())
    nc = prob.grid.nc
    cs = prob.cell[perm_o[st]].astype(np.int64)
    lin = torch.from_numpy(1 + cs[:, 0] + nc[0] * (cs[:, 1] + nc[1] * cs[:, 2])).cuda()
    rows = tab[lin].cpu().numpy().astype(np.int64)
    assert np.array_equal(rows[:, 0], st) and np.array_equal(rows[:, 1], ct) and np.all(rows[:, 2] == epoch)
    assert int((tab[1:, 2] == epoch).sum().item()) == len(ck)

    x, v, r = oracle_inputs(prob)
    r_max = float(r.max())
    dx = prob.grid.dx
    halo = 2 * r_max + 2 * dx
    box, core, lo, hi = _sub_box(prob, x, 100_000, halo)
    assert len(core) > 50_000
    Fo, _ = oracle.contact(prob.grid, prob.params, x[box], v[box], r[box])
    in_core = np.isin(box, core)
    Fg = by_id(sim.F_c, sim.B.id)[:, :3][box]
    err = np.abs(Fg - Fo)[in_core].max()
    scale = np.abs(Fo[in_core]).max()
    assert err <= (tol_force(prob, FP32) + 1e-5 * scale if prec == FP32 else 1e-9 * scale)  # 0 when no contacts
    Ffl_o, af_o, afp_o = oracle.g2p(prob.grid, prob.params, x[box], v[box], r[box], prob.u, prob.vf, prob.wf, prob.p,
                                    prob.alpha_f)
    rel = 2e-6 if prec == FP32 else 1e-12
    Ffl = by_id(sim.F_fl, sim.B.id)[:, :3][box]
    assert np.abs(Ffl - Ffl_o).max() <= rel * np.abs(Ffl_o).max()
    af = by_id(sim.a_f, sim.B.id)[:, :3][box]
    assert np.abs(af - af_o).max() <= rel * 9.8

    gic.gic_integrate(sim.grid, sim.params, sim.B, sim.F_c, sim.F_fl, sim.a_f, sim.A, sim.f_ex)
    sim.zero_transfer()
    gic.gic_p2g(sim.grid, sim.params, sim.B, sim.A, sim.f_ex, sim.alpha_s, sim.Fs, sim.sums)
    torch.cuda.synchronize()
    xb, _ = sim.positions(sim.B)
    xa, _ = sim.positions(sim.A)
    xb = xb.cpu().numpy()[box]
    xa = xa.cpu().numpy()[box]
    fex = by_id(sim.f_ex, sim.A.id)[:, :3].astype(np.float64)[box]
    a_o, Fs_o, _ = oracle.p2g(prob.grid, prob.params, xb, xa, r[box], fex)
    g = prob.grid
    pad = r_max + 3 * dx

    org = np.asarray(g.origin, dtype=np.float64)

    def interior(sx, sy, sz, off):
        # grids are stored x fastest: index = i + sx (j + sy k)
        cx = org[0] + (np.arange(sx) + off[0]) * dx
        cy = org[1] + (np.arange(sy) + off[1]) * dx
        mx = (cx >= lo[0] + pad) & (cx < hi[0] - pad)
        my = (cy >= lo[1] + pad) & (cy < hi[1] - pad)
        return np.broadcast_to(my[None, :, None] & mx[None, None, :], (sz, sy, sx)).ravel()

    cells = interior(g.nx, g.ny, g.nz, np.full(3, 0.5))
    a_g = sim.alpha_s.cpu().numpy()
    assert np.count_nonzero(a_o[cells]) > 1000
    assert np.abs(a_g[cells] - a_o[cells]).max() <= 1e-9
    dims = ((g.nx + 1, g.ny, g.nz), (g.nx, g.ny + 1, g.nz), (g.nx, g.ny, g.nz + 1))
    for c in range(3):
        off = np.full(3, 0.5)
        off[c] = 0.0
        faces = interior(*dims[c], off)
        got = sim.Fs[c].cpu().numpy()[faces]
        want = Fs_o[c][faces]
        assert np.abs(got - want).max() <= (FS_TOL_FP32 if prec == FP32 else 1e-12) * np.abs(want).max()
    assert gic.gic_check_status() == 0


@pytest.mark.slow
@pytest.mark.parametrize("name,K", [("scale_sweep_16m", 20), ("polydisperse_bed_8m", 10)])
@pytest.mark.parametrize("prec", PRECS)
def test_full_size_subregion_window(name, K, prec):
    """16M granules on 384^3 (its full 20 substeps) and the 8M-granule bed on
    256^3 (10 substeps) on the GPU, against the oracle's substeps on a
    100k-granule box grown by a halo of K (2 r_max + v_max dt) + 2 dx:
    contacts carry information at most 2 r_max per substep and a granule
    moves at most v_max dt, so the granules that start in the box, and the
    alpha_s cells whose stencils stay inside it, see exactly the oracle's
    inputs."""
    prob = gi.make(name)
    sim = sim_for(prob, prec)
    sim.run(K)
    torch.cuda.synchronize()
    assert gic.gic_check_status() == 0
    xg, vg = sim.positions()
    x, v, r = oracle_inputs(prob)
    r_max = float(r.max())
    dx = prob.grid.dx
    v_max = 2.0 * max(np.abs(a).max() for a in (prob.u, prob.vf, prob.wf)) + 1.0
    halo = K * (2 * r_max + v_max * prob.params.dt_sub) + 2 * dx
    box, core, lo, hi = _sub_box(prob, x, 100_000, halo)
    sub = dataclasses.replace(prob, cell=prob.cell[box].copy(), q=prob.q[box].copy(), r=prob.r[box].copy(),
                              v=prob.v[box].copy())
    ref, taint = onset_taint(sub, K)
    # granules whose trajectory hangs on a contact within rounding of onset
    # are compared only for plausibility (the settled bed has hundreds of
    # pairs crossing touch per substep, and taint spreads through its contact
    # network: about a third of it is tainted after ten substeps)
    in_core = np.isin(box, core)
    assert taint[in_core].mean() < 0.5
    keep = in_core & ~taint
    xg = xg.cpu().numpy()[box]
    vg = vg.cpu().numpy()[box]
    assert np.abs(xg[keep] - ref["x"][keep]).max() <= (1e-5 if prec == FP32 else 1e-12) * dx
    vref = np.linalg.norm(ref["v"], axis=1).max()
    # FP64: both sides form the overlap r_i + r_j - d from coordinates of
    # ~0.5 m (ulp 1e-16 m) against overlaps of ~1e-6 m, so a stiff contact
    # network moves velocities by ~K dt k_n 1e-16 / m_min ~ 1e-11 m/s
    assert np.linalg.norm(vg[keep] - ref["v"][keep], axis=1).max() <= (1e-4 if prec == FP32 else 1e-9) * vref
    assert np.abs(xg[in_core] - ref["x"][in_core]).max() <= 1e-3 * dx
    g = prob.grid
    pad = r_max + 3 * dx + K * v_max * prob.params.dt_sub
    cx = g.origin[0] + (np.arange(g.nx) + 0.5) * dx
    cy = g.origin[1] + (np.arange(g.ny) + 0.5) * dx
    mx = (cx >= lo[0] + pad) & (cx < hi[0] - pad)
    my = (cy >= lo[1] + pad) & (cy < hi[1] - pad)
    cells = np.broadcast_to(my[None, :, None] & mx[None, None, :], (g.nz, g.ny, g.nx)).ravel().copy()
    # and not the cells within a stencil of a tainted granule's final position
    org = np.asarray(g.origin, dtype=np.float64)
    base = np.floor((ref["x"][taint] - org) / dx - 0.5).astype(np.int64)
    for k in range(8):
        c = base + np.array([k & 1, (k >> 1) & 1, k >> 2])
        ok = np.all((c >= 0) & (c < np.array([g.nx, g.ny, g.nz])), axis=1)
        cells[c[ok, 0] + g.nx * (c[ok, 1] + g.ny * c[ok, 2])] = False
    a_o = ref["alpha_s"][cells]
    assert np.count_nonzero(a_o) > 200
    a_g = sim.alpha_s.cpu().numpy()
    # the FP64 accumulation itself: the oracle's alpha_s at the GPU's own final positions
    rb = r[box]
    a_same = oracle.p2g(g, prob.params, xg, xg, rb, np.zeros_like(xg))[0]
    assert np.abs(a_g[cells] - a_same[cells]).max() <= 1e-9
    # against the oracle's trajectory: 1e-9 plus what the (within-tolerance)
    # position differences move it, |d alpha| <= V / dx^3 sum_a |dx_a| / dx
    # over the granules whose stencils reach the cell
    vol = 4.0 / 3.0 * np.pi * rb ** 3 / dx ** 3
    e = vol * np.abs(xg - ref["x"]).sum(axis=1) / dx
    bound = np.zeros(g.nx * g.ny * g.nz)
    for xs in (xg, ref["x"]):
        base = np.floor((xs - org) / dx - 0.5).astype(np.int64)
        for k in range(8):
            c = base + np.array([k & 1, (k >> 1) & 1, k >> 2])
            ok = np.all((c >= 0) & (c < np.array([g.nx, g.ny, g.nz])), axis=1)
            np.add.at(bound, c[ok, 0] + g.nx * (c[ok, 1] + g.ny * c[ok, 2]), e[ok])
    assert np.all(np.abs(a_g[cells] - a_o) <= 1e-9 + bound[cells])


# ----------------------------------------------------------------------------- public host-buffer window, failures

@pytest.mark.parametrize("prec", PRECS)
def test_host_window_matches_oracle(prec):
    """gic_window_forward_host (host buffers in, host buffers out, copies
    inside) against the oracle's 10-substep window."""
    prob = shuffled(gi.make("dense_block"))
    g = gic.make_grid(prob.grid)
    P = gic.make_params(prob.params)
    real = np.float32 if prec == FP32 else np.float64
    host = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a if dt is None else a.astype(dt))).pin_memory()
    nx, ny, nz = prob.grid.nx, prob.grid.ny, prob.grid.nz
    x = torch.empty((prob.n, 3), dtype=torch.float64).pin_memory()
    v = torch.empty((prob.n, 3), dtype=torch.float64).pin_memory()
    a = torch.empty(nx * ny * nz, dtype=torch.float64).pin_memory()
    tr = torch.float32 if prec == FP32 else torch.float64
    Fs = [torch.empty(m, dtype=tr).pin_memory() for m in ((nx + 1) * ny * nz, nx * (ny + 1) * nz, nx * ny * (nz + 1))]
    sums = torch.empty(2, dtype=torch.float64).pin_memory()
    ws = torch.empty(gic.gic_window_host_workspace_size(g, prob.n, prec), dtype=torch.uint8, device="cuda")
    gic.gic_window_forward_host(g, P, prec, host(prob.cell), host(prob.q.astype(np.int64), np.int32), host(prob.r),
                                host(prob.v), *[host(f, real) for f in (prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)],
                                prob.K, x, v, a, Fs, sums, ws)
    ref = oracle.run(prob)
    dx = prob.grid.dx
    assert np.abs(x.numpy() - ref["x"]).max() <= (1e-5 if prec == FP32 else 1e-12) * dx
    vref = np.linalg.norm(ref["v"], axis=1).max()
    assert np.linalg.norm(v.numpy() - ref["v"], axis=1).max() <= (1e-4 if prec == FP32 else 1e-10) * vref
    assert np.abs(a.numpy() - ref["alpha_s"]).max() <= 1e-9
    for c in range(3):
        assert np.abs(Fs[c].numpy() - ref["Fs"][c]).max() <= 1e-4 * np.abs(ref["Fs"][c]).max()
    _conserved(sums.numpy(), prec)


def test_status_wait_has_a_deadline():
    """The status query waits for the stream against a deadline: with work
    still running it returns GIC_ERR_TIMEOUT instead of blocking, and the
    context stays usable afterwards (no GPU fault is involved)."""
    prob = gi.make("dam_break_1m")
    sim = sim_for(prob, FP32)
    torch.cuda.synchronize()
    for _ in range(30):  # ~15 ms of GPU work, enqueued in ~3 ms
        sim.substep()
    with pytest.raises(gic.GicError, match="still busy"):
        gic.gic_check_status(clear=False, timeout_ms=1)
    torch.cuda.synchronize()
    assert gic.gic_check_status(timeout_ms=5000) == 0
