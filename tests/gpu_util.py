"""Helpers of the GPU parity tests: move inputs to the device, read results
back in original granule order, shuffle problems so the sort has work."""
import dataclasses

import numpy as np
import torch

import gic_inputs as gi
import oracle
from paper_2504_00745_gb300 import gic
from paper_2504_00745_gb300.window import Simulator

FP32, FP64 = gic.GIC_FP32, gic.GIC_FP64


def shuffled(prob, seed=123):
    """Same problem with the granules in a random order."""
    rng = np.random.default_rng(seed)
    p = rng.permutation(prob.n)
    out = dataclasses.replace(prob, cell=prob.cell[p].copy(), q=prob.q[p].copy(), r=prob.r[p].copy(),
                              v=prob.v[p].copy())
    if prob.target is not None:
        out.target = prob.target[p].copy()
    return out


def subset(prob, n):
    return dataclasses.replace(prob, cell=prob.cell[:n].copy(), q=prob.q[:n].copy(), r=prob.r[:n].copy(),
                               v=prob.v[:n].copy())


def sim_for(prob, precision):
    return Simulator.from_problem(prob, precision)


def by_id(t: torch.Tensor, ids: torch.Tensor):
    """Rows of t (state order) scattered to original-id order, as numpy."""
    a = t.detach().cpu().numpy()
    out = np.empty_like(a)
    out[ids.cpu().numpy()] = a
    return out


def state_positions(sim, st):
    """FP64 absolute positions and velocities of a state, original order."""
    return sim.positions(st)


def tol_force(prob, precision):
    """Absolute force tolerance of the FP32 contact path: the relative vector
    x_ij has an error of a few FP32 ulps of |x_ij| <= 2 r_max, which the
    spring turns into k_n times that; FP64 is held to 1e-9 of the force scale."""
    if precision == FP64:
        return 0.0
    r_max = float(prob.r.max())
    return prob.params.k_n * 16 * 2.0 ** -24 * 2 * r_max


def oracle_inputs(prob):
    x = oracle.decode(prob.grid, prob.cell, prob.q)
    return x, prob.v.astype(np.float64), prob.r.astype(np.float64)


def onset_taint(prob, K, eps=2e-10):
    """The oracle's K substeps, one at a time, with the granules whose
    trajectory depends on a contact that starts or ends within `eps` of
    touching.  The normal dashpot makes the force jump by c_n v_n at contact
    onset, so where a pair (or a granule and a wall) that moves along its
    normal is within rounding of touching, FP32 and FP64 may disagree on
    whether it is in contact at all (eps: a few times the FP32 path's
    position error after ten substeps); such a granule is tainted, and taint
    spreads to contact partners one contact per substep.
    Returns (oracle result after K substeps, taint)."""
    g = prob.grid
    r = prob.r.astype(np.float64)
    x = oracle.decode(g, prob.cell, prob.q)
    v = prob.v.astype(np.float64)
    n = prob.n
    lo = np.asarray(g.origin, dtype=np.float64)
    hi = lo + np.array([g.nx, g.ny, g.nz], dtype=np.float64) * g.dx
    taint = np.zeros(n, dtype=bool)
    out = None
    for _ in range(K):
        near = oracle.contact_pairs(g, x, r + 0.5 * eps)
        I, J = near[:, 0], near[:, 1]
        sep = x[I] - x[J]
        d = np.linalg.norm(sep, axis=1)
        gap = d - r[I] - r[J]
        vn = np.abs(np.sum((v[I] - v[J]) * sep, axis=1)) / np.maximum(d, 1e-300)
        amb = (np.abs(gap) < eps) & (vn > 0)
        taint[I[amb]] = True
        taint[J[amb]] = True
        if prob.params.walls:
            wgap = np.minimum(x - lo, hi - x) - r[:, None]
            taint |= np.any((np.abs(wgap) < eps) & (v != 0), axis=1)
        con = gap < 0
        spread = con & (taint[I] | taint[J])
        taint[I[spread]] = True
        taint[J[spread]] = True
        out = oracle.run(prob, K=1, x=x, v=v)
        x, v = out["x"], out["v"]
    return out, taint


# The FP32 path's F_s: each deposit is rounded to 2^-22 (2^-21 in the
# 512-thread P2G kernel) of the largest |exch f_ex| in its CTA, which may be
# several times the largest F_s entry where granules are sparse; bound
# relative to max |F_s|.
FS_TOL_FP32 = 1e-5


def assert_elementwise(got, want, tol, floor, what=""):
    """Element by element: |got_i - want_i| <= tol * max(|want_i|, floor).

    `floor` is an absolute scale below which an element is compared to the
    floor rather than to itself (each test states where its floor comes
    from).  Reports the worst element on failure."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape, f"{what}: shape {got.shape} != {want.shape}"
    err = np.abs(got - want)
    bound = tol * np.maximum(np.abs(want), floor)
    ratio = err / bound
    k = int(np.argmax(ratio)) if ratio.size else 0
    assert ratio.size == 0 or ratio.flat[k] <= 1.0, (
        f"{what}: element {np.unravel_index(k, got.shape)} got {got.flat[k]:.9e} want {want.flat[k]:.9e} "
        f"(|err| {err.flat[k]:.3e} > bound {bound.flat[k]:.3e}; floor {floor:.3e})")
    return float(ratio.max()) if ratio.size else 0.0
