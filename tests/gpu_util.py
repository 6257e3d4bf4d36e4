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
