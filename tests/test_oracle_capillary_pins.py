"""Pins of the oracle's concentration-gradient (capillary) pair force,
Sec. 5.4: F_ij = -Gamma((sr_i + sr_j) / 2) F^st(s_ij) (x_i - x_j) / |x_i - x_j|
for 0 < s_ij < d_r, with the readings of the design notes (pair radius
2 r_i r_j / (r_i + r_j), V* = bridge_frac times the mean granule volume,
the rupture distance in units of the pair radius, Gamma the quadratic
Bezier curve through (0, 0), (2 peak - 1/2, 2), (1, 0)).

Each pin checks the oracle against something other than its own formula:
the bridge energy printed in the paper (F^st must be its derivative), the
limits the paper states (F^st -> 2 pi sigma R as s -> 0, -> 0 as V* -> 0;
Gamma = 0 when dry and when saturated, largest at the absorption ratio),
the Bezier curve in its parametric form, the raw rupture formula at the
paper's sizes, Newton's third law and the momentum of a free pair.
"""
import dataclasses
import math

import numpy as np
import pytest

import gic_inputs as gi
import oracle

SIGMA = 0.07


def _energy(s, R, Vs, sigma=SIGMA):
    """The liquid-bridge energy of Sec. 5.4 with cos(theta) = 1."""
    return -2.0 * math.pi * sigma * R * (-s + math.sqrt(s * s + 2.0 * Vs / (math.pi * R)))


def _vstar(r, frac=1e-4):
    return frac * 4.0 / 3.0 * math.pi * r ** 3


@pytest.mark.parametrize("r", [3.9e-4, 4e-3])
def test_bridge_force_is_the_derivative_of_the_bridge_energy(r):
    Vs = _vstar(r)
    dr = oracle.rupture(r, Vs)
    for s in np.linspace(0.02, 0.98, 9) * dr:
        h = 1e-6 * s
        dEds = (_energy(s + h, r, Vs) - _energy(s - h, r, Vs)) / (2 * h)
        assert abs(oracle.bridge_force(SIGMA, r, Vs, s) - dEds) <= 1e-7 * abs(dEds)
    # and it falls monotonically with the separation
    vals = [oracle.bridge_force(SIGMA, r, Vs, s) for s in np.linspace(0.01, 1.0, 50) * dr]
    assert all(a > b for a, b in zip(vals, vals[1:]))


def test_bridge_force_limits():
    """s -> 0: 2 pi sigma R (the bridge of a touching pair); V* -> 0: 0."""
    r = 4e-3
    top = 2.0 * math.pi * SIGMA * r
    assert abs(oracle.bridge_force(SIGMA, r, _vstar(r), 1e-12 * r) - top) <= 1e-6 * top
    assert oracle.bridge_force(SIGMA, r, 1e-40, 0.01 * r) <= 1e-12 * top


def test_rupture_distance_reading():
    """The reading (the cited formula in units of the pair radius) against
    the formula as printed, V*^(1/3) + 0.1 V*^(2/3) in metres, at the paper's
    granule radius 3.9e-4 m and V* = 0.01% of the granule volume: within
    1% (the second term, 0.1 V*^(2/3), is 0.75% of the first in units of the
    radius and nothing in metres); and the dimensionless value at that
    V*/R^3."""
    r = 3.9e-4
    Vs = _vstar(r)
    printed = Vs ** (1 / 3) + 0.1 * Vs ** (2 / 3)
    assert abs(oracle.rupture(r, Vs) - printed) <= 1e-2 * printed
    v = 1e-4 * 4.0 / 3.0 * math.pi
    assert abs(oracle.rupture(1.0, v) - (v ** (1 / 3) + 0.1 * v ** (2 / 3))) < 1e-15


@pytest.mark.parametrize("peak", [0.3, 0.5, 0.7])
def test_gamma_is_the_bezier_curve(peak):
    """Gamma traced along the curve's own parametrisation: the point
    B(t) = (1-t)^2 P0 + 2 t (1-t) P1 + t^2 P2 with P0 = (0, 0), P1 = (2 peak -
    1/2, 2), P2 = (1, 0) lies on the graph of Gamma for every t."""
    P0, P1, P2 = np.array([0.0, 0.0]), np.array([2 * peak - 0.5, 2.0]), np.array([1.0, 0.0])
    for t in np.linspace(0.0, 1.0, 41):
        B = (1 - t) ** 2 * P0 + 2 * t * (1 - t) * P1 + t ** 2 * P2
        assert abs(oracle.gamma(B[0], peak) - B[1]) <= 1e-12
    assert oracle.gamma(0.0, peak) == 0.0 and oracle.gamma(1.0, peak) == 0.0
    assert oracle.gamma(1.5, peak) == 0.0 and oracle.gamma(-0.1, peak) == 0.0
    assert abs(oracle.gamma(peak, peak) - 1.0) <= 1e-12
    grid = np.linspace(0.0, 1.0, 2001)
    vals = np.array([oracle.gamma(x, peak) for x in grid])
    assert vals.min() >= 0.0 and vals.max() <= 1.0 + 1e-12
    assert abs(grid[vals.argmax()] - peak) <= 1e-3


def test_moisture_ratio():
    """sr = r + alpha / (1 - alpha): dry sand (alpha = 0, r = 0) gives 0,
    alpha = 1/2 gives r + 1, no sand (alpha = 1) infinity."""
    assert oracle.moisture_ratio(0.0, 0.0) == 0.0
    assert oracle.moisture_ratio(0.2, 0.5) == 1.2
    assert math.isinf(oracle.moisture_ratio(0.0, 1.0))


def _pair(s_over_r, alpha, peak=0.3, moisture=0.0, r0=float(np.float32(4e-3)), sigma=SIGMA,
          v=((0, 0, 0), (0, 0, 0)), axis=0):
    grid = gi.Grid(16, 16, 16, 1.0 / 16, k_contact=1)
    P = gi.Params(rho_f=0.0, c_drag=0.0, g=(0.0, 0.0, 0.0), walls=0, sigma=sigma, moisture=moisture,
                  moisture_peak=peak)
    c = np.array([0.5, 0.5, 0.5])
    e = np.zeros(3)
    e[axis] = 1.0
    half = (2 * r0 + s_over_r * r0) / 2
    x = np.array([c - half * e, c + half * e])
    af = np.full(16 ** 3, alpha)
    return grid, P, x, np.array(v, float), np.array([r0, r0]), af


def test_capillary_pair_force_attracts_along_the_line_of_centres():
    """Two equal granules 3% of r apart with the fluid fraction chosen so
    that sr = peak (Gamma = 1): each is pulled towards the other by exactly
    dE/ds of the bridge energy; Newton's third law holds."""
    peak = 0.3
    alpha = peak / (1.0 + peak)  # alpha / (1 - alpha) = peak
    for axis in range(3):
        grid, P, x, v, r, af = _pair(0.03, alpha, peak, axis=axis)
        F, st = oracle.contact(grid, P, x, v, r, alpha_f=af)
        s = 0.03 * r[0]
        Vs = _vstar(r[0])
        h = 1e-6 * s
        want = (_energy(s + h, r[0], Vs) - _energy(s - h, r[0], Vs)) / (2 * h)
        assert st == 0
        assert abs(F[0, axis] - want) <= 1e-7 * want  # granule 0 sits below: pulled up the axis
        assert np.abs(np.delete(F[0], axis)).max() == 0.0
        assert np.abs(F[0] + F[1]).max() <= 1e-15


@pytest.mark.parametrize("alpha,moisture,what", [(0.0, 0.0, "dry"), (1.0, 0.0, "no sand"), (0.6, 0.0, "saturated")])
def test_no_capillary_force_when_dry_or_saturated(alpha, moisture, what):
    grid, P, x, v, r, af = _pair(0.03, alpha, moisture=moisture)
    F, _ = oracle.contact(grid, P, x, v, r, alpha_f=af)  # alpha 0.6: sr = 1.5 >= 1
    assert np.abs(F).max() == 0.0, what


def test_force_ends_at_the_rupture_distance_and_at_contact():
    alpha = 0.3 / 1.3
    r0 = float(np.float32(4e-3))
    dr = oracle.rupture(r0, _vstar(r0))
    for frac, on in ((0.999, True), (1.001, False)):
        grid, P, x, v, r, af = _pair(frac * dr / r0, alpha)
        F, _ = oracle.contact(grid, P, x, v, r, alpha_f=af)
        assert (np.abs(F).max() > 0.0) == on
    # overlapping by 0.1% of r: the contact law alone, no bridge
    grid, P, x, v, r, af = _pair(-1e-3, alpha)
    F, _ = oracle.contact(grid, P, x, v, r, alpha_f=af)
    F0, _ = oracle.contact(grid, dataclasses.replace(P, sigma=0.0), x, v, r)
    assert np.array_equal(F, F0) and F[0, 0] < 0.0  # pushed apart


def test_free_pair_keeps_its_momentum_and_closes_the_gap():
    """Two equal granules in the bridge range, no gravity, no fluid force:
    the pair's momentum stays zero and after one substep each velocity is
    dt' F / m exactly (symplectic Euler, no added mass)."""
    alpha = 0.3 / 1.3
    grid, P, x, v, r, af = _pair(0.03, alpha)
    prob = gi.Problem("pair", grid, P, 1, *gi.encode_positions(x, grid), r.astype(np.float32),
                      v.astype(np.float32), np.zeros(17 * 16 * 16), np.zeros(17 * 16 * 16), np.zeros(17 * 16 * 16),
                      np.zeros(16 ** 3), af)
    F, _ = oracle.contact(grid, P, x, v, r, alpha_f=af)
    out = oracle.run(prob, K=1, x=x, v=v)
    m = P.rho_s * 4.0 / 3.0 * math.pi * r[0] ** 3
    assert np.abs(out["v"][0] - P.dt_sub * F[0] / m).max() <= 1e-15
    assert np.abs(out["v"][0] + out["v"][1]).max() <= 1e-18
    assert out["v"][0, 0] > 0.0 and out["v"][1, 0] < 0.0


def test_capillary_forces_binned_equal_brute_force_and_cancel():
    prob = gi.make("wet_block")
    x, r = prob.positions(), prob.r.astype(np.float64)
    P = dataclasses.replace(prob.params, walls=0)
    Fb, _ = oracle.contact(prob.grid, P, x, prob.v, r, brute=True, alpha_f=prob.alpha_f)
    Fc, _ = oracle.contact(prob.grid, P, x, prob.v, r, brute=False, alpha_f=prob.alpha_f)
    F0, _ = oracle.contact(prob.grid, dataclasses.replace(P, sigma=0.0), x, prob.v, r)
    scale = np.abs(Fb).max()
    assert np.abs(Fb - Fc).max() <= 1e-12 * scale
    assert np.abs(Fb.sum(axis=0)).max() <= 1e-11 * scale
    assert np.abs(Fb - F0).max() > 1e-4  # the bridges are there (~1.8e-3 N each)
