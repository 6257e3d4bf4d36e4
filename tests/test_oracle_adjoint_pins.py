"""Pins of the oracle's hand-derived adjoint.

Each adjoint is checked against central finite differences of the oracle's
own FORWARD functions (an independent route: the Jacobians are written out
explicitly, the forward is plain arithmetic), per function and over whole
windows.  Window checks are only asserted on contact-stable windows: the
contact set and the stick/slip flags must be the same in the +h and -h runs
(non-smooth points otherwise), detected from the oracle's contact signature.
"""
import dataclasses

import numpy as np
import pytest

import gic_inputs as gi
import oracle


def _fd_rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


def _small_cloud(seed=21):
    return gi.make("random_cloud", seed=seed)


@pytest.mark.parametrize("name,walls", [("dense_block", 1), ("dense_block", 0), ("random_cloud", 1)])
def test_contact_vjp_matches_fd(name, walls):
    prob = gi.make(name)
    P = dataclasses.replace(prob.params, walls=walls)
    x, v, r = prob.positions(), prob.v.astype(float), prob.r.astype(float)
    rng = np.random.default_rng(1)
    lam = rng.normal(size=x.shape)
    dX = rng.normal(size=x.shape)
    dV = rng.normal(size=x.shape)
    gx, gv, gmu = oracle.contact_adj(prob.grid, P, x, v, r, lam)
    hx = 1e-9  # metres: well inside every overlap (>= 1e-5 r), so no pair switches
    f = lambda xx, vv, PP=P: np.sum(lam * oracle.contact(prob.grid, PP, xx, vv, r)[0])
    fd_x = (f(x + hx * dX, v) - f(x - hx * dX, v)) / (2 * hx)
    assert _fd_rel(np.sum(gx * dX), fd_x) < 1e-5
    hv = 1e-7
    fd_v = (f(x, v + hv * dV) - f(x, v - hv * dV)) / (2 * hv)
    assert _fd_rel(np.sum(gv * dV), fd_v) < 1e-5
    hm = 1e-6
    fd_m = (f(x, v, dataclasses.replace(P, mu_fric=P.mu_fric + hm))
            - f(x, v, dataclasses.replace(P, mu_fric=P.mu_fric - hm))) / (2 * hm)
    assert _fd_rel(gmu, fd_m) < 1e-5


def test_g2p_vjp_matches_fd():
    prob = gi.make("random_cloud")
    x, v, r = prob.positions(), prob.v.astype(float), prob.r.astype(float)
    fl = (prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)
    rng = np.random.default_rng(2)
    lF, la, lal = rng.normal(size=x.shape), rng.normal(size=x.shape), rng.normal(size=len(r))
    dX, dV = rng.normal(size=x.shape), rng.normal(size=x.shape)
    gx, gv, gc = oracle.g2p_adj(prob.grid, prob.params, x, v, r, *fl, lF, la, lal)

    def f(xx, vv, P=prob.params):
        F, a, al = oracle.g2p(prob.grid, P, xx, vv, r, *fl)
        return np.sum(lF * F) + np.sum(la * a) + np.sum(lal * al)

    h = 1e-8
    assert _fd_rel(np.sum(gx * dX), (f(x + h * dX, v) - f(x - h * dX, v)) / (2 * h)) < 1e-5
    assert _fd_rel(np.sum(gv * dV), (f(x, v + h * dV) - f(x, v - h * dV)) / (2 * h)) < 1e-6
    P = prob.params
    hc = 1e-6
    fd_c = (f(x, v, dataclasses.replace(P, c_drag=P.c_drag + hc)) - f(x, v, dataclasses.replace(P, c_drag=P.c_drag - hc))) / (2 * hc)
    assert _fd_rel(gc, fd_c) < 1e-6  # F_fl is linear in c_drag: FD error is rounding only


def test_integrate_vjp_matches_fd():
    prob = gi.make("random_cloud")
    x, v, r = prob.positions(), prob.v.astype(float), prob.r.astype(float)
    rng = np.random.default_rng(3)
    Fc, Ffl, af = (rng.normal(size=x.shape) * 1e-3 for _ in range(3))
    gX, gV, gF = (rng.normal(size=x.shape) for _ in range(3))
    gx, gv, gFc, gFfl, gaf = oracle.integrate_adj(prob.grid, prob.params, r, gX, gV, gF)

    def f(xx, vv, a, b, c):
        xn, vn, fe, _ = oracle.integrate(prob.grid, prob.params, xx, vv, r, a, b, c)
        return np.sum(gX * xn) + np.sum(gV * vn) + np.sum(gF * fe)

    base = (x, v, Fc, Ffl, af)
    grads = (gx, gv, gFc, gFfl, gaf)
    for k in range(5):
        d = rng.normal(size=x.shape)
        # the map is linear: large steps only reduce cancellation -- except that
        # positions must stay inside the box, where granules are put back
        # on the boundary (reading R12)
        h = 1e-3 * prob.grid.dx if k == 0 else 0.1 * np.abs(base[k]).max()
        plus = list(base)
        minus = list(base)
        plus[k] = base[k] + h * d
        minus[k] = base[k] - h * d
        fd = (f(*plus) - f(*minus)) / (2 * h)
        assert _fd_rel(np.sum(grads[k] * d), fd) < 1e-6, k


def test_p2g_vjp_matches_fd():
    prob = gi.make("random_cloud")
    x, r = prob.positions(), prob.r.astype(float)
    rng = np.random.default_rng(4)
    xn = x + rng.normal(size=x.shape) * 1e-4
    fex = rng.normal(size=x.shape)
    g = prob.grid
    ga = rng.normal(size=g.nx * g.ny * g.nz)
    gFs = (rng.normal(size=(g.nx + 1) * g.ny * g.nz), rng.normal(size=g.nx * (g.ny + 1) * g.nz),
           rng.normal(size=g.nx * g.ny * (g.nz + 1)))
    gxo, gxn, gfe = oracle.p2g_adj(g, prob.params, x, xn, r, fex, ga, gFs)

    def f(a, b, c):
        al, Fs, _ = oracle.p2g(g, prob.params, a, b, r, c)
        return np.dot(ga, al) + sum(np.dot(gFs[k], Fs[k]) for k in range(3))

    h = 1e-9
    for k, (base, grad) in enumerate(((x, gxo), (xn, gxn), (fex, gfe))):
        d = rng.normal(size=x.shape)
        args_p = [x, xn, fex]
        args_m = [x, xn, fex]
        args_p[k] = base + h * d
        args_m[k] = base - h * d
        fd = (f(*args_p) - f(*args_m)) / (2 * h)
        assert _fd_rel(np.sum(grad * d), fd) < 1e-5, k


def _window_problem(seed=4):
    """A small version of the differentiable window: 1,000 granules of
    r = 0.002 at volume fraction 0.3 on a 16^3 grid, 50 substeps of 2e-5 s."""
    return gi.make("diff_window_100k", seed=seed, n=1000, grid_n=16)


def _loss(prob, x):
    return np.mean(np.sum((x - prob.target) ** 2, axis=1))


def test_window_gradients_match_central_fd():
    """dL/dv0 (random direction), dL/dc_drag, dL/dmu over a 50-substep window
    against central FD (h = 1e-4 relative), on contact-stable windows."""
    prob = _window_problem()
    # enough contact to make mu matter: squeeze the packing by moving every granule towards the floor
    K = prob.K
    x0 = prob.positions()
    n = prob.n
    gxK = 2 * (oracle.run(prob, K=K)["x"] - prob.target) / n
    adj = oracle.run_adjoint(prob, gxK, K=K, signature=True)
    out = oracle.run(prob, K=K)
    assert np.allclose(adj["x"], out["x"], rtol=0, atol=0)
    rng = np.random.default_rng(7)
    w = rng.normal(size=(n, 3))
    v0 = prob.v.astype(float)
    h = 1e-4 * np.abs(v0).max()

    def L_of(v=None, P=None):
        r = oracle.run_adjoint(prob, np.zeros((n, 3)), K=K, v=v, params=P, signature=True)
        return _loss(prob, r["x"]), r["sig"]

    Lp, sp = L_of(v=v0 + h * w)
    Lm, sm = L_of(v=v0 - h * w)
    checked = 0
    if sp == sm == adj["sig"]:
        assert _fd_rel(np.sum(adj["g_v0"] * w), (Lp - Lm) / (2 * h)) < 1e-3
        checked += 1
    P = prob.params
    for name, g in (("c_drag", adj["g_c"]), ("mu_fric", adj["g_mu"])):
        val = getattr(P, name)
        hh = 1e-4 * val
        Lp, sp = L_of(P=dataclasses.replace(P, **{name: val + hh}))
        Lm, sm = L_of(P=dataclasses.replace(P, **{name: val - hh}))
        if sp == sm == adj["sig"]:
            fd = (Lp - Lm) / (2 * hh)
            assert _fd_rel(g, fd) < 1e-3 or abs(g - fd) < 1e-12 * abs(_loss(prob, out["x"])), (name, g, fd)
            checked += 1
    assert checked >= 2


def test_window_adjoint_with_contacts_matches_fd():
    """A window with real contacts (the dense block): dL/dv0 and dL/dmu by FD."""
    prob = gi.make("dense_block", n_side=(4, 4, 4))
    K = 10
    n = prob.n
    rng = np.random.default_rng(9)
    target = prob.positions() + rng.normal(size=(n, 3)) * 1e-4
    out = oracle.run(prob, K=K)
    gxK = 2 * (out["x"] - target) / n
    adj = oracle.run_adjoint(prob, gxK, K=K, signature=True)
    w = rng.normal(size=(n, 3))
    v0 = prob.v.astype(float)
    h = 1e-4 * np.abs(v0).max()
    L = lambda r: np.mean(np.sum((r["x"] - target) ** 2, axis=1))
    rp = oracle.run_adjoint(prob, np.zeros((n, 3)), K=K, v=v0 + h * w, signature=True)
    rm = oracle.run_adjoint(prob, np.zeros((n, 3)), K=K, v=v0 - h * w, signature=True)
    assert rp["sig"] == rm["sig"] == adj["sig"], "contact set changed: pick another seed"
    assert _fd_rel(np.sum(adj["g_v0"] * w), (L(rp) - L(rm)) / (2 * h)) < 1e-3
    P = prob.params
    hm = 1e-4 * P.mu_fric
    rp = oracle.run_adjoint(prob, np.zeros((n, 3)), K=K, params=dataclasses.replace(P, mu_fric=P.mu_fric + hm), signature=True)
    rm = oracle.run_adjoint(prob, np.zeros((n, 3)), K=K, params=dataclasses.replace(P, mu_fric=P.mu_fric - hm), signature=True)
    assert rp["sig"] == rm["sig"] == adj["sig"]
    assert _fd_rel(adj["g_mu"], (L(rp) - L(rm)) / (2 * hm)) < 1e-3
    assert adj["sig"][1] > 0  # some contacts slip: the Coulomb branch is exercised


def test_contact_vjp_with_capillary_matches_fd():
    """The contact adjoint with the capillary pair force (Sec. 5.4) on the wet
    block (most neighbours 1-3% of r apart, a fluid fraction rising in z, so
    that sr and with it Gamma vary with position): positions and velocities,
    against central FD of the forward.  The position step stays far inside
    every band where a pair would switch between contact, bridge and
    nothing."""
    prob = gi.make("wet_block")
    P = prob.params
    x, v, r = prob.positions(), prob.v.astype(float), prob.r.astype(float)
    rng = np.random.default_rng(7)
    lam = rng.normal(size=x.shape)
    dX, dV = rng.normal(size=x.shape), rng.normal(size=x.shape)
    gx, gv, gmu = oracle.contact_adj(prob.grid, P, x, v, r, lam, alpha_f=prob.alpha_f)
    f = lambda xx, vv, PP=P: np.sum(lam * oracle.contact(prob.grid, PP, xx, vv, r, alpha_f=prob.alpha_f)[0])
    hx = 1e-10
    fd_x = (f(x + hx * dX, v) - f(x - hx * dX, v)) / (2 * hx)
    assert _fd_rel(np.sum(gx * dX), fd_x) < 1e-5
    hv = 1e-7
    assert _fd_rel(np.sum(gv * dV), (f(x, v + hv * dV) - f(x, v - hv * dV)) / (2 * hv)) < 1e-5
    # the capillary part alone carries a position gradient: sigma = 0 changes it
    gx0, _, _ = oracle.contact_adj(prob.grid, dataclasses.replace(P, sigma=0.0), x, v, r, lam)
    assert np.abs(gx - gx0).max() > 1e-4 * np.abs(gx).max()


def test_window_adjoint_with_capillary_matches_fd():
    """A 10-substep window of a small wet block with the capillary force:
    dL/dv0 . w and dL/dmu against central FD (h = 1e-4 relative), on a
    contact-stable window (contact, slip and bridge flags identical in the
    +h and -h runs)."""
    prob = gi.make("wet_block", n_side=(3, 3, 3), K=10)
    n, K = prob.n, prob.K
    rng = np.random.default_rng(8)
    target = prob.positions() + rng.normal(size=(n, 3)) * 1e-4
    x0 = prob.positions()
    out = oracle.run(prob, K=K)
    gxK = 2 * (out["x"] - target) / n
    adj = oracle.run_adjoint(prob, gxK, K=K, signature=True)
    L = lambda r_: float(np.mean(np.sum((r_["x"] - target) ** 2, axis=1)))
    w = rng.normal(size=(n, 3))
    v0 = prob.v.astype(float)
    h = 1e-4 * np.abs(v0).max()
    rp = oracle.run_adjoint(prob, np.zeros((n, 3)), K=K, v=v0 + h * w, signature=True)
    rm = oracle.run_adjoint(prob, np.zeros((n, 3)), K=K, v=v0 - h * w, signature=True)
    assert rp["sig"] == rm["sig"] == adj["sig"], "window not contact-stable"
    assert adj["sig"][1] > 0  # bridges (and perhaps slipping contacts) took part
    fd = (L(rp) - L(rm)) / (2 * h)
    assert _fd_rel(np.sum(adj["g_v0"] * w), fd) < 1e-3
    P = prob.params
    hm = 1e-4 * P.mu_fric
    rp = oracle.run_adjoint(prob, np.zeros((n, 3)), K=K, params=dataclasses.replace(P, mu_fric=P.mu_fric + hm),
                            signature=True)
    rm = oracle.run_adjoint(prob, np.zeros((n, 3)), K=K, params=dataclasses.replace(P, mu_fric=P.mu_fric - hm),
                            signature=True)
    assert rp["sig"] == rm["sig"]
    assert _fd_rel(adj["g_mu"], (L(rp) - L(rm)) / (2 * hm)) < 1e-3
    assert np.abs(x0 - prob.positions()).max() == 0.0
