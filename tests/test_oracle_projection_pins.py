"""Pins of the projection oracle (oracle/projection.py) against what the paper
and the mathematics fix, independently of the oracle's own construction:

* Eq. backward Euler: after the density projection the displacement obeys
  alpha_f' - alpha_f* + div(alpha_f' dx) = 0 (with dx = v' dt of Eq.
  position change), and after the velocity projection div(alpha_f' v') = 0;
  both checked with a divergence written here with array slicing.
* uniform alpha_f': the operator is the textbook 7-point Laplacian
  (Kronecker sums of 1-D second differences with Neumann ends at walls and a
  p = 0 ghost cell beyond an open side).
* a 1-D column with uniform alpha_f' and uniform density right-hand side has
  the closed-form quadratic solution.
* a discretely divergence-free v* (the MAC curl of a vector potential) with
  uniform alpha_f' is left unchanged (p1 = 0).
* the densest-packing, ratio and one-cell limits stated after Eq. position
  change; symmetry and definiteness of the operator.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import gic_inputs as gi
from oracle import projection as pj


def faces3(case, f, axis):
    nx, ny, nz = case.shape if hasattr(case, "shape") else case
    shp = [nz, ny, nx]
    shp[2 - axis] += 1
    return np.asarray(f, np.float64).reshape(shp)


def slice_divergence(shape, h, alpha_p, open_sides, fu, fv, fw):
    """div(alpha f) per cell with numpy slicing: interior face weight = mean
    of the two cells, open boundary face = the inner cell's value, solid
    boundary face = no flux.  Returns an (nz, ny, nx) array."""
    nx, ny, nz = shape
    a = np.asarray(alpha_p, np.float64).reshape(nz, ny, nx)
    div = np.zeros((nz, ny, nx))
    for axis, f in enumerate((fu, fv, fw)):
        ax = 2 - axis
        F = faces3(shape, f, axis)
        m = a.shape[ax]
        beta = np.zeros(F.shape)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        mid = [slice(None)] * 3
        lo[ax], hi[ax], mid[ax] = slice(0, m - 1), slice(1, m), slice(1, m)
        beta[tuple(mid)] = 0.5 * (a[tuple(lo)] + a[tuple(hi)])
        s0 = [slice(None)] * 3
        s0[ax] = 0
        s1 = [slice(None)] * 3
        s1[ax] = m
        c0 = [slice(None)] * 3
        c0[ax] = 0
        c1 = [slice(None)] * 3
        c1[ax] = m - 1
        if open_sides[2 * axis]:
            beta[tuple(s0)] = a[tuple(c0)]
        if open_sides[2 * axis + 1]:
            beta[tuple(s1)] = a[tuple(c1)]
        flux = beta * F
        up = [slice(None)] * 3
        dn = [slice(None)] * 3
        up[ax] = slice(1, m + 1)
        dn[ax] = slice(0, m)
        div += (flux[tuple(up)] - flux[tuple(dn)]) / h
    return div


def slice_gradient(shape, h, p, open_sides, axis):
    """(p_R - p_L) / h on the faces of grid `axis`, p = 0 beyond open sides, 0 on solid sides."""
    nx, ny, nz = shape
    P = np.asarray(p, np.float64).reshape(nz, ny, nx)
    ax = 2 - axis
    m = P.shape[ax]
    pad = [(0, 0)] * 3
    pad[ax] = (1, 1)
    Pp = np.pad(P, pad)  # zero ghosts
    up = [slice(None)] * 3
    dn = [slice(None)] * 3
    up[ax] = slice(1, m + 2)
    dn[ax] = slice(0, m + 1)
    g = (Pp[tuple(up)] - Pp[tuple(dn)]) / h
    s0 = [slice(None)] * 3
    s0[ax] = 0
    s1 = [slice(None)] * 3
    s1[ax] = m
    if not open_sides[2 * axis]:
        g[tuple(s0)] = 0.0
    if not open_sides[2 * axis + 1]:
        g[tuple(s1)] = 0.0
    return g


CASES = [
    dict(seed=31, shape=(21, 18, 25), open_sides=(0, 0, 0, 0, 0, 1)),
    dict(seed=32, shape=(12, 9, 7), open_sides=(1, 1, 1, 1, 1, 1)),
    dict(seed=33, shape=(16, 5, 11), open_sides=(0, 1, 0, 0, 1, 0)),
]


@pytest.mark.parametrize("kw", CASES)
def test_continuity_after_projection(kw):
    """Eq. backward Euler for both projections (the one-cell limit is inactive in these cases)."""
    c = gi.projection_case(dt=2e-4, **kw)
    out = pj.project(c.shape, c.dx, c.alpha_s, c.alpha_star, c.u, c.v, c.w, c.dt, c.rho_f, c.open_sides)
    ap = out["alpha_p"]
    nx, ny, nz = c.shape
    # velocity projection: div(alpha' v') = 0, relative to the divergence of v*
    d0 = slice_divergence(c.shape, c.dx, ap, c.open_sides, c.u, c.v, c.w)
    d1 = slice_divergence(c.shape, c.dx, ap, c.open_sides, out["u"], out["v"], out["w"])
    assert np.abs(d0).max() > 1.0
    assert np.abs(d1).max() <= 1e-10 * np.abs(d0).max()
    # v' = v* - (dt / rho) grad p1 on non-solid faces
    for axis, (f0, f1) in enumerate(((c.u, out["u"]), (c.v, out["v"]), (c.w, out["w"]))):
        g = slice_gradient(c.shape, c.dx, out["p1"], c.open_sides, axis)
        want = faces3(c.shape, f0, axis) - (c.dt / c.rho_f) * g
        F1 = faces3(c.shape, f1, axis)
        nonsolid = np.ones_like(g, bool)
        ax = 2 - axis
        m = [nz, ny, nx][ax]
        for side, idx in ((2 * axis, 0), (2 * axis + 1, m)):
            if not c.open_sides[side]:
                s = [slice(None)] * 3
                s[ax] = idx
                nonsolid[tuple(s)] = False
        assert np.allclose(F1[nonsolid], want[nonsolid], rtol=0, atol=1e-12)
        assert np.all(F1[~nonsolid] == 0)
    # density projection: alpha' - alpha*_clamped + div(alpha' dx) = 0
    a3 = ap.reshape(nz, ny, nx)
    star = np.asarray(c.alpha_star, np.float64).reshape(nz, ny, nx)
    star_c = np.clip(star, 0.5 * a3, 1.5 * a3)
    assert np.any(star != star_c)  # the ratio limit is active somewhere
    disp = [out["dxu"], out["dxv"], out["dxw"]]
    assert max(np.abs(d).max() for d in disp) < c.dx  # one-cell limit inactive here
    dd = slice_divergence(c.shape, c.dx, ap, c.open_sides, *disp)
    resid = a3 - star_c + dd
    assert np.abs(resid).max() <= 1e-10
    assert np.abs(dd).max() > 0.1


def test_uniform_fraction_gives_textbook_laplacian():
    """alpha_f' = 1 (no sand): A is the 7-point Laplacian built from 1-D
    second-difference matrices (Neumann at walls, Dirichlet ghost at open
    sides); alpha_f' = 0.4 everywhere scales it by 0.4."""
    def lap1(m, open_lo, open_hi):
        main = np.full(m, 2.0)
        main[0] = 2.0 if open_lo else 1.0
        main[-1] = 2.0 if open_hi else 1.0
        if m == 1:
            main[0] = float(open_lo) + float(open_hi)
        return sp.diags([main, -np.ones(m - 1), -np.ones(m - 1)], [0, -1, 1])

    for shape, sides in (((6, 5, 4), (0, 0, 0, 0, 0, 1)), ((3, 7, 5), (1, 1, 0, 1, 1, 0)), ((4, 1, 3), (1, 0, 0, 0, 0, 1))):
        nx, ny, nz = shape
        Lx, Ly, Lz = lap1(nx, sides[0], sides[1]), lap1(ny, sides[2], sides[3]), lap1(nz, sides[4], sides[5])
        Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
        # x fastest: index = i + nx (j + ny k)
        L = sp.kron(Iz, sp.kron(Iy, Lx)) + sp.kron(Iz, sp.kron(Ly, Ix)) + sp.kron(Lz, sp.kron(Iy, Ix))
        for level in (0.0, 0.6):
            A, _ = pj.operator(shape, pj.target_fraction(np.full(nx * ny * nz, level)), sides)
            assert abs(A - (1.0 - level) * L).max() <= 1e-15


def test_column_closed_form():
    """1-D column (nx = ny = 1, walls on x and y, floor solid, top open),
    uniform alpha_f' = a and alpha_f* = q a (q < 1): the density right-hand side is
    uniform, b = -(rho h^2/dt^2) a (1 - q), and the discrete solution is the
    quadratic p_k = b ((n + 1/2)^2 - (k + 1/2)^2) / (2 a) (zero slope at the
    floor, p = 0 half a cell above the top)."""
    n, h, dt, rho = 37, 0.01, 1e-3, 1000.0
    a, q = 0.7, 0.99
    alpha_s = np.full(n, 1.0 - a)
    out = pj.project((1, 1, n), h, alpha_s, np.full(n, q * a), np.zeros(2 * n), np.zeros(2 * n), np.zeros(n + 1), dt,
                     rho, (0, 0, 0, 0, 0, 1))
    b = -(rho * h * h / (dt * dt)) * a * (1.0 - q)
    k = np.arange(n)
    want = b * ((n + 0.5) ** 2 - (k + 0.5) ** 2) / (2 * a)
    assert np.allclose(out["p2"], want, rtol=1e-11, atol=0)
    assert np.all(out["p1"] == 0)
    # displacement on the z-faces: -(dt^2 / rho) dp/dz, zero at the floor
    dz = out["dxw"]
    assert dz[0] == 0.0
    zf = np.arange(1, n + 1)
    slope = -b * ((zf + 0.5) ** 2 - (zf - 0.5) ** 2) / (2 * a) / h  # p(z_k) - p(z_{k-1}) over h, k = 1..n (p_n = 0)
    assert np.abs(dz).max() < h  # the one-cell limit is not active
    assert np.allclose(dz[1:], -(dt * dt / rho) * slope, rtol=1e-10, atol=1e-18)
    # fluid below its target (q < 1) is drawn down into the column through the open top
    assert np.all(dz[1:] < 0)


def test_divergence_free_field_is_unchanged():
    """With uniform alpha_f' and every side open, the MAC curl of a random
    edge potential is discretely divergence-free: p1 = 0 and v' = v*."""
    nx, ny, nz = 9, 8, 7
    h = 0.05
    rng = np.random.default_rng(5)
    # edge potentials: psi_x on x-edges (nx, ny+1, nz+1), psi_y (nx+1, ny, nz+1), psi_z (nx+1, ny+1, nz) as [k, j, i]
    px = rng.normal(size=(nz + 1, ny + 1, nx))
    py = rng.normal(size=(nz + 1, ny, nx + 1))
    pz = rng.normal(size=(nz, ny + 1, nx + 1))
    # u = d psi_z/dy - d psi_y/dz on x-faces; v = d psi_x/dz - d psi_z/dx; w = d psi_y/dx - d psi_x/dy
    u = (pz[:, 1:, :] - pz[:, :-1, :]) / h - (py[1:, :, :] - py[:-1, :, :]) / h
    v = (px[1:, :, :] - px[:-1, :, :]) / h - (pz[:, :, 1:] - pz[:, :, :-1]) / h
    w = (py[:, :, 1:] - py[:, :, :-1]) / h - (px[:, 1:, :] - px[:, :-1, :]) / h
    sides = (1, 1, 1, 1, 1, 1)
    ap = np.full(nx * ny * nz, 0.55)
    d = slice_divergence((nx, ny, nz), h, ap, sides, u.ravel(), v.ravel(), w.ravel())
    assert np.abs(d).max() <= 1e-12 * np.abs(u).max() / h
    out = pj.project((nx, ny, nz), h, 1.0 - ap, ap, u.ravel(), v.ravel(), w.ravel(), 1e-3, 1000.0, sides)
    assert np.abs(out["p1"]).max() <= 1e-9 * (1000.0 * h / 1e-3) * np.abs(u).max()
    assert np.allclose(out["u"], u.ravel(), rtol=0, atol=1e-10 * np.abs(u).max())
    assert np.allclose(out["w"], w.ravel(), rtol=0, atol=1e-10 * np.abs(w).max())
    # alpha* = alpha' everywhere: nothing to move
    assert np.all(out["p2"] == 0) and np.all(out["dxu"] == 0)


def test_limits():
    """alpha_s beyond 0.740 gives alpha_f' = 0.26; the ratio limit
    [0.5, 1.5] and the one-cell displacement limit."""
    ap = pj.target_fraction(np.array([0.0, 0.5, 0.74, 0.9, 1.2]))
    assert np.allclose(ap, [1.0, 0.5, 0.26, 0.26, 0.26], rtol=0, atol=1e-15)
    b = pj.rhs_density(0.1, 1.0, 1.0, np.array([0.5, 0.5, 0.5]), np.array([0.1, 0.5, 2.0]))
    # ratio 0.2 -> 0.5, 1 -> 1, 4 -> 1.5: b = -h^2 a (1 - ratio)
    assert np.allclose(b, [-0.01 * 0.5 * 0.5, 0.0, 0.01 * 0.5 * 0.5], rtol=1e-14, atol=0)
    # a column with alpha_f* = 0.3 alpha_f' (clamped to 0.5): the unlimited
    # displacement on z-face k is -(1 - 0.5) k h (the column closed form), so
    # the one-cell limit binds from k = 2 upwards
    n, h = 12, 0.02
    a = 0.6
    out = pj.project((1, 1, n), h, np.full(n, 1.0 - a), np.full(n, 0.3 * a), np.zeros(2 * n), np.zeros(2 * n),
                     np.zeros(n + 1), 1e-3, 1000.0, (0, 0, 0, 0, 0, 1))
    k = np.arange(n + 1)
    assert np.allclose(out["dxw"], np.maximum(-0.5 * k * h, -h), rtol=1e-12, atol=1e-18)


def test_operator_symmetric_positive_definite():
    c = gi.projection_case(seed=35, shape=(8, 7, 9))
    ap = pj.target_fraction(c.alpha_s)
    A, _ = pj.operator(c.shape, ap, c.open_sides)
    assert abs(A - A.T).max() == 0.0
    lmin = spla.eigsh(A.tocsc(), k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    assert lmin > 0
    # every side solid: the constants are a null vector, and project refuses
    A0, _ = pj.operator(c.shape, ap, (0, 0, 0, 0, 0, 0))
    assert np.abs(A0 @ np.ones(A0.shape[0])).max() <= 1e-14
    with pytest.raises(ValueError):
        pj.project(c.shape, c.dx, c.alpha_s, c.alpha_star, c.u, c.v, c.w, c.dt, c.rho_f, (0, 0, 0, 0, 0, 0))
