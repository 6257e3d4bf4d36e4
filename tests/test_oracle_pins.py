"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed
form of the contact or drag law, an invariant (conservation, antisymmetry,
transposition), a special case with a textbook answer, or a brute-force
enumeration.  A plausible slip in the oracle (a dropped term, a wrong sign, a
shifted index, a transposed operand) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import gic_inputs as gi
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _empty_fluid(grid):
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    return (np.zeros((nx + 1) * ny * nz), np.zeros(nx * (ny + 1) * nz), np.zeros(nx * ny * (nz + 1)),
            np.zeros(nx * ny * nz), np.ones(nx * ny * nz))


def _problem(grid, params, x, v, r, fluid, K):
    cell, q = gi.encode_positions(np.asarray(x, float), grid)
    u, vf, wf, p, af = fluid
    return gi.Problem("pin", grid, params, K, cell, q, np.asarray(r, np.float32), np.asarray(v, np.float32),
                      u, vf, wf, p, af)


def _hydro_p64(grid, rho_f, g=9.8):
    """Hydrostatic pressure in FP64 (p = rho_f g (H - z) at centres)."""
    cc = gi.centre_coords(grid)
    H = grid.origin[2] + grid.nz * grid.dx
    p3 = np.broadcast_to(rho_f * g * (H - cc[2])[None, None, :], (grid.nx, grid.ny, grid.nz))
    return np.ascontiguousarray(np.transpose(p3, (2, 1, 0))).ravel()


# ----------------------------------------------------------------------------- sort

def _morton_py(x, y, z):
    """Bit interleave written with strings: bit b of x, y, z -> 3b, 3b+1, 3b+2."""
    bx, by, bz = (format(t, "021b") for t in (x, y, z))
    s = "".join(bz[i] + by[i] + bx[i] for i in range(21))
    return int(s, 2)


def test_morton_small_values():
    assert oracle.morton(1, 0, 0) == 1
    assert oracle.morton(0, 1, 0) == 2
    assert oracle.morton(0, 0, 1) == 4
    assert oracle.morton(2, 0, 0) == 8
    assert oracle.morton(3, 5, 7) == 431  # x=011, y=101, z=111 -> 110 101 111 (binary, high to low)
    rng = np.random.default_rng(3)
    for _ in range(200):
        x, y, z = (int(t) for t in rng.integers(0, 1024, 3))
        assert oracle.morton(x, y, z) == _morton_py(x, y, z)


def test_sort_is_the_stable_key_order():
    rng = np.random.default_rng(5)
    c = rng.integers(0, 6, size=(3000, 3)).astype(np.int32)  # many ties
    perm, keys = oracle.sort(c)
    want = sorted(range(len(c)), key=lambda i: (_morton_py(*c[i]), i))
    assert np.array_equal(perm, np.array(want))
    assert all(keys[k] == _morton_py(*c[perm[k]]) for k in range(len(c)))
    ck, st, ct = oracle.cell_table(keys)
    assert ct.sum() == len(c) and np.all(np.diff(ck.astype(np.int64)) > 0)
    for k, s, n in zip(ck, st, ct):
        assert np.all(keys[s:s + n] == k)


def test_cells_floor_of_position():
    prob = gi.make("dense_block")
    x = prob.positions()
    c = oracle.cells(prob.grid, x)
    assert np.array_equal(c, prob.cell)


# ----------------------------------------------------------------------------- contact set

@pytest.mark.parametrize("name", ["dense_block", "random_cloud"])
def test_contact_pairs_binned_equals_bruteforce(name):
    prob = gi.make(name)
    x = prob.positions()
    r = prob.r.astype(np.float64)
    brute = oracle.contact_pairs(prob.grid, x, r, brute=True)
    binned = oracle.contact_pairs(prob.grid, x, r, brute=False)
    as_set = lambda P: set(map(tuple, np.sort(P, axis=1).tolist()))
    assert as_set(brute) == as_set(binned)
    # independent enumeration with numpy pairwise distances
    d = np.linalg.norm(x[:, None, :] - x[None, :, :], axis=2)
    R = r[:, None] + r[None, :]
    ii, jj = np.nonzero(np.triu(d < R, k=1))
    assert as_set(np.stack([ii, jj], 1)) == as_set(brute)
    assert len(brute) > 0


def test_contact_forces_binned_equals_bruteforce_and_antisymmetric():
    prob = gi.make("dense_block")
    x = prob.positions()
    P = prob.params
    Pw = gi.Params(**{**P.__dict__, "walls": 0})
    Fb, st1 = oracle.contact(prob.grid, Pw, x, prob.v, prob.r, brute=True)
    Fc, st2 = oracle.contact(prob.grid, Pw, x, prob.v, prob.r, brute=False)
    assert st1 == 0 and st2 == 0
    scale = np.abs(Fb).max()
    assert np.abs(Fb - Fc).max() <= 1e-12 * scale
    # Newton's third law: without walls the pair forces cancel in the sum
    assert np.abs(Fb.sum(axis=0)).max() <= 1e-11 * scale


# ----------------------------------------------------------------------------- contact law closed forms

def _head_on(zeta, dt_frac, vimp=0.1):
    r0 = 0.004
    grid = gi.Grid(8, 8, 8, 1.0 / 8, k_contact=1)
    P = gi.Params(rho_f=0.0, zeta=zeta, g=(0.0, 0.0, 0.0), walls=0, virtual_mass=1)
    m = P.rho_s * 4 / 3 * math.pi * r0 ** 3
    meff = m / 2
    w0 = math.sqrt(P.k_n / meff)
    tc = math.pi / (w0 * math.sqrt(1 - zeta ** 2))
    dt = tc * dt_frac
    P.dt_sub = dt
    P.dt_fluid = dt
    gap = 2e-7
    x = np.array([[0.5 - r0 - gap / 2, 0.5, 0.5], [0.5 + r0 + gap / 2, 0.5, 0.5]])
    v = np.array([[vimp, 0, 0], [-vimp, 0, 0]])
    steps = int(2.0 / dt_frac)
    prob = _problem(grid, P, x, v, [r0, r0], _empty_fluid(grid), steps)
    out = oracle.run(prob, K=steps, x=x, v=v)
    return out, m


@pytest.mark.parametrize("zeta", [0.3, 0.1])
def test_two_sphere_restitution(zeta):
    """Linear spring-dashpot head-on impact: the normal ODE m_eff d'' + c d' +
    k d = 0 during contact gives e = exp(-pi zeta / sqrt(1 - zeta^2)) exactly
    (textbook result for c = 2 zeta sqrt(k m_eff)); the symplectic Euler error
    is O(dt / t_c)."""
    e_exact = math.exp(-math.pi * zeta / math.sqrt(1 - zeta ** 2))
    if zeta == 0.3:
        assert abs(e_exact - _golden()["restitution_zeta_0.3"]["value"]) < 1e-5
    errs = []
    for frac in (1 / 200, 1 / 400):
        out, _ = _head_on(zeta, frac)
        v = out["v"]
        e = (v[1, 0] - v[0, 0]) / (2 * 0.1)
        assert abs(v[0, 1]) + abs(v[0, 2]) < 1e-14
        errs.append(abs(e - e_exact) / e_exact)
    assert errs[0] < 1e-2
    assert errs[1] < errs[0]  # first-order convergence in dt


def test_coulomb_sliding_on_floor():
    """A granule resting on the floor (normal force m g at the equilibrium
    overlap m g / k_n) and sliding at v0 decelerates at exactly mu g while the
    Coulomb cap is active (Sec. 3.1: F_t = min(|f_t|, |F_n| tan(phi)))."""
    r0 = 0.004
    grid = gi.Grid(8, 8, 8, 1.0 / 8, k_contact=1)
    P = gi.Params(rho_f=0.0, g=(0.0, 0.0, -9.8), dt_sub=1e-5, dt_fluid=1e-5)
    m = P.rho_s * 4 / 3 * math.pi * r0 ** 3
    delta = m * 9.8 / P.k_n
    v0 = 0.1
    x = np.array([[0.5, 0.5, r0 - delta]])
    v = np.array([[v0, 0.0, 0.0]])
    t_half = 0.5 * v0 / (P.mu_fric * 9.8)
    K = int(round(t_half / P.dt_sub))
    prob = _problem(grid, P, x, v, [r0], _empty_fluid(grid), K)
    out = oracle.run(prob, K=K, x=x, v=v)
    vx = out["v"][0, 0]
    want = v0 - P.mu_fric * 9.8 * K * P.dt_sub
    assert abs(vx - want) <= 1e-9 * v0
    assert abs(out["v"][0, 2]) < 1e-9


@pytest.mark.parametrize("kt_over_cn", [1.0, 0.5])
def test_viscous_tangential_below_the_cap_on_floor(kt_over_cn):
    """The sub-cap branch of the tangential law (Sec. 3.1: f_t = -k_t v_t on
    the relative tangential velocity, used while |f_t| < tan(phi) |F_n|),
    with the reading k_t = kt_over_cn c_n, c_n = 2 zeta sqrt(k_n m_eff) and
    m_eff = m for a wall.  A granule resting on the floor at the equilibrium
    overlap m g / k_n, sliding at v0 well under the cap (k_t v0 < mu m g / 5),
    has v_t = (v_x, 0, 0) exactly (the floor normal is z), so symplectic Euler
    gives v_x after K substeps = v0 (1 - dt' k_t / m)^K, whatever the small
    normal motion does.  With the constants below dt' k_t / m = 0.071
    (kt_over_cn = 1): after 20 substeps the factor is 0.228.  Plausible
    mistakes all fail by far more than the 1e-9 tolerance: k_t = c_n / 2 gives
    0.484, k_t = kt_over_cn k_n gives a growing oscillation (dt' k_t / m =
    1408), m_eff = m / 2 (a granule pair's) gives 0.356, and a dropped dashpot
    factor 2 in c_n gives 0.484."""
    r0 = float(np.float32(0.004))  # radii are stored as float32
    grid = gi.Grid(8, 8, 8, 1.0 / 8, k_contact=1)
    P = gi.Params(rho_f=0.0, c_drag=0.0, kt_over_cn=kt_over_cn, g=(0.0, 0.0, -9.8), dt_sub=1e-5, dt_fluid=1e-5)
    m = P.rho_s * 4 / 3 * math.pi * r0 ** 3
    delta = m * 9.8 / P.k_n
    cn = 2 * P.zeta * math.sqrt(P.k_n * m)
    kt = kt_over_cn * cn
    v0 = 0.2 * P.mu_fric * m * 9.8 / kt
    x = np.array([[0.5, 0.5, r0 - delta]])
    v = np.array([[v0, 0.0, 0.0]])
    K = 20
    prob = _problem(grid, P, x, v, [r0], _empty_fluid(grid), K)
    out = oracle.run(prob, K=K, x=x, v=v)
    want = v0 * (1.0 - P.dt_sub * kt / m) ** K
    assert abs(out["v"][0, 0] - want) <= 1e-9 * v0
    assert out["v"][0, 1] == 0.0
    # the branch really is the viscous one: the speed decays geometrically,
    # not linearly at mu g (the slip branch of test_coulomb_sliding_on_floor)
    assert abs(out["v"][0, 0] - (v0 - P.mu_fric * 9.8 * K * P.dt_sub)) > 1e-3 * v0
    assert out["status"] == 0


@pytest.mark.parametrize("c_drag,key", [(0.22, "terminal_velocity_cdrag_0.22"), (5.28, "terminal_velocity_cdrag_5.28")])
def test_terminal_settling_velocity(c_drag, key):
    """Quadratic drag F_d = c_drag pi r^2 rho_f |dv| dv balancing the buoyant
    weight (rho_s - rho_f) V g gives v_t = sqrt(4 (rho_s - rho_f) r g / (3
    c_drag rho_f)); the virtual mass changes only the transient."""
    r0 = 0.004
    grid = gi.Grid(4, 4, 32, 1.0 / 16, k_contact=1)
    P = gi.Params(c_drag=c_drag, dt_sub=1e-4, dt_fluid=1e-4, walls=0)
    vt = math.sqrt(4 * (P.rho_s - P.rho_f) * r0 * 9.8 / (3 * c_drag * P.rho_f))
    assert abs(vt - _golden()[key]["value"]) < 1e-4
    u, vf, wf, _, af = _empty_fluid(grid)
    p = _hydro_p64(grid, P.rho_f)
    x = np.array([[0.125, 0.125, 1.9]])
    v = np.zeros((1, 3))
    K = 15000 if c_drag < 1 else 3000
    prob = _problem(grid, P, x, v, [r0], (u, vf, wf, p, af), K)
    out = oracle.run(prob, K=K, x=x, v=v)
    assert out["x"][0, 2] > 0.2
    assert abs(-out["v"][0, 2] - vt) <= 1e-6 * vt
    assert abs(out["v"][0, 0]) + abs(out["v"][0, 1]) < 1e-12


@pytest.mark.parametrize("vm,rho_s,key", [(1, 2650.0, "first_step_accel_vm"), (0, 2650.0, "first_step_accel_novm"),
                                          (1, 1000.0, None)])
def test_buoyancy_and_virtual_mass_first_step(vm, rho_s, key):
    """From rest in hydrostatic fluid: (m + m_a) a = (m - rho_f V) g, so
    a = (rho_s - rho_f) / (rho_s + rho_f / 2) g with virtual mass (Eq. sand
    kine, m_a = (2/3) pi r^3 rho_f) and (rho_s - rho_f) / rho_s g without;
    neutrally buoyant granules do not move."""
    r0 = 0.004
    grid = gi.Grid(8, 8, 8, 1.0 / 8, k_contact=1)
    P = gi.Params(rho_s=rho_s, virtual_mass=vm, walls=0, dt_sub=1e-5, dt_fluid=1e-5)
    u, vf, wf, _, af = _empty_fluid(grid)
    p = _hydro_p64(grid, P.rho_f)
    x = np.array([[0.41, 0.52, 0.47]])
    prob = _problem(grid, P, x, np.zeros((1, 3)), [r0], (u, vf, wf, p, af), 1)
    out = oracle.run(prob, K=1, x=x, v=np.zeros((1, 3)))
    a = out["v"][0] / P.dt_sub
    want = (rho_s - P.rho_f) / (rho_s + (0.5 * P.rho_f if vm else 0.0)) * 9.8
    if key is not None:
        assert abs(want - _golden()[key]["value"]) < 1e-4
    assert abs(a[2] + want) <= 1e-10 * 9.8
    assert abs(a[0]) + abs(a[1]) <= 1e-10


# ----------------------------------------------------------------------------- interpolation

def _sample_field(grid, comp, fn):
    axes = gi.face_coords(grid, comp) if comp < 3 else gi.centre_coords(grid)
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    return np.ascontiguousarray(np.transpose(fn(X, Y, Z), (2, 1, 0))).ravel()


def _interior_points(grid, n, seed=0):
    rng = np.random.default_rng(seed)
    lo = np.array(grid.origin) + 1.0 * grid.dx
    hi = np.array(grid.origin) + grid.extent - 1.0 * grid.dx
    return lo + rng.uniform(size=(n, 3)) * (hi - lo)


@pytest.mark.parametrize("comp", [0, 1, 2, 3])
def test_trilinear_reproduces_affine_fields(comp):
    grid = gi.Grid(7, 9, 6, 0.1, origin=(0.3, -0.2, 1.0))
    fn = lambda X, Y, Z: 1.5 - 2.0 * X + 3.0 * Y + 0.25 * Z
    f = _sample_field(grid, comp, fn)
    x = _interior_points(grid, 500)
    got = oracle.interp(grid, comp, f, x)
    assert np.abs(got - fn(x[:, 0], x[:, 1], x[:, 2])).max() < 1e-12


def test_boundary_clamp_takes_end_sample():
    grid = gi.Grid(5, 5, 5, 0.2)
    f = _sample_field(grid, 3, lambda X, Y, Z: X + 10 * Y + 100 * Z)
    # a point in the outer half-cell: x below the first centre
    x = np.array([[0.05, 0.5, 0.5]])
    got = oracle.interp(grid, 3, f, x)[0]
    assert abs(got - (0.1 + 10 * 0.5 + 100 * 0.5)) < 1e-12


def test_grad_p_face_differences_are_centred():
    """For p = x^2 + 2y^2 + 3z^2 the face difference (p_i - p_{i-1}) / dx equals
    the exact derivative at the face, so the interpolated gradient is exact
    at interior points; an index shift would be off by 2 dx."""
    grid = gi.Grid(8, 7, 9, 0.125, origin=(0.1, 0.0, -0.3))
    p = _sample_field(grid, 3, lambda X, Y, Z: X ** 2 + 2 * Y ** 2 + 3 * Z ** 2)
    x = _interior_points(grid, 300, seed=1)
    gp = oracle.interp_grad_p(grid, p, x)
    want = np.stack([2 * x[:, 0], 4 * x[:, 1], 6 * x[:, 2]], 1)
    assert np.abs(gp - want).max() < 1e-11


def test_hydrostatic_gradient_exact_up_to_walls():
    grid = gi.Grid(6, 6, 10, 0.1)
    p = _hydro_p64(grid, 1000.0)
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, size=(400, 3)) * grid.extent
    gp = oracle.interp_grad_p(grid, p, x)
    assert np.abs(gp - np.array([0, 0, -9800.0])).max() < 1e-9


# ----------------------------------------------------------------------------- P2G

def _random_granules(grid, n, seed):
    rng = np.random.default_rng(seed)
    x = np.array(grid.origin) + rng.uniform(0, 1, size=(n, 3)) * grid.extent
    r = rng.uniform(0.2, 0.45, size=n) * grid.dx
    return x, r


def test_p2g_is_transpose_of_g2p():
    """<P2G f, g> = <f, G2P g>: the scatter uses exactly the weights of the
    gather (pins the folding of out-of-domain weights and the staggering)."""
    grid = gi.Grid(6, 5, 7, 0.1, origin=(0.0, 0.2, -0.1))
    x_old, r = _random_granules(grid, 400, 7)
    x_new = x_old + np.random.default_rng(8).normal(0, 0.02, size=x_old.shape)
    fex = np.random.default_rng(9).normal(size=x_old.shape)
    P = gi.Params(dt_sub=1e-5, dt_fluid=3e-5)
    alpha, Fs, sums = oracle.p2g(grid, P, x_old, x_new, r, fex)
    rng = np.random.default_rng(10)
    g = rng.normal(size=alpha.shape)
    V = 4 / 3 * np.pi * r ** 3
    lhs = np.dot(alpha, g) * grid.dx ** 3
    rhs = np.dot(V, oracle.interp(grid, 3, g, x_new))
    assert abs(lhs - rhs) <= 1e-13 * np.abs(V).sum() * np.abs(g).max()
    for comp in range(3):
        h = rng.normal(size=Fs[comp].shape)
        lhs = np.dot(Fs[comp], h)
        rhs = -(P.dt_sub / P.dt_fluid) * np.dot(fex[:, comp], oracle.interp(grid, comp, h, x_old))
        assert abs(lhs - rhs) <= 1e-12 * np.abs(fex).sum() * np.abs(h).max()


def test_volume_and_momentum_conservation():
    grid = gi.Grid(6, 5, 7, 0.1)
    x_old, r = _random_granules(grid, 1000, 11)
    x_new = x_old.copy()
    fex = np.random.default_rng(12).normal(size=x_old.shape)
    P = gi.Params(dt_sub=1e-5, dt_fluid=4e-5)
    alpha, Fs, sums = oracle.p2g(grid, P, x_old, x_new, r, fex)
    V = 4 / 3 * np.pi * r ** 3
    assert abs(sums[1] - V.sum()) <= 1e-14 * V.sum()
    assert abs(sums[0] - V.sum()) <= 1e-12 * V.sum()
    for comp in range(3):
        assert abs(Fs[comp].sum() + P.dt_sub / P.dt_fluid * fex[:, comp].sum()) <= 1e-12 * np.abs(fex).sum()


def test_alpha_s_of_uniform_lattice():
    """One granule per cell centre -> alpha_s = V / dx^3 in every cell."""
    grid = gi.Grid(4, 4, 4, 0.25)
    cc = gi.centre_coords(grid)
    X, Y, Z = np.meshgrid(*cc, indexing="ij")
    x = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    r = np.full(x.shape[0], 0.05)
    alpha, _, _ = oracle.p2g(grid, gi.Params(), x, x, r, np.zeros_like(x))
    assert np.allclose(alpha, 4 / 3 * np.pi * 0.05 ** 3 / 0.25 ** 3, rtol=1e-14, atol=0)


# ----------------------------------------------------------------------------- integrate

def test_exchange_force_is_total_fluid_force_on_granule():
    """f_ex is every force the fluid exerts on the granule (Sec. 5.2): from
    Newton's law for the granule alone, f_ex = m (v' - v) / dt - m g - F_c."""
    prob = gi.make("dense_block")
    x = prob.positions()
    P = prob.params
    F_c, _ = oracle.contact(prob.grid, P, x, prob.v, prob.r)
    F_fl, a_f, _ = oracle.g2p(prob.grid, P, x, prob.v, prob.r, prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)
    xn, vn, fex, st = oracle.integrate(prob.grid, P, x, prob.v, prob.r, F_c, F_fl, a_f)
    m = P.rho_s * 4 / 3 * np.pi * prob.r.astype(np.float64) ** 3
    want = m[:, None] * (vn - prob.v) / P.dt_sub - m[:, None] * np.array(P.g) - F_c
    scale = np.abs(F_c).max() + np.abs(F_fl).max()
    assert np.abs(fex - want).max() <= 1e-9 * scale
    assert np.allclose(xn, x + P.dt_sub * vn, rtol=0, atol=1e-15)


def test_drag_law_direction_and_magnitude_single_granule():
    """Uniform fluid velocity, granule at rest, no pressure: F_d = c pi r^2
    rho_f |u| u, directed along u."""
    grid = gi.Grid(4, 4, 4, 0.25)
    nx = 4
    U = np.array([0.3, -0.2, 0.1])
    u = np.full((nx + 1) * nx * nx, U[0])
    vf = np.full(nx * (nx + 1) * nx, U[1])
    wf = np.full(nx * nx * (nx + 1), U[2])
    p = np.zeros(nx ** 3)
    af = np.ones(nx ** 3)
    P = gi.Params(c_drag=0.22)
    r = 0.01
    F, a_f, afp = oracle.g2p(grid, P, np.array([[0.4, 0.6, 0.5]]), np.zeros((1, 3)), np.array([r]), u, vf, wf, p, af)
    want = 0.22 * math.pi * r * r * 1000.0 * np.linalg.norm(U) * U
    assert np.allclose(F[0], want, rtol=1e-13, atol=0)
    assert np.allclose(a_f[0], P.g, rtol=0, atol=1e-15)
    assert afp[0] == 1.0


def test_oracle_run_plain_config_is_quiet():
    """The plain 8k configuration has no initial contacts: after 10 substeps
    the oracle reports no status bit and the granule volume is conserved."""
    prob = gi.make("plain_fp64_8k")
    out = oracle.run(prob)
    assert out["status"] == 0
    assert abs(out["sums"][0] - out["sums"][1]) <= 1e-12 * out["sums"][1]
