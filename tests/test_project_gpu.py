"""GPU parity of gic_project (the velocity and density projections that
consume alpha_s, Sec. 5.1) against the FP64 oracle (oracle/projection.py).

The solver stops at an FP64 relative residual tol, so the GPU pressure is
compared with the oracle's direct solution within the bound the residual
implies: |p - p*|_2 <= |b - A p|_2 / lambda_min(A), lambda_min from scipy on
the small grids.  The face outputs are checked against the oracle's face
formulas evaluated on the GPU's own pressures (FP32 rounding of the output)
and through the constraints they must meet: div(alpha_f' v') = 0 and
alpha_f' - alpha_f* + div(alpha_f' dx) = 0 (Eq. backward Euler).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import gic_inputs as gi
from oracle import projection as pj
from paper_2504_00745_gb300 import gic

pytestmark = pytest.mark.gpu

TOL = 1e-9  # the solver's relative residual target in these tests


def grid_of(shape, h):
    import ctypes as C
    return gic.GicGrid(shape[0], shape[1], shape[2], 1, float(h), (C.c_double * 3)(0, 0, 0))


def run_gpu(c, tol=TOL, alpha_s=None, **kw):
    dev = torch.device("cuda")
    nx, ny, nz = c.shape
    n = nx * ny * nz
    a_s = torch.as_tensor(c.alpha_s if alpha_s is None else alpha_s, dtype=torch.float64, device=dev)
    star = torch.as_tensor(c.alpha_star, dtype=torch.float32, device=dev)
    u, v, w = (torch.as_tensor(f, dtype=torch.float32, device=dev) for f in (c.u, c.v, c.w))
    p1 = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
    p2 = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
    vo = [torch.full_like(f, np.nan) for f in (u, v, w)]
    do = [torch.full_like(f, np.nan) for f in (u, v, w)]
    params = gic.make_proj_params(c.dt, c.rho_f, c.open_sides, tol=tol, **kw)
    info = gic.gic_project(grid_of(c.shape, c.dx), params, a_s, star, u, v, w, p1, p2, vo, do)
    torch.cuda.synchronize()
    out = {"p1": p1.cpu().numpy(), "p2": p2.cpu().numpy(), "u": vo[0].cpu().numpy(), "v": vo[1].cpu().numpy(),
           "w": vo[2].cpu().numpy(), "dxu": do[0].cpu().numpy(), "dxv": do[1].cpu().numpy(),
           "dxw": do[2].cpu().numpy()}
    return out, info


def faces_from_p(ref, c, p1, p2):
    """The oracle's face formulas on given pressures."""
    h = c.dx
    g1 = pj.face_gradient(ref["ops"], p1, h)
    g2 = pj.face_gradient(ref["ops"], p2, h)
    vel, disp = [], []
    for (G, beta, mask), f, a, b in zip(ref["ops"], (c.u, c.v, c.w), g1, g2):
        vel.append(np.where(mask, np.asarray(f, np.float64) - (c.dt / c.rho_f) * a, 0.0))
        disp.append(np.where(mask, np.clip(-(c.dt * c.dt / c.rho_f) * b, -h, h), 0.0))
    return vel, disp


CASES = [
    dict(seed=31, shape=(21, 18, 25), open_sides=(0, 0, 0, 0, 0, 1)),
    dict(seed=32, shape=(12, 9, 7), open_sides=(1, 1, 1, 1, 1, 1)),
    dict(seed=33, shape=(16, 5, 11), open_sides=(0, 1, 0, 0, 1, 0)),
    dict(seed=36, shape=(1, 1, 40), open_sides=(0, 0, 0, 0, 0, 1)),
    dict(seed=37, shape=(67, 3, 2), open_sides=(1, 0, 0, 0, 0, 0)),
    dict(seed=38, shape=(40, 36, 44), open_sides=(0, 0, 0, 0, 0, 1)),
]


@pytest.mark.parametrize("kw", CASES, ids=lambda k: "x".join(map(str, k["shape"])))
def test_projection_matches_oracle(kw):
    c = gi.projection_case(**kw)
    ref = pj.project(c.shape, c.dx, c.alpha_s, c.alpha_star, c.u, c.v, c.w, c.dt, c.rho_f, c.open_sides)
    out, info = run_gpu(c)
    A = ref["A"]
    lmin = spla.eigsh(A.tocsc(), k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    for s, (p_key, b_key) in enumerate((("p1", "b1"), ("p2", "b2"))):
        b = ref[b_key]
        p = out[p_key]
        assert np.all(np.isfinite(p))
        res = np.linalg.norm(b - A @ p)
        nb = np.linalg.norm(b)
        assert info.converged[s] == 1
        assert info.rel_residual[s] <= TOL
        # the oracle's residual of the GPU solution agrees with the solver's own
        assert res <= 4 * TOL * nb + 1e-12 * np.abs(A).max() * np.abs(p).max()
        assert np.linalg.norm(p - ref[p_key]) <= res / lmin * 1.01 + 1e-12 * np.linalg.norm(ref[p_key])
    # face outputs: the oracle's formulas on the GPU's pressures, to FP32 rounding
    vel, disp = faces_from_p(ref, c, out["p1"], out["p2"])
    for key, want in list(zip(("u", "v", "w"), vel)) + list(zip(("dxu", "dxv", "dxw"), disp)):
        assert np.allclose(out[key], want, rtol=2 ** -23, atol=1e-9 * np.abs(want).max() + 1e-30)
    # constraints: div(alpha' v') = 0; alpha' - alpha*_clamped + div(alpha' dx) = 0 where no face is clamped
    d0 = pj.weighted_divergence(c.shape, c.dx, ref["ops"], (c.u, c.v, c.w))
    d1 = pj.weighted_divergence(c.shape, c.dx, ref["ops"], (out["u"], out["v"], out["w"]))
    assert np.abs(d1).max() <= 4e-6 * max(np.abs(d0).max(), 1e-30)  # FP32 rounding of v'
    ap = ref["alpha_p"]
    star_c = np.clip(np.asarray(c.alpha_star, np.float64), 0.5 * ap, 1.5 * ap)
    dd = pj.weighted_divergence(c.shape, c.dx, ref["ops"], (out["dxu"], out["dxv"], out["dxw"]))
    clamped = any(np.any(np.abs(d) >= c.dx) for d in disp)
    if not clamped:
        assert np.abs(ap - star_c + dd).max() <= 1e-5


def test_repeatable_and_zero_rhs():
    """Two calls give the same bits (fixed-order reductions); alpha_f* =
    alpha_f' with v* = 0 needs no iteration and gives p = 0."""
    c = gi.projection_case(seed=39, shape=(17, 13, 9))
    a, ia = run_gpu(c)
    b, ib = run_gpu(c)
    for k in a:
        assert np.array_equal(a[k], b[k])
    assert list(ia.inner) == list(ib.inner)
    ap = pj.target_fraction(c.alpha_s)
    z = gi.ProjectionCase(name="zero", shape=c.shape, dx=c.dx, alpha_s=c.alpha_s, alpha_star=ap.astype(np.float32),
                          u=np.zeros_like(c.u), v=np.zeros_like(c.v), w=np.zeros_like(c.w), dt=c.dt, rho_f=c.rho_f,
                          open_sides=c.open_sides)
    # alpha* rounded to float: the ratio is 1 to float rounding; p2 is the solution of that tiny right-hand side
    out, info = run_gpu(z)
    assert np.all(out["p1"] == 0) and info.inner[0] == 0 and info.converged[0] == 1
    assert np.all(out["u"] == 0) and np.all(out["v"] == 0) and np.all(out["w"] == 0)
    assert np.abs(out["dxu"]).max() <= 1e-6 * c.dx


def test_iteration_limits_report_not_converged():
    """A solve cut short by max_outer returns with converged = 0 and the
    residual it reached (larger than tol)."""
    c = gi.projection_case(seed=40, shape=(30, 30, 30))
    _, info = run_gpu(c, tol=1e-12, inner_tol=1e-10, max_outer=1, max_inner=5)
    assert info.converged[0] == 0 and info.converged[1] == 0
    assert info.outer[0] == 1 and info.inner[0] == 5
    assert info.rel_residual[0] > 1e-12


def test_argument_errors_with_device_buffers():
    c = gi.projection_case(seed=41, shape=(6, 5, 4))
    dev = torch.device("cuda")
    n = 6 * 5 * 4
    a_s = torch.as_tensor(c.alpha_s, device=dev)
    star = torch.as_tensor(c.alpha_star, device=dev)
    u, v, w = (torch.as_tensor(f, device=dev) for f in (c.u, c.v, c.w))
    p1, p2 = (torch.zeros(n, dtype=torch.float64, device=dev) for _ in range(2))
    g = grid_of(c.shape, c.dx)
    with pytest.raises(gic.GicError, match="open"):
        gic.gic_project(g, gic.make_proj_params(c.dt, c.rho_f, (0,) * 6), a_s, star, u, v, w, p1, p2)
    small = torch.empty(64, dtype=torch.uint8, device=dev)
    with pytest.raises(gic.GicError, match="workspace"):
        gic.gic_project(g, gic.make_proj_params(c.dt, c.rho_f), a_s, star, u, v, w, p1, p2, ws=small)
    bad = a_s.clone()
    bad[7] = float("nan")
    with pytest.raises(gic.GicError, match="non-finite"):
        gic.gic_project(g, gic.make_proj_params(c.dt, c.rho_f), bad, star, u, v, w, p1, p2)
    gic.gic_check_status(clear=True)
