"""FP64 CPU oracle of the pressure projections that consume alpha_s.

TEST INFRASTRUCTURE ONLY: imported by the test-suite and the benchmark's
CPU-baseline leg, never by the product package.  Plain numpy / scipy: the
operator is assembled as a sparse matrix and each system is solved directly
(SuperLU), so the result is the exact solution of the discrete equations up
to rounding.

What it computes (Sec. 5.1, Eqs. discret momentum, backward Euler, bring2,
ppe1 a/b, position change; the limits on alpha_s, on alpha_f*/alpha_f' and on
|dx| stated after Eq. position change; the face coefficient beta of the
appendix on the Push-Out boundary condition):

  alpha_f' = 1 - min(alpha_s, alpha_s_max)                       (target fluid fraction)
  (dt / rho0)   div(alpha_f' grad p1) = div(alpha_f' v*)          (velocity projection, Eq. ppe1 a times alpha_f')
  (dt^2 / rho0) div(alpha_f' grad p2) = alpha_f' (1 - clamp(alpha_f* / alpha_f', lo, hi))
                                                                  (density projection, Eq. ppe1 b times alpha_f')
  v'  = v* - (dt / rho0) grad p1                                  (Eq. discret momentum)
  dx  = clamp(-(dt^2 / rho0) grad p2, -h, h)                      (Eq. position change, |dx| within one cell)

on the MAC grid (cells nx ny nz of side h, x fastest; u on x-faces etc.):

  * grad is the face difference (p_R - p_L) / h; div the cell's net face flux / h.
  * The face weight beta between two cells is the mean of their alpha_f'
    (the appendix's beta_j).  A side of the box is either a solid wall at
    rest (no flux: v = 0 there and no pressure coupling; the Push-Out term of
    the appendix vanishes without fluid particles inside the wall) or open
    (fluid-air interface: p = 0 in the cell beyond, face weight the inner
    cell's alpha_f').
  * Both equations are multiplied by alpha_f' (so the matrix is symmetric);
    the solution is that of Eq. ppe1 itself.

With G the face-difference matrix (rows: non-solid faces, open faces have
the outside cell at p = 0) and B = diag(beta), the discrete operator is
div(alpha grad p) = -(1/h^2) G^T B G p, so the systems are

  A p1 = (rho0 h / dt) G^T (B v*)                 with A = G^T B G
  A p2 = -(rho0 h^2 / dt^2) alpha' (1 - clamp(alpha*/alpha'))

A is symmetric positive definite when at least one side is open.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

SIDES = ("-x", "+x", "-y", "+y", "-z", "+z")


def target_fraction(alpha_s, alpha_s_max=0.740):
    """alpha_f' = 1 - min(alpha_s, alpha_s_max) (the densest-packing limit
    stated after Eq. position change)."""
    return 1.0 - np.minimum(np.asarray(alpha_s, np.float64), alpha_s_max)


def _cell_id(shape):
    nx, ny, nz = shape
    return np.arange(nx * ny * nz).reshape(nz, ny, nx)  # [k, j, i], x fastest


def face_operator(shape, alpha_p, open_sides):
    """Face-difference matrices and face weights for the three face grids.

    Returns, per axis a (0 = x-faces, ...), (G_a, beta_a, mask_a): G_a maps
    cell values to (p_R - p_L) on every face of that grid (solid boundary
    faces get an empty row), beta_a the face weights and mask_a the faces
    that are not solid.  Face arrays are flattened x fastest with
    n_a + 1 samples along axis a."""
    nx, ny, nz = shape
    n = nx * ny * nz
    ap = np.asarray(alpha_p, np.float64).reshape(nz, ny, nx)
    ids = _cell_id(shape)
    out = []
    for a in range(3):
        ax = 2 - a  # numpy axis of the grid axis a in the [k, j, i] layout
        nf = list(ap.shape)
        nf[ax] += 1
        nfaces = int(np.prod(nf))
        fid = np.arange(nfaces).reshape(nf)
        beta = np.zeros(nf)
        mask = np.zeros(nf, bool)
        rows, cols, vals = [], [], []
        m = ap.shape[ax]
        # interior faces 1 .. m-1: between cell f-1 (L) and cell f (R)
        sl_face = [slice(None)] * 3
        sl_L = [slice(None)] * 3
        sl_R = [slice(None)] * 3
        sl_face[ax] = slice(1, m)
        sl_L[ax] = slice(0, m - 1)
        sl_R[ax] = slice(1, m)
        f = fid[tuple(sl_face)].ravel()
        L = ids[tuple(sl_L)].ravel()
        R = ids[tuple(sl_R)].ravel()
        beta[tuple(sl_face)] = 0.5 * (ap[tuple(sl_L)] + ap[tuple(sl_R)])
        mask[tuple(sl_face)] = True
        rows += [f, f]
        cols += [R, L]
        vals += [np.ones(f.size), -np.ones(f.size)]
        # boundary faces 0 (low side) and m (high side)
        for side, fidx, cidx, sign in ((2 * a, 0, 0, +1.0), (2 * a + 1, m, m - 1, -1.0)):
            if not open_sides[side]:
                continue
            sf = [slice(None)] * 3
            sc = [slice(None)] * 3
            sf[ax] = fidx
            sc[ax] = cidx
            fb = fid[tuple(sf)].ravel()
            cb = ids[tuple(sc)].ravel()
            beta[tuple(sf)] = ap[tuple(sc)]
            mask[tuple(sf)] = True
            # low face: p_R - p_L = p_c - 0; high face: 0 - p_c
            rows.append(fb)
            cols.append(cb)
            vals.append(np.full(fb.size, sign))
        G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nfaces, n))
        out.append((G, beta.ravel(), mask.ravel()))
    return out


def operator(shape, alpha_p, open_sides):
    """A = sum_a G_a^T diag(beta_a) G_a (symmetric; positive definite with an
    open side)."""
    ops = face_operator(shape, alpha_p, open_sides)
    A = None
    for G, beta, _ in ops:
        term = (G.T @ sp.diags(beta) @ G).tocsr()
        A = term if A is None else A + term
    return A.tocsr(), ops


def weighted_divergence(shape, h, ops, faces):
    """div(alpha_f' f) per cell from face values f = (fu, fv, fw): the net
    outward flux of beta f over the cell's faces divided by h (solid faces
    carry no flux)."""
    d = 0.0
    for (G, beta, mask), f in zip(ops, faces):
        d = d - (G.T @ (np.where(mask, beta, 0.0) * np.asarray(f, np.float64)))
    return d / h


def face_gradient(ops, p, h):
    """(p_R - p_L) / h on every face of the three grids (0 on solid faces)."""
    return [(G @ np.asarray(p, np.float64)) / h for G, _, _ in ops]


def rhs_velocity(shape, h, dt, rho0, ops, u, v, w):
    """Right-hand side of A p1 = -(rho0 h^2 / dt) div(alpha_f' v*)."""
    return -(rho0 * h * h / dt) * weighted_divergence(shape, h, ops, (u, v, w))


def rhs_density(h, dt, rho0, alpha_p, alpha_star, ratio_min=0.5, ratio_max=1.5):
    """Right-hand side of A p2 = -(rho0 h^2 / dt^2) alpha' (1 - clamp(alpha*/alpha'))."""
    ap = np.asarray(alpha_p, np.float64)
    ratio = np.clip(np.asarray(alpha_star, np.float64) / ap, ratio_min, ratio_max)
    return -(rho0 * h * h / (dt * dt)) * ap * (1.0 - ratio)


def solve(A, b):
    """Direct sparse solve (SuperLU) in FP64."""
    if not np.any(b):
        return np.zeros_like(b)
    return spla.spsolve(A.tocsc(), b)


def project(shape, h, alpha_s, alpha_star, u, v, w, dt, rho0, open_sides=(0, 0, 0, 0, 0, 1),
            alpha_s_max=0.740, ratio_min=0.5, ratio_max=1.5):
    """Both projections.  Returns a dict with alpha_p, p1, p2, the projected
    face velocities (u, v, w), the face displacements (dxu, dxv, dxw), the
    operator A, the two right-hand sides and the face operators."""
    if not any(open_sides):
        raise ValueError("at least one side must be open (Dirichlet p = 0)")
    ap = target_fraction(alpha_s, alpha_s_max)
    A, ops = operator(shape, ap, open_sides)
    b1 = rhs_velocity(shape, h, dt, rho0, ops, u, v, w)
    b2 = rhs_density(h, dt, rho0, ap, alpha_star, ratio_min, ratio_max)
    p1 = solve(A, b1)
    p2 = solve(A, b2)
    g1 = face_gradient(ops, p1, h)
    g2 = face_gradient(ops, p2, h)
    vel = []
    disp = []
    for (G, beta, mask), f, a, b in zip(ops, (u, v, w), g1, g2):
        vel.append(np.where(mask, np.asarray(f, np.float64) - (dt / rho0) * a, 0.0))
        disp.append(np.where(mask, np.clip(-(dt * dt / rho0) * b, -h, h), 0.0))
    return {"alpha_p": ap, "A": A, "ops": ops, "b1": b1, "b2": b2, "p1": p1, "p2": p2,
            "u": vel[0], "v": vel[1], "w": vel[2], "dxu": disp[0], "dxv": disp[1], "dxw": disp[2]}
