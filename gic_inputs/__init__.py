"""Seeded synthetic inputs for the granule-grid coupling substep.

This module is shared by the tests, the benchmark and the smoke check. It
holds NONE of the method's arithmetic: it only builds granule packings, fluid
fields and parameter sets, and encodes granule positions in the canonical
input format that both the CPU oracle and the CUDA library read exactly.

Canonical input format (every field is exactly representable in FP32, so the
FP64 oracle and the FP32 GPU path start from identical numbers):

* ``cell``  int32 [N, 3]  contact-cell coordinates (cx, cy, cz)
* ``q``     uint32 [N, 3] offset inside the contact cell, as a 30-bit
  fixed-point fraction: x = origin + (cell + q / 2**30) * h_c
* ``r``     float32 [N]   radius
* ``v``     float32 [N, 3] velocity
* fluid fields on the MAC grid, float32, x-fastest:
  ``u`` (nx+1, ny, nz) on x-faces, ``vf`` (nx, ny+1, nz), ``wf`` (nx, ny, nz+1),
  ``p`` and ``alpha_f`` at cell centres.

Random numbers come from numpy's Philox counter-based generator keyed by
(config seed, stream id), so every input is a pure function of its seed.

Recipes follow the workload descriptions of the five configurations
(plain 8k FP64 substep, 1M dam-break column, 8M polydisperse bed, 100k
differentiable window, 16M scale sweep) plus small parity cases with real
contacts.
"""
from __future__ import annotations

import dataclasses
import functools
import math
from typing import Optional

import numpy as np

FRAC_BITS = 30
FRAC_ONE = 1 << FRAC_BITS
# offsets closer than this (in 2**-30 cell units) to a contact-cell face are
# nudged inwards so that floor() of the FP64 absolute position is unambiguous
FRAC_GUARD = 1 << 10

STREAM_POS, STREAM_RAD, STREAM_VEL, STREAM_FLUID, STREAM_TARGET, STREAM_MISC = range(6)


def rng(seed: int, stream: int) -> np.random.Generator:
    """Counter-based Philox stream keyed by (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=np.array([seed, stream], dtype=np.uint64)))


@dataclasses.dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    origin: tuple = (0.0, 0.0, 0.0)
    k_contact: int = 1

    @property
    def h_c(self) -> float:
        return self.dx / self.k_contact

    @property
    def nc(self) -> tuple:
        return (self.nx * self.k_contact, self.ny * self.k_contact, self.nz * self.k_contact)

    @property
    def extent(self) -> np.ndarray:
        return np.array([self.nx, self.ny, self.nz], dtype=np.float64) * self.dx


@dataclasses.dataclass
class Params:
    rho_s: float = 2650.0
    rho_f: float = 1000.0
    k_n: float = 1.0e5
    zeta: float = 0.3
    kt_over_cn: float = 1.0
    mu_fric: float = 0.5
    c_drag: float = 0.22
    g: tuple = (0.0, 0.0, -9.8)
    dt_sub: float = 1.0e-5
    dt_fluid: float = 1.0e-4
    virtual_mass: int = 1
    walls: int = 1
    # concentration-gradient / capillary pair force (Sec. 5.4); sigma = 0 leaves it out
    sigma: float = 0.0           # surface tension coefficient (the paper's scenes: 0.07 N/m)
    bridge_frac: float = 1.0e-4  # liquid-bridge volume as a fraction of the granule volume (0.01%)
    moisture: float = 0.0        # water ratio held by every granule
    moisture_peak: float = 0.3   # moisture ratio where the capillary factor peaks


@dataclasses.dataclass
class Problem:
    name: str
    grid: Grid
    params: Params
    K: int
    cell: np.ndarray
    q: np.ndarray
    r: np.ndarray
    v: np.ndarray
    u: np.ndarray
    vf: np.ndarray
    wf: np.ndarray
    p: np.ndarray
    alpha_f: np.ndarray
    target: Optional[np.ndarray] = None
    note: str = ""

    @property
    def n(self) -> int:
        return int(self.r.shape[0])

    def positions(self) -> np.ndarray:
        """FP64 absolute positions decoded from the canonical encoding."""
        return decode_positions(self.cell, self.q, self.grid)


# --------------------------------------------------------------------------
# position encoding
# --------------------------------------------------------------------------

def contact_k(dx: float, r_max: float) -> int:
    """Contact cells per MAC cell: the largest k with dx / k >= 2 r_max."""
    return max(1, int(math.floor(dx / (2.0 * r_max) * (1.0 - 1e-12))))


def encode_positions(x: np.ndarray, grid: Grid):
    """Absolute FP64 positions -> (cell int32[N,3], q uint32[N,3]).

    The fraction is rounded to 30 bits and kept FRAC_GUARD away from the
    cell faces."""
    o = np.asarray(grid.origin, dtype=np.float64)
    s = (np.asarray(x, dtype=np.float64) - o) / grid.h_c
    c = np.floor(s).astype(np.int64)
    nc = np.array(grid.nc, dtype=np.int64)
    c = np.clip(c, 0, nc - 1)
    f = s - c
    q = np.rint(f * FRAC_ONE).astype(np.int64)
    q = np.clip(q, FRAC_GUARD, FRAC_ONE - FRAC_GUARD)
    return c.astype(np.int32), q.astype(np.uint32)


def decode_positions(cell: np.ndarray, q: np.ndarray, grid: Grid) -> np.ndarray:
    o = np.asarray(grid.origin, dtype=np.float64)
    return o + (cell.astype(np.float64) + q.astype(np.float64) / FRAC_ONE) * grid.h_c


# --------------------------------------------------------------------------
# packings
# --------------------------------------------------------------------------

def cubic_lattice(counts, spacing, start):
    ii, jj, kk = np.meshgrid(np.arange(counts[0]), np.arange(counts[1]), np.arange(counts[2]), indexing="ij")
    pts = np.stack([ii.ravel(order="F"), jj.ravel(order="F"), kk.ravel(order="F")], axis=1).astype(np.float64)
    return np.asarray(start, dtype=np.float64) + pts * spacing


def fcc_fill(lo, hi, nn, n_max=None):
    """FCC lattice points with nearest-neighbour distance nn inside the box
    [lo, hi], filled layer by layer upwards in z (x fastest) until n_max
    (all sites of the box when n_max is None)."""
    a = nn * math.sqrt(2.0)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) * a
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    ncell = np.floor((hi - lo) / a + 1.0).astype(int) + 1
    out = []
    total = 0
    for kz in range(ncell[2] * 2 + 2):
        # atomic layers: even -> basis z=0, odd -> basis z=a/2
        z_layer = lo[2] + (kz // 2) * a + (kz % 2) * 0.5 * a
        if z_layer > hi[2]:
            break
        sel = basis[np.isclose(basis[:, 2], (kz % 2) * 0.5 * a)]
        ii, jj = np.meshgrid(np.arange(ncell[0]), np.arange(ncell[1]), indexing="ij")
        base = np.stack([ii.ravel(order="F") * a, jj.ravel(order="F") * a], axis=1)
        for b in sel:
            pts = np.empty((base.shape[0], 3))
            pts[:, 0] = lo[0] + base[:, 0] + b[0]
            pts[:, 1] = lo[1] + base[:, 1] + b[1]
            pts[:, 2] = z_layer
            keep = (pts[:, 0] <= hi[0]) & (pts[:, 1] <= hi[1])
            pts = pts[keep]
            # x fastest inside the layer
            order = np.lexsort((pts[:, 0], pts[:, 1]))
            out.append(pts[order])
            total += pts.shape[0]
        if n_max is not None and total >= n_max:
            break
    pts = np.concatenate(out, axis=0)
    # stable order: by z, then y, then x
    order = np.lexsort((pts[:, 0], pts[:, 1], pts[:, 2]))
    pts = pts[order]
    if n_max is None:
        return pts
    if pts.shape[0] < n_max:
        raise ValueError(f"box holds only {pts.shape[0]} FCC sites, wanted {n_max}")
    return pts[:n_max]


# --------------------------------------------------------------------------
# neighbour pairs (input validation only: the contact-band guard)
# --------------------------------------------------------------------------

def pairs_within(x: np.ndarray, r: np.ndarray, extra: float, chunk: int = 1 << 21):
    """All pairs i<j with |x_i - x_j| < r_i + r_j + extra.

    Returns (i, j, d). Binned search with bins of width 2 r_max + extra."""
    n = x.shape[0]
    if n < 2:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0)
    hb = 2.0 * float(r.max()) + extra
    lo = x.min(axis=0)
    b = np.floor((x - lo) / hb).astype(np.int64)
    nb = b.max(axis=0) + 3
    b += 1
    lin = b[:, 0] + nb[0] * (b[:, 1] + nb[1] * b[:, 2])
    order = np.argsort(lin, kind="stable")
    lin_s = lin[order]
    ub, first, cnt = np.unique(lin_s, return_index=True, return_counts=True)
    I, J, D = [], [], []
    offs = [(a, bb, c) for c in (-1, 0, 1) for bb in (-1, 0, 1) for a in (-1, 0, 1)]
    for (ox, oy, oz) in offs:
        q = lin + ox + nb[0] * (oy + nb[1] * oz)
        pos = np.searchsorted(ub, q)
        pos = np.minimum(pos, ub.shape[0] - 1)
        hit = ub[pos] == q
        idx = np.nonzero(hit)[0]
        st = first[pos[idx]]
        ct = cnt[pos[idx]]
        for s0 in range(0, idx.shape[0], chunk):
            ii = idx[s0:s0 + chunk]
            ss = st[s0:s0 + chunk]
            cc = ct[s0:s0 + chunk]
            tot = int(cc.sum())
            if tot == 0:
                continue
            rep_i = np.repeat(ii, cc)
            base = np.repeat(ss - np.cumsum(cc) + cc, cc)
            kk = base + np.arange(tot)
            jj = order[kk]
            m = rep_i < jj
            rep_i = rep_i[m]
            jj = jj[m]
            d = np.linalg.norm(x[rep_i] - x[jj], axis=1)
            keep = d < r[rep_i] + r[jj] + extra
            I.append(rep_i[keep])
            J.append(jj[keep])
            D.append(d[keep])
    if not I:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0)
    return np.concatenate(I), np.concatenate(J), np.concatenate(D)


def band_pairs(x, r, band):
    """Pairs whose gap |d - (r_i + r_j)| is below `band` (ambiguous contact predicate)."""
    i, j, d = pairs_within(x, r, band)
    m = np.abs(d - (r[i] + r[j])) < band
    return i[m], j[m]


def wall_band(x, r, grid: Grid, band):
    o = np.asarray(grid.origin)
    hi = o + grid.extent
    gap_lo = x - o
    gap_hi = hi - x
    return np.nonzero(((np.abs(gap_lo - r[:, None]) < band) | (np.abs(gap_hi - r[:, None]) < band)).any(axis=1))[0]


def _clear_band(x, r, grid, gen, jitter, band, max_iter=50):
    """Re-jitter granules taking part in an ambiguous contact (pair or wall)."""
    x0 = x.copy()
    for _ in range(max_iter):
        cell, q = encode_positions(x, grid)
        xe = decode_positions(cell, q, grid)
        i, j = band_pairs(xe, r.astype(np.float64), band)
        w = wall_band(xe, r.astype(np.float64), grid, band)
        bad = np.unique(np.concatenate([i, j, w]))
        if bad.size == 0:
            return x
        x[bad] = x0[bad] + gen.uniform(-jitter, jitter, size=(bad.size, 3))
    raise RuntimeError("could not clear the contact band")


# --------------------------------------------------------------------------
# fluid fields
# --------------------------------------------------------------------------

def face_coords(grid: Grid, comp: int):
    """Sample coordinates of MAC component `comp` (0=u,1=v,2=w) as 1-D axes."""
    n = [grid.nx, grid.ny, grid.nz]
    axes = []
    for a in range(3):
        if a == comp:
            axes.append(grid.origin[a] + np.arange(n[a] + 1) * grid.dx)
        else:
            axes.append(grid.origin[a] + (np.arange(n[a]) + 0.5) * grid.dx)
    return axes


def centre_coords(grid: Grid):
    n = [grid.nx, grid.ny, grid.nz]
    return [grid.origin[a] + (np.arange(n[a]) + 0.5) * grid.dx for a in range(3)]


def _flat(arr3):
    """(X, Y, Z) array -> x-fastest flat float32."""
    return np.ascontiguousarray(np.transpose(arr3, (2, 1, 0))).ravel().astype(np.float32)


def zero_wall_normal(u, vf, wf, grid):
    """Solid walls: the wall-normal velocity on boundary faces is zero."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    u3 = u.reshape(nz, ny, nx + 1)
    u3[:, :, 0] = 0
    u3[:, :, nx] = 0
    v3 = vf.reshape(nz, ny + 1, nx)
    v3[:, 0, :] = 0
    v3[:, ny, :] = 0
    w3 = wf.reshape(nz + 1, ny, nx)
    w3[0] = 0
    w3[nz] = 0
    return u, vf, wf


def uniform_noise_velocity(grid: Grid, gen, amp):
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    u = gen.uniform(-amp, amp, size=(nx + 1) * ny * nz).astype(np.float32)
    vf = gen.uniform(-amp, amp, size=nx * (ny + 1) * nz).astype(np.float32)
    wf = gen.uniform(-amp, amp, size=nx * ny * (nz + 1)).astype(np.float32)
    return zero_wall_normal(u, vf, wf, grid)


def fourier_velocity(grid: Grid, gen, n_modes, kmax, scale_to, scale_kind="max"):
    """Divergence-free sum of random Fourier modes a_m sin(k_m . x + phi_m),
    a_m orthogonal to k_m, k_m = 2 pi (integer vector in +-{1..kmax}) / L.

    Each component is evaluated on its MAC samples with one inverse FFT (the
    modes are periodic on the box, the half-cell staggering is a phase
    shift); scaled so that the max (or RMS) speed over the cell centres
    equals `scale_to`.  Requires a cubic grid."""
    import scipy.fft as sfft

    N = grid.nx
    if not (grid.ny == N and grid.nz == N):
        raise ValueError("fourier_velocity needs a cubic grid")
    nvec = gen.integers(1, kmax + 1, size=(n_modes, 3)) * gen.choice([-1, 1], size=(n_modes, 3))
    ph = gen.uniform(0, 2 * np.pi, size=n_modes)
    amps = np.empty((n_modes, 3))
    for m in range(n_modes):
        a = gen.normal(size=3)
        kh = nvec[m] / np.linalg.norm(nvec[m])
        a -= a.dot(kh) * kh
        amps[m] = a / np.linalg.norm(a)

    def evaluate(comp, shift):
        # samples at (i + shift_a) dx; field = Im(sum_m c_m exp(2 pi i n_m . x / L))
        Y = np.zeros((N, N, N), dtype=np.complex128)
        for m in range(n_modes):
            c = amps[m, comp] * np.exp(1j * ph[m]) * np.exp(2j * np.pi * np.dot(nvec[m], shift) / N)
            Y[tuple(int(v) % N for v in nvec[m])] += c * N ** 3
        X = sfft.ifftn(Y, workers=-1).imag  # [i, j, k] = x, y, z
        return X

    centre = np.array([0.5, 0.5, 0.5])
    speed2 = sum(evaluate(c, centre) ** 2 for c in range(3))
    s_ = scale_to / (np.sqrt(speed2.max()) if scale_kind == "max" else np.sqrt(speed2.mean()))
    out = []
    for comp in range(3):
        shift = centre.copy()
        shift[comp] = 0.0
        X = evaluate(comp, shift) * s_
        # the face axis has N + 1 samples; the last equals the first (periodic modes)
        X = np.concatenate([X, np.take(X, [0], axis=comp)], axis=comp)
        out.append(_flat(X))
    u, vf, wf = out
    return zero_wall_normal(u, vf, wf, grid)


def shear_velocity(grid: Grid, rate):
    """u_x = rate * z on x-faces, v = w = 0."""
    ax = face_coords(grid, 0)
    u3 = np.broadcast_to(rate * ax[2][None, None, :], (ax[0].size, ax[1].size, ax[2].size))
    u = _flat(u3)
    vf = np.zeros(grid.nx * (grid.ny + 1) * grid.nz, np.float32)
    wf = np.zeros(grid.nx * grid.ny * (grid.nz + 1), np.float32)
    return zero_wall_normal(u, vf, wf, grid)


def hydrostatic_pressure(grid: Grid, rho_f, g=9.8):
    """p = rho_f g (H - z) at cell centres, free surface at the top of the box."""
    cc = centre_coords(grid)
    H = grid.origin[2] + grid.nz * grid.dx
    p3 = np.broadcast_to(rho_f * g * (H - cc[2])[None, None, :], (grid.nx, grid.ny, grid.nz))
    return _flat(p3)


def box_fluid_fraction(grid: Grid, lo, hi, phi):
    """Given fluid fraction: 1 - phi in cells whose centre lies inside the
    packing's bounding box [lo, hi], 1 elsewhere."""
    cc = centre_coords(grid)
    inside = [(cc[a] >= lo[a]) & (cc[a] <= hi[a]) for a in range(3)]
    m = inside[0][:, None, None] & inside[1][None, :, None] & inside[2][None, None, :]
    return _flat(np.where(m, 1.0 - phi, 1.0))


# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------

def _finish(name, grid, params, K, x, r, v, u, vf, wf, p, af, target=None, note=""):
    cell, q = encode_positions(x, grid)
    return Problem(name=name, grid=grid, params=params, K=K, cell=cell, q=q,
                   r=np.asarray(r, np.float32), v=np.asarray(v, np.float32),
                   u=u, vf=vf, wf=wf, p=p, alpha_f=af, target=target, note=note)


def plain_fp64(seed=1, n_side=20):
    """8,000 monodisperse granules (r = 0.004) on a jittered simple-cubic
    lattice (spacing 2.2 r, jitter U[-0.05 r, 0.05 r]^3) in the lower half of
    a unit cube with a 32^3 MAC grid; fluid velocity iid U[-0.1, 0.1] on the
    faces, hydrostatic pressure, 10 substeps of 1e-5 s."""
    r0 = 0.004
    grid = Grid(32, 32, 32, 1.0 / 32, k_contact=contact_k(1.0 / 32, r0))
    spacing = 2.2 * r0
    span = (n_side - 1) * spacing
    start = np.array([0.5 - span / 2, 0.5 - span / 2, 1.1 * r0])
    x = cubic_lattice((n_side,) * 3, spacing, start)
    gen = rng(seed, STREAM_POS)
    x = x + gen.uniform(-0.05 * r0, 0.05 * r0, size=x.shape)
    n = x.shape[0]
    r = np.full(n, r0, np.float32)
    v = np.zeros((n, 3), np.float32)
    u, vf, wf = uniform_noise_velocity(grid, rng(seed, STREAM_FLUID), 0.1)
    params = Params(dt_sub=1e-5, dt_fluid=10 * 1e-5)
    p = hydrostatic_pressure(grid, params.rho_f)
    phi = (4.0 / 3.0 * np.pi * r0 ** 3) / spacing ** 3
    af = box_fluid_fraction(grid, x.min(0) - r0, x.max(0) + r0, phi)
    return _finish("plain_fp64_8k", grid, params, 10, x, r, v, u, vf, wf, p, af)


def dam_break(seed=2, n=1_000_000):
    """1,000,000 granules (r = 0.0015) on an FCC lattice at volume fraction
    0.55 (nearest neighbour 2.208 r, jitter 0.05 r) filling the 0.3 x 1.0
    footprint of a corner column upwards from the floor; 128^3 grid; smooth
    divergence-free noise (8 modes, max speed 0.5 m/s); 100 substeps of 2e-5 s.

    The column 0.3 x 1.0 x 0.5 at volume fraction 0.55 would hold about
    5.8M granules, more than the 1M asked for, so the column is filled from
    the floor until 1M granules are placed (height about 0.086)."""
    r0 = 0.0015
    dx = 1.0 / 128
    grid = Grid(128, 128, 128, dx, k_contact=contact_k(dx, r0))
    lo = np.array([1.1 * r0, 1.1 * r0, 1.1 * r0])
    hi = np.array([0.3 - 1.1 * r0, 1.0 - 1.1 * r0, 0.5])
    x = fcc_fill(lo, hi, 2.208 * r0, n)
    gen = rng(seed, STREAM_POS)
    x = x + gen.uniform(-0.05 * r0, 0.05 * r0, size=x.shape)
    r = np.full(n, r0, np.float32)
    v = np.zeros((n, 3), np.float32)
    u, vf, wf = fourier_velocity(grid, rng(seed, STREAM_FLUID), 8, 4, 0.5, "max")
    params = Params(dt_sub=2e-5, dt_fluid=100 * 2e-5)
    p = hydrostatic_pressure(grid, params.rho_f)
    af = box_fluid_fraction(grid, x.min(0) - r0, x.max(0) + r0, 0.55)
    return _finish("dam_break_1m", grid, params, 100, x, r, v, u, vf, wf, p, af)


def differentiable_window(seed=4, n=100_000, r0=0.002, grid_n=64):
    """100,000 granules (r = 0.002) in a loose packing at volume fraction 0.3:
    a simple-cubic lattice of spacing (V/0.3)^(1/3) with uniform jitter
    +-0.2 r per coordinate, in a cube centred in x, y and resting on the
    floor; initial velocities iid U[-0.01, 0.01]; 64^3 grid with smooth noise
    (amplitude 0.1 m/s); 50 substeps of 2e-5 s; target cloud = initial
    positions + N(0, (0.5 r)^2)."""
    dx = 1.0 / grid_n
    grid = Grid(grid_n, grid_n, grid_n, dx, k_contact=contact_k(dx, r0))
    vol = 4.0 / 3.0 * np.pi * r0 ** 3
    spacing = (vol / 0.3) ** (1.0 / 3.0)
    side = int(math.ceil(n ** (1.0 / 3.0)))
    x = cubic_lattice((side, side, side), spacing, (0.0, 0.0, 0.0))[:n]
    span = (side - 1) * spacing
    x[:, 0] += 0.5 - span / 2
    x[:, 1] += 0.5 - span / 2
    x[:, 2] += 1.25 * r0
    gen = rng(seed, STREAM_POS)
    x = x + gen.uniform(-0.2 * r0, 0.2 * r0, size=x.shape)
    r = np.full(n, r0, np.float32)
    v = rng(seed, STREAM_VEL).uniform(-0.01, 0.01, size=(n, 3)).astype(np.float32)
    u, vf, wf = fourier_velocity(grid, rng(seed, STREAM_FLUID), 8, 4, 0.1, "max")
    params = Params(dt_sub=2e-5, dt_fluid=50 * 2e-5)
    p = hydrostatic_pressure(grid, params.rho_f)
    af = box_fluid_fraction(grid, x.min(0) - r0, x.max(0) + r0, 0.3)
    prob = _finish("diff_window_100k", grid, params, 50, x, r, v, u, vf, wf, p, af)
    xe = prob.positions()
    prob.target = xe + rng(seed, STREAM_TARGET).normal(0.0, 0.5 * r0, size=xe.shape)
    return prob


def dense_block(seed=11, n_side=(8, 8, 8), r0=0.004, nn_factor=1.98, jitter=0.01, grid_n=32,
                poly=0.0, fluid_amp=0.1, K=10, dt=1e-5):
    """Parity case with real contacts: an FCC block whose nearest-neighbour
    distance is `nn_factor` * r (so neighbours overlap by about (2 - nn_factor)
    r, i.e. 2% of r by default), jittered, standing on the floor next to the x = 0 wall, so that pair
    forces, wall forces, Coulomb capping and the dashpot all take part.

    Optional polydispersity: radii scaled by exp(poly * N(0,1)), clipped to
    [0.5, 2] x r0 then capped so the contact cell still holds 2 r_max."""
    nside = np.array(n_side)
    nn = nn_factor * r0           # nearest-neighbour distance; overlap (2 - nn_factor) r
    a = nn * math.sqrt(2.0)
    lo = np.array([0.985 * r0, 0.25, 0.985 * r0])
    hi = lo + (nside - 1) * a + 0.75 * a
    x = fcc_fill(lo, hi, nn, None)
    gen = rng(seed, STREAM_POS)
    n = x.shape[0]
    if poly > 0:
        rr = r0 * np.exp(poly * rng(seed, STREAM_RAD).normal(size=n))
        r = np.clip(rr, 0.5 * r0, 1.2 * r0)
    else:
        r = np.full(n, r0)
    r = r.astype(np.float32)
    dxg = 1.0 / grid_n
    grid = Grid(grid_n, grid_n, grid_n, dxg, k_contact=contact_k(dxg, float(r.max())))
    x = x + gen.uniform(-jitter * r0, jitter * r0, size=x.shape)
    x = _clear_band(x, r.astype(np.float64), grid, gen, jitter * r0, 1e-5 * float(r.min()))
    v = rng(seed, STREAM_VEL).uniform(-0.05, 0.05, size=(n, 3)).astype(np.float32)
    u, vf, wf = uniform_noise_velocity(grid, rng(seed, STREAM_FLUID), fluid_amp)
    params = Params(dt_sub=dt, dt_fluid=K * dt)
    p = hydrostatic_pressure(grid, params.rho_f)
    af = box_fluid_fraction(grid, x.min(0) - r0, x.max(0) + r0, 0.7)
    return _finish("dense_block", grid, params, K, x, r, v, u, vf, wf, p, af)


def wet_block(seed=12, n_side=(5, 5, 5), r0=0.004, nn_factor=2.02, jitter=0.01, grid_n=32, sigma=0.07, K=10,
              dt=1e-5, alpha_lo=0.15, alpha_hi=0.45):
    """Parity case for the capillary pair force: the FCC block of dense_block
    with its nearest neighbours 2% of r apart (jittered by 1% of r, so most
    pairs sit in the liquid-bridge range, a few touch), surface tension 0.07
    N/m, and a fluid fraction that rises linearly in z across the block from
    alpha_lo to alpha_hi (1 outside it), so that the moisture ratio of the
    granules varies on both sides of the capillary factor's peak."""
    prob = dense_block(seed=seed, n_side=n_side, r0=r0, nn_factor=nn_factor, jitter=jitter, grid_n=grid_n, K=K, dt=dt)
    grid = prob.grid
    x = prob.positions()
    lo, hi = x.min(0) - r0, x.max(0) + r0
    cc = centre_coords(grid)
    t = np.clip((cc[2] - lo[2]) / (hi[2] - lo[2]), 0.0, 1.0)
    inside = [(cc[a] >= lo[a]) & (cc[a] <= hi[a]) for a in range(3)]
    m = inside[0][:, None, None] & inside[1][None, :, None] & inside[2][None, None, :]
    ramp = np.broadcast_to((alpha_lo + (alpha_hi - alpha_lo) * t)[None, None, :], m.shape)
    af = _flat(np.where(m, ramp, 1.0))
    params = dataclasses.replace(prob.params, sigma=sigma)
    return dataclasses.replace(prob, name="wet_block", params=params, alpha_f=af)


def random_cloud(seed=21, n=2000, r0=0.004, grid_n=16, fluid_amp=0.2, K=10, dt=1e-5, phi=0.35):
    """Small random cloud with overlaps: a simple-cubic lattice at volume
    fraction `phi` with uniform jitter of +-0.35 lattice spacings, after which
    one granule of every pair closer than 1.9 r is dropped (overlaps stay
    below 5% of r). The brute-force O(N^2) enumeration is cheap at this size."""
    dxg = 1.0 / grid_n
    grid = Grid(grid_n, grid_n, grid_n, dxg, k_contact=contact_k(dxg, r0))
    gen = rng(seed, STREAM_POS)
    spacing = (4 / 3 * np.pi * r0 ** 3 / phi) ** (1 / 3)
    side = int(math.ceil((1.3 * n) ** (1 / 3)))
    x = cubic_lattice((side, side, side), spacing, (0.3, 0.3, 1.05 * r0 + 0.35 * spacing))
    x = x + gen.uniform(-0.35 * spacing, 0.35 * spacing, size=x.shape)
    r = np.full(x.shape[0], r0)
    while True:
        i, j, d = pairs_within(x, r, 0.0)
        bad = np.unique(i[d < 1.9 * r0])
        if bad.size == 0:
            break
        x = np.delete(x, bad, axis=0)
        r = r[: x.shape[0]]
    x = x[:n]
    n = x.shape[0]
    r = np.full(n, r0, np.float32)
    x = _clear_band(x, r.astype(np.float64), grid, gen, 0.01 * r0, 1e-5 * r0)
    v = rng(seed, STREAM_VEL).uniform(-0.05, 0.05, size=(n, 3)).astype(np.float32)
    u, vf, wf = uniform_noise_velocity(grid, rng(seed, STREAM_FLUID), fluid_amp)
    params = Params(dt_sub=dt, dt_fluid=K * dt)
    p = hydrostatic_pressure(grid, params.rho_f)
    af = box_fluid_fraction(grid, x.min(0) - r0, x.max(0) + r0, 1.0 - phi)
    return _finish("random_cloud", grid, params, K, x, r, v, u, vf, wf, p, af)


def _fcc_neighbour_table():
    """For each FCC basis atom b and each of the 12 nearest-neighbour vectors:
    (cell offset, neighbour basis index), in units of the cubic cell."""
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    dirs = []
    for a in range(3):
        for b in range(a + 1, 3):
            for sa in (-0.5, 0.5):
                for sb in (-0.5, 0.5):
                    d = np.zeros(3)
                    d[a], d[b] = sa, sb
                    dirs.append(d)
    table = np.zeros((4, 12, 4), dtype=np.int64)
    for bi in range(4):
        for k, d in enumerate(dirs):
            q = basis[bi] + d
            cell = np.floor(q + 1e-9).astype(np.int64)
            frac = q - cell
            bj = int(np.argmin(np.abs(basis - frac).sum(1)))
            table[bi, k, :3] = cell
            table[bi, k, 3] = bj
    return basis, table


def _periodic_pairs(pos, reach, L):
    """Index pairs (i < j) closer than `reach` with x, y periodic of period
    L[0], L[1] (z open), and their minimum-image separations."""
    from scipy.spatial import cKDTree

    p = pos.copy()
    p[:, 0] %= L[0]
    p[:, 1] %= L[1]
    z0 = p[:, 2].min()
    p[:, 2] -= z0
    tree = cKDTree(p, boxsize=[L[0], L[1], 2.0 * (p[:, 2].max() + reach) + 1.0])
    P = tree.query_pairs(reach, output_type="ndarray")
    I, J = P[:, 0], P[:, 1]
    d = pos[I] - pos[J]
    d[:, 0] -= np.round(d[:, 0] / L[0]) * L[0]
    d[:, 1] -= np.round(d[:, 1] / L[1]) * L[1]
    return I, J, d


def _settle_tile(pos, rr, L, iters, push, skin, relax, tol):
    """Settle a periodic tile: `iters` rounds of averaged Jacobi overlap
    removal (each overlapping pair split by inverse volume, a granule moves by
    1.5 x the mean of its corrections), each round after a downward shift of
    `push` (decreasing to zero), with the floor at z = r; then up to `relax`
    rounds without the push, until no overlap exceeds `tol`.  Neighbour pairs
    are re-found whenever a granule has moved 0.4 `skin` since the last
    search."""
    m = len(rr)
    w = 1.0 / rr ** 3
    ref = None
    for it in range(iters + relax):
        if ref is None or np.abs(pos - ref).max() > 0.4 * skin:
            I, J, _ = _periodic_pairs(pos, 2 * rr.max() + skin, L)
            ref = pos.copy()
        d = pos[I] - pos[J]
        d[:, 0] -= np.round(d[:, 0] / L[0]) * L[0]
        d[:, 1] -= np.round(d[:, 1] / L[1]) * L[1]
        dist = np.linalg.norm(d, axis=1)
        ov = rr[I] + rr[J] - dist
        k = ov > 0
        if it >= iters and not (ov > tol).any():
            break
        Ik, Jk = I[k], J[k]
        nrm = d[k] / dist[k][:, None] * ov[k][:, None]
        fi = (w[Ik] / (w[Ik] + w[Jk]))[:, None]
        disp = np.zeros_like(pos)
        cnt = np.zeros(m)
        np.add.at(disp, Ik, nrm * fi)
        np.add.at(disp, Jk, -nrm * (1 - fi))
        np.add.at(cnt, Ik, 1)
        np.add.at(cnt, Jk, 1)
        pos += 1.5 * disp / np.maximum(cnt, 1)[:, None]
        if it < iters:
            pos[:, 2] -= push * (1 - it / iters)
        pos[:, 2] = np.maximum(pos[:, 2], rr)
    return pos


@functools.lru_cache(maxsize=2)
def _bed_tile(seed, tile_cells, iters, relax):
    """The settled periodic tile of the polydisperse bed: positions, radii,
    periods and (neighbours, contacts, packing fraction, height)."""
    med = 8e-4
    gen = rng(seed, STREAM_POS)
    a = 2.35 * med * math.sqrt(2.0)
    cx, cy, cz = tile_cells
    basis, _ = _fcc_neighbour_table()
    ii, jj, kk, bb = np.meshgrid(np.arange(cx), np.arange(cy), np.arange(cz), np.arange(4), indexing="ij")
    m = ii.size
    pos = (np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1) + basis[bb.ravel()]) * a
    pos[:, 2] += med
    pos += gen.uniform(-0.02 * med, 0.02 * med, size=pos.shape)
    rr = np.clip(med * np.exp(0.25 * rng(seed, STREAM_RAD).normal(size=m)), 0.5 * med, 2.0 * med)
    L = (cx * a, cy * a)
    pos = _settle_tile(pos, rr, L, iters, 0.004 * med, 0.3 * med, relax, 0.01 * rr.min())
    tol = 0.001 * rr.min()
    for _ in range(50):
        I, J, d = _periodic_pairs(pos, 2 * rr.max(), L)
        excess = rr[I] + rr[J] - np.linalg.norm(d, axis=1) - tol
        bad = excess > 0
        if not bad.any():
            break
        big = np.where(rr[I] >= rr[J], I, J)[bad]
        shrink = np.zeros(m)
        np.maximum.at(shrink, big, excess[bad] * (1 + 1e-9) + 1e-12)
        rr = rr - shrink
    else:
        raise RuntimeError("bed overlap capping did not converge")
    pos[:, 0] %= L[0]
    pos[:, 1] %= L[1]
    I, J, d = _periodic_pairs(pos, 2 * rr.max() + 0.02 * med, L)
    gap = np.linalg.norm(d, axis=1) - rr[I] - rr[J]
    nbr = 2.0 * np.count_nonzero(gap < 0.02 * med) / m
    con = 2.0 * np.count_nonzero(gap < 0) / m
    height = pos[:, 2].max() + med
    phi = (4.0 / 3.0 * np.pi * rr ** 3).sum() / (L[0] * L[1] * height)
    return pos, rr, L, (nbr, con, phi, height)


def polydisperse_bed(seed=3, n=8_000_000, tile_cells=(12, 12, 15), iters=300, relax=1500):
    """8,000,000 granules with lognormal radii (median 8e-4, sigma_log 0.25,
    clipped to [0.5, 2] x median) in a settled-bed layout on a 256^3 grid,
    under the shear flow u_x = 0.8 z; 50 substeps of 1e-5, k_n = 4e3.

    Layout: a tile periodic in x and y, started as an FCC lattice whose
    nearest-neighbour spacing (2.35 x median, jitter 0.02 x median) holds the
    lognormal volumes at a packing fraction near 0.6, settled by `iters`
    rounds of overlap removal under a decreasing downward push and up to
    `relax` more without it (or until no overlap exceeds 1% of the smallest
    radius); where a pair still overlaps by more than 0.1% of the smallest
    radius, the larger granule is shrunk by the excess.  Copies of the tile placed side by side over the
    floor meet with the same neighbour structure; the bed is those copies
    until n granules.  The tile's neighbour statistics (neighbours within
    r_i + r_j + 0.02 x median, contacts, packing fraction) go in `note`."""
    med = 8e-4
    dx = 1.0 / 256
    grid = Grid(256, 256, 256, dx, k_contact=contact_k(dx, 2 * med))
    pos, rr, L, (nbr, con, phi, height) = _bed_tile(seed, tuple(tile_cells), iters, relax)
    m = len(rr)
    # replicate the tile over the floor
    nx_t, ny_t = int(np.floor((1.0 - 4 * med) / L[0])), int(np.floor((1.0 - 4 * med) / L[1]))
    reps = int(math.ceil(n / m))
    if reps > nx_t * ny_t:
        raise ValueError("bed tile does not fit the box floor")
    off = np.array([(2 * med + ix * L[0], 2 * med + iy * L[1], 0.0) for iy in range(ny_t) for ix in range(nx_t)][:reps])
    x = (pos[None, :, :] + off[:, None, :]).reshape(-1, 3)[:n]
    r = np.tile(rr, reps)[:n].astype(np.float32)
    v = np.zeros((n, 3), np.float32)
    u, vf, wf = shear_velocity(grid, 0.8)
    # k_n = 4e3: at dt 1e-5 the explicit spring-dashpot is stable for the
    # smallest pair (omega dt = 0.97 for two r = 0.5 x median granules with
    # their virtual mass); k_n = 1e5 gives omega dt = 4.9 there and the bed
    # blows up within a few substeps
    params = Params(dt_sub=1e-5, dt_fluid=50 * 1e-5, k_n=4e3)
    p = hydrostatic_pressure(grid, params.rho_f)
    af = box_fluid_fraction(grid, x.min(0) - med, x.max(0) + med, 0.6)
    prob = _finish("polydisperse_bed_8m", grid, params, 50, x, r, v, u, vf, wf, p, af)
    prob.note = (f"tile of {m} granules, {reps} copies; radii {r.min() / med:.2f}-{r.max() / med:.2f} x median; "
                 f"{nbr:.2f} neighbours and {con:.2f} contacts per granule; packing {phi:.3f}, height {height:.4f}")
    return prob


def scale_sweep(seed=5, n=16_000_000, grid_n=384):
    """16,000,000 granules (r = 6e-4) on an FCC lattice at volume fraction 0.6
    (nearest neighbour 2.145 r, jitter 0.05 r) as a full-footprint slab from
    the floor (height about 0.024) on a 384^3 grid; 32 divergence-free Fourier
    modes (k in 2 pi {1..8}^3) scaled to an RMS speed of 1 m/s; 20 substeps of
    1e-5.  The jitter leaves a few small initial overlaps."""
    r0 = 6e-4
    dx = 1.0 / grid_n
    grid = Grid(grid_n, grid_n, grid_n, dx, k_contact=contact_k(dx, r0))
    lo = np.array([1.1 * r0, 1.1 * r0, 1.1 * r0])
    hi = np.array([1.0 - 1.1 * r0, 1.0 - 1.1 * r0, 0.5])
    x = fcc_fill(lo, hi, 2.145 * r0, n)
    gen = rng(seed, STREAM_POS)
    x = x + gen.uniform(-0.05 * r0, 0.05 * r0, size=x.shape)
    r = np.full(n, r0, np.float32)
    v = np.zeros((n, 3), np.float32)
    u, vf, wf = fourier_velocity(grid, rng(seed, STREAM_FLUID), 32, 8, 1.0, "rms")
    params = Params(dt_sub=1e-5, dt_fluid=20 * 1e-5)
    p = hydrostatic_pressure(grid, params.rho_f)
    af = box_fluid_fraction(grid, x.min(0) - r0, x.max(0) + r0, 0.6)
    return _finish("scale_sweep_16m", grid, params, 20, x, r, v, u, vf, wf, p, af)


def make(name: str, **kw) -> Problem:
    table = {
        "plain_fp64_8k": plain_fp64,
        "dam_break_1m": dam_break,
        "diff_window_100k": differentiable_window,
        "dense_block": dense_block,
        "wet_block": wet_block,
        "random_cloud": random_cloud,
        "polydisperse_bed_8m": polydisperse_bed,
        "scale_sweep_16m": scale_sweep,
    }
    return table[name](**kw)


# --------------------------------------------------------------------------
# inputs of the pressure projections that consume alpha_s
# --------------------------------------------------------------------------

@dataclasses.dataclass
class ProjectionCase:
    """Cell-centred alpha_s (FP64) and current fluid fraction alpha_f*
    (float32), face velocities v* (float32, x fastest), the fluid step and
    density, and the open sides (-x, +x, -y, +y, -z, +z)."""
    name: str
    shape: tuple
    dx: float
    alpha_s: np.ndarray
    alpha_star: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    dt: float
    rho_f: float
    open_sides: tuple


def projection_case(seed=31, shape=(21, 18, 25), dx=1.0 / 32, dt=2e-3, rho_f=1000.0, amp=0.5,
                    open_sides=(0, 0, 0, 0, 0, 1), pack_max=0.85, name="projection_random"):
    """A sediment-like alpha_s: a smooth bed (a sum of 4 seeded Gaussian bumps
    over a layer in the lower third) up to pack_max, so that the densest-packing
    limit is exceeded in places, plus seeded cell noise; alpha_f* = (1 -
    alpha_s) times a seeded factor in [0.3, 1.8] (beyond the [0.5, 1.5] ratio
    limit in places); face velocities iid U[-amp, amp], zero on solid walls'
    normal faces."""
    nx, ny, nz = shape
    gen = rng(seed, STREAM_MISC)
    c = [(np.arange(m) + 0.5) / m for m in (nx, ny, nz)]
    X, Y, Z = np.meshgrid(c[0], c[1], c[2], indexing="ij")
    bed = np.clip(1.5 - 4.5 * Z, 0.0, 1.0)
    for _ in range(4):
        cx, cy, cz = gen.uniform(0.1, 0.9, 3)
        s = gen.uniform(0.1, 0.3)
        bed = bed + 0.6 * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) / (2 * s * s))
    a_s = np.clip(pack_max * bed / bed.max() + gen.uniform(-0.03, 0.03, size=bed.shape), 0.0, pack_max)
    factor = gen.uniform(0.3, 1.8, size=bed.shape)
    a_star = (1.0 - a_s) * factor
    alpha_s = np.ascontiguousarray(np.transpose(a_s, (2, 1, 0))).ravel().astype(np.float64)
    alpha_star = _flat(a_star)
    grid = Grid(nx, ny, nz, dx)
    u = gen.uniform(-amp, amp, size=(nx + 1) * ny * nz).astype(np.float32)
    vf = gen.uniform(-amp, amp, size=nx * (ny + 1) * nz).astype(np.float32)
    wf = gen.uniform(-amp, amp, size=nx * ny * (nz + 1)).astype(np.float32)
    u3 = u.reshape(nz, ny, nx + 1)
    v3 = vf.reshape(nz, ny + 1, nx)
    w3 = wf.reshape(nz + 1, ny, nx)
    for side, (arr, idx) in enumerate(((u3, (slice(None), slice(None), 0)), (u3, (slice(None), slice(None), nx)),
                                       (v3, (slice(None), 0, slice(None))), (v3, (slice(None), ny, slice(None))),
                                       (w3, (0,)), (w3, (nz,)))):
        if not open_sides[side]:
            arr[idx] = 0
    return ProjectionCase(name=name, shape=tuple(shape), dx=dx, alpha_s=alpha_s, alpha_star=alpha_star, u=u, v=vf,
                          w=wf, dt=dt, rho_f=rho_f, open_sides=tuple(open_sides))
