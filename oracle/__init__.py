"""FP64 CPU oracle for the GIC granule-grid coupling substep (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the smoke check and the
benchmark's CPU-baseline leg, never by the product package.  The C source is
`gic_oracle.c`; it is built with gcc into `oracle/_build/liboracle.so`.

Inputs arrive in the canonical encoding of `gic_inputs` (cell + 30-bit
fraction, FP32 radii / velocities / fluid fields); the oracle converts them
to FP64 itself (exactly) and works with absolute positions.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "gic_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

OUT_OF_DOMAIN = 1
COINCIDENT = 2
NONFINITE = 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no fast-math)."""
    srcs = [s for s in _SRC if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC", *srcs, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("k", C.c_int), ("dx", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double)]


class OrParams(C.Structure):
    _fields_ = [("rho_s", C.c_double), ("rho_f", C.c_double), ("k_n", C.c_double), ("zeta", C.c_double),
                ("kt_over_cn", C.c_double), ("mu", C.c_double), ("c_drag", C.c_double), ("gx", C.c_double),
                ("gy", C.c_double), ("gz", C.c_double), ("dt", C.c_double), ("dt_fluid", C.c_double),
                ("virtual_mass", C.c_int), ("walls", C.c_int), ("sigma", C.c_double), ("bridge_frac", C.c_double),
                ("moisture", C.c_double), ("moisture_peak", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.or_morton.restype = C.c_uint64
        _lib.or_morton.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32]
        _lib.or_cell_table.restype = C.c_int64
        _lib.or_contact_pairs.restype = C.c_int64
        for fn, args in (("or_gamma", [C.c_double, C.c_double]), ("or_moisture_ratio", [C.c_double, C.c_double]),
                         ("or_bridge_force", [C.c_double] * 4), ("or_rupture", [C.c_double] * 2)):
            f = getattr(_lib, fn)
            f.restype = C.c_double
            f.argtypes = args
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def grid_struct(grid) -> OrGrid:
    return OrGrid(grid.nx, grid.ny, grid.nz, grid.k_contact, grid.dx, *[float(o) for o in grid.origin])


def params_struct(P) -> OrParams:
    return OrParams(P.rho_s, P.rho_f, P.k_n, P.zeta, P.kt_over_cn, P.mu_fric, P.c_drag, P.g[0], P.g[1], P.g[2],
                    P.dt_sub, P.dt_fluid, int(P.virtual_mass), int(P.walls), float(getattr(P, "sigma", 0.0)),
                    float(getattr(P, "bridge_frac", 1e-4)), float(getattr(P, "moisture", 0.0)),
                    float(getattr(P, "moisture_peak", 0.3)))


# ---------------------------------------------------------------- encoding

def decode(grid, cell, q) -> np.ndarray:
    n = cell.shape[0]
    x = np.empty((n, 3))
    lib().or_decode(C.byref(grid_struct(grid)), C.c_int64(n), _p(np.ascontiguousarray(cell, np.int32)),
                    _p(np.ascontiguousarray(q, np.uint32)), _p(x))
    return x


# ---------------------------------------------------------------- sort

def cells(grid, x) -> np.ndarray:
    x = _f64(x)
    c = np.empty((x.shape[0], 3), np.int32)
    lib().or_cells(C.byref(grid_struct(grid)), C.c_int64(x.shape[0]), _p(x), _p(c))
    return c


def morton(ix, iy, iz) -> int:
    return int(lib().or_morton(ix, iy, iz))


def sort(c):
    """Stable Morton sort of contact cells c [N,3] -> (perm int64[N], keys uint64[N])."""
    c = np.ascontiguousarray(c, np.int32)
    n = c.shape[0]
    perm = np.empty(n, np.int64)
    keys = np.empty(n, np.uint64)
    lib().or_sort(C.c_int64(n), _p(c), _p(perm), _p(keys))
    return perm, keys


def cell_table(keys):
    keys = np.ascontiguousarray(keys, np.uint64)
    n = keys.shape[0]
    ck = np.empty(max(n, 1), np.uint64)
    st = np.empty(max(n, 1), np.int64)
    ct = np.empty(max(n, 1), np.int64)
    m = lib().or_cell_table(C.c_int64(n), _p(keys), _p(ck), _p(st), _p(ct))
    return ck[:m], st[:m], ct[:m]


# ---------------------------------------------------------------- contact

def contact_pairs(grid, x, r, brute=False):
    x = _f64(x)
    r = _f64(r)
    n = x.shape[0]
    cap = max(16, 16 * n)
    while True:
        pairs = np.empty((cap, 2), np.int64)
        m = lib().or_contact_pairs(C.byref(grid_struct(grid)), C.c_int64(n), _p(x), _p(r), C.c_int(int(brute)),
                                   C.c_int64(cap), _p(pairs))
        if m <= cap:
            return pairs[:m]
        cap = m


def _alpha_field(params, alpha_f):
    if float(getattr(params, "sigma", 0.0)) > 0.0:
        if alpha_f is None:
            raise ValueError("the capillary force (sigma > 0) needs the fluid fraction field alpha_f")
        return _f64(alpha_f)
    return None


def contact(grid, params, x, v, r, brute=False, alpha_f=None):
    """Pair (contact and, with sigma > 0, capillary) and wall forces; alpha_f:
    the cell-centred fluid fraction field (needed with sigma > 0)."""
    x, v, r = _f64(x), _f64(v), _f64(r)
    af = _alpha_field(params, alpha_f)
    n = x.shape[0]
    F = np.empty((n, 3))
    st = C.c_uint32(0)
    lib().or_contact(C.byref(grid_struct(grid)), C.byref(params_struct(params)), C.c_int64(n), _p(x), _p(v), _p(r),
                     None if af is None else _p(af), C.c_int(int(brute)), _p(F), C.byref(st))
    return F, st.value


def gamma(sr, peak):
    """Gamma of Sec. 5.4 (the reading's quadratic Bezier curve)."""
    return lib().or_gamma(float(sr), float(peak))


def moisture_ratio(moisture, af):
    return lib().or_moisture_ratio(float(moisture), float(af))


def bridge_force(sigma, R, Vs, s):
    """F^st of the liquid bridge at separation s (Sec. 5.4)."""
    return lib().or_bridge_force(float(sigma), float(R), float(Vs), float(s))


def rupture(R, Vs):
    """Rupture distance d_r of a bridge of volume Vs between granules of pair radius R."""
    return lib().or_rupture(float(R), float(Vs))


# ---------------------------------------------------------------- G2P

def interp(grid, comp, field, x):
    """Interpolate MAC field `comp` (0,1,2 faces; 3 centres) at points x."""
    f = _f64(field)
    x = _f64(x)
    out = np.empty(x.shape[0])
    lib().or_interp(C.byref(grid_struct(grid)), C.c_int(comp), _p(f), C.c_int64(x.shape[0]), _p(x), _p(out))
    return out


def interp_grad_p(grid, p, x):
    p = _f64(p)
    x = _f64(x)
    out = np.empty((x.shape[0], 3))
    lib().or_interp_grad_p(C.byref(grid_struct(grid)), _p(p), C.c_int64(x.shape[0]), _p(x), _p(out))
    return out


def g2p(grid, params, x, v, r, u, vf, wf, p, af):
    x, v, r = _f64(x), _f64(v), _f64(r)
    u, vf, wf, p, af = _f64(u), _f64(vf), _f64(wf), _f64(p), _f64(af)
    n = x.shape[0]
    F_fl = np.empty((n, 3))
    a_f = np.empty((n, 3))
    afp = np.empty(n)
    lib().or_g2p(C.byref(grid_struct(grid)), C.byref(params_struct(params)), C.c_int64(n), _p(x), _p(v), _p(r),
                 _p(u), _p(vf), _p(wf), _p(p), _p(af), _p(F_fl), _p(a_f), _p(afp))
    return F_fl, a_f, afp


# ---------------------------------------------------------------- integrate

def integrate(grid, params, x, v, r, F_c, F_fl, a_f):
    x, v, r, F_c, F_fl, a_f = map(_f64, (x, v, r, F_c, F_fl, a_f))
    n = x.shape[0]
    xn = np.empty((n, 3))
    vn = np.empty((n, 3))
    fex = np.empty((n, 3))
    st = C.c_uint32(0)
    lib().or_integrate(C.byref(grid_struct(grid)), C.byref(params_struct(params)), C.c_int64(n), _p(x), _p(v), _p(r),
                       _p(F_c), _p(F_fl), _p(a_f), _p(xn), _p(vn), _p(fex), C.byref(st))
    return xn, vn, fex, st.value


# ---------------------------------------------------------------- P2G

def p2g(grid, params, x_old, x_new, r, f_ex, Fs=None):
    x_old, x_new, r, f_ex = map(_f64, (x_old, x_new, r, f_ex))
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    alpha = np.empty(nx * ny * nz)
    if Fs is None:
        Fs = (np.zeros((nx + 1) * ny * nz), np.zeros(nx * (ny + 1) * nz), np.zeros(nx * ny * (nz + 1)))
    sums = np.zeros(2)
    lib().or_p2g(C.byref(grid_struct(grid)), C.byref(params_struct(params)), C.c_int64(x_old.shape[0]), _p(x_old),
                 _p(x_new), _p(r), _p(f_ex), _p(alpha), _p(Fs[0]), _p(Fs[1]), _p(Fs[2]), _p(sums))
    return alpha, Fs, sums


# ---------------------------------------------------------------- K substeps

def run(prob, K=None, brute=False, x=None, v=None, params=None):
    """Run K substeps of the oracle on a gic_inputs.Problem.

    Returns dict(x, v, alpha_s, Fs=(u, v, w), sums, status)."""
    grid = prob.grid
    P = params if params is not None else prob.params
    K = prob.K if K is None else K
    x = decode(grid, prob.cell, prob.q) if x is None else _f64(x).copy()
    v = _f64(prob.v).copy() if v is None else _f64(v).copy()
    r = _f64(prob.r)
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    alpha = np.zeros(nx * ny * nz)
    Fs = (np.zeros((nx + 1) * ny * nz), np.zeros(nx * (ny + 1) * nz), np.zeros(nx * ny * (nz + 1)))
    sums = np.zeros(2)
    st = C.c_uint32(0)
    fl = [_f64(a) for a in (prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)]
    lib().or_run(C.byref(grid_struct(grid)), C.byref(params_struct(P)), C.c_int64(x.shape[0]), C.c_int(K), _p(x),
                 _p(v), _p(r), *[_p(a) for a in fl], _p(alpha), _p(Fs[0]), _p(Fs[1]), _p(Fs[2]), _p(sums),
                 C.c_int(int(brute)), C.byref(st))
    return dict(x=x, v=v, alpha_s=alpha, Fs=Fs, sums=sums, status=st.value)


# ---------------------------------------------------------------- adjoints

def contact_adj(grid, params, x, v, r, gF, brute=False, alpha_f=None):
    """(gx, gv, g_mu) of <gF, contact(x, v)>."""
    x, v, r, gF = map(_f64, (x, v, r, gF))
    af = _alpha_field(params, alpha_f)
    n = x.shape[0]
    gx = np.zeros((n, 3))
    gv = np.zeros((n, 3))
    gmu = C.c_double(0.0)
    lib().or_contact_adj(C.byref(grid_struct(grid)), C.byref(params_struct(params)), C.c_int64(n), _p(x), _p(v),
                         _p(r), None if af is None else _p(af), _p(gF), C.c_int(int(brute)), _p(gx), _p(gv),
                         C.byref(gmu))
    return gx, gv, gmu.value


def g2p_adj(grid, params, x, v, r, u, vf, wf, p, af, gFfl, gaf, galpha=None):
    """(gx, gv, g_cdrag) of <gFfl, F_fl> + <gaf, a_f> + <galpha, alpha_f_p>."""
    x, v, r, gFfl, gaf = map(_f64, (x, v, r, gFfl, gaf))
    u, vf, wf, p, af = map(_f64, (u, vf, wf, p, af))
    n = x.shape[0]
    gx = np.zeros((n, 3))
    gv = np.zeros((n, 3))
    gc = C.c_double(0.0)
    ga = None if galpha is None else _f64(galpha)
    lib().or_g2p_adj(C.byref(grid_struct(grid)), C.byref(params_struct(params)), C.c_int64(n), _p(x), _p(v), _p(r),
                     _p(u), _p(vf), _p(wf), _p(p), _p(af), _p(gFfl), _p(gaf), None if ga is None else _p(ga), _p(gx),
                     _p(gv), C.byref(gc))
    return gx, gv, gc.value


def integrate_adj(grid, params, r, gx_new, gv_new, gfex=None):
    """(gx, gv, gFc, gFfl, gaf) of <gx_new, x'> + <gv_new, v'> + <gfex, f_ex>."""
    r, gx_new, gv_new = map(_f64, (r, gx_new, gv_new))
    n = r.shape[0]
    outs = [np.empty((n, 3)) for _ in range(5)]
    gf = None if gfex is None else _f64(gfex)
    lib().or_integrate_adj(C.byref(grid_struct(grid)), C.byref(params_struct(params)), C.c_int64(n), _p(r),
                           _p(gx_new), _p(gv_new), None if gf is None else _p(gf), *[_p(o) for o in outs])
    return tuple(outs)


def p2g_adj(grid, params, x_old, x_new, r, f_ex, g_alpha=None, gFs=None):
    """(gx_old, gx_new, gfex) of <g_alpha, alpha_s> + sum_c <gFs_c, F_s,c>."""
    x_old, x_new, r, f_ex = map(_f64, (x_old, x_new, r, f_ex))
    n = x_old.shape[0]
    gxo = np.zeros((n, 3))
    gxn = np.zeros((n, 3))
    gfe = np.zeros((n, 3))
    ga = None if g_alpha is None else _f64(g_alpha)
    gf = [None, None, None] if gFs is None else [_f64(a) for a in gFs]
    lib().or_p2g_adj(C.byref(grid_struct(grid)), C.byref(params_struct(params)), C.c_int64(n), _p(x_old), _p(x_new),
                     _p(r), _p(f_ex), None if ga is None else _p(ga), *[None if a is None else _p(a) for a in gf],
                     _p(gxo), _p(gxn), _p(gfe))
    return gxo, gxn, gfe


def run_adjoint(prob, gxK, gvK=None, K=None, params=None, x=None, v=None, brute=False, signature=False):
    """K substeps forward then the reverse pass.

    Returns dict(x, v (final), g_x0, g_v0, g_c (d/dc_drag), g_mu, sig, status)."""
    grid = prob.grid
    P = params if params is not None else prob.params
    K = prob.K if K is None else K
    x = decode(grid, prob.cell, prob.q) if x is None else _f64(x).copy()
    v = _f64(prob.v).copy() if v is None else _f64(v).copy()
    r = _f64(prob.r)
    n = x.shape[0]
    fl = [_f64(a) for a in (prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)]
    gx0 = np.empty((n, 3))
    gv0 = np.empty((n, 3))
    gc = C.c_double(0.0)
    gm = C.c_double(0.0)
    sig = np.zeros(3, np.uint64)
    st = C.c_uint32(0)
    gxK = _f64(gxK)
    gvK = None if gvK is None else _f64(gvK)
    lib().or_run_adjoint(C.byref(grid_struct(grid)), C.byref(params_struct(P)), C.c_int64(n), C.c_int(K), _p(x),
                         _p(v), _p(r), *[_p(a) for a in fl], _p(gxK), None if gvK is None else _p(gvK), _p(gx0),
                         _p(gv0), C.byref(gc), C.byref(gm), _p(sig) if signature else None, C.c_int(int(brute)),
                         C.byref(st))
    return dict(x=x, v=v, g_x0=gx0, g_v0=gv0, g_c=gc.value, g_mu=gm.value, sig=tuple(int(s) for s in sig),
                status=st.value)
