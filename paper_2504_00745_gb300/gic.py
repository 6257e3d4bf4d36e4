"""Thin ctypes binding of libgic.so (include/gic.h): argument marshalling only.

Every function here has the name of the C entry point it calls and takes
torch CUDA tensors (device memory) plus the enqueueing stream (default: the
current torch stream).  All arithmetic happens in the library's kernels; if
the library is missing this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import torch

from . import build as _build

GIC_FP32, GIC_FP64 = 0, 1
STATUS_OUT_OF_DOMAIN = 1
STATUS_COINCIDENT = 2
STATUS_NONFINITE = 4
STATUS_RADIUS = 8
STATUS_BAD_CELL = 16
STATUS_FAST = 32
STATUS_DEBUG_INDEX = 64  # set only by the GIC_DEBUG build


class GicError(RuntimeError):
    pass


class GicGrid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("k_contact", C.c_int32),
                ("dx", C.c_double), ("origin", C.c_double * 3)]


class GicParams(C.Structure):
    _fields_ = [("rho_s", C.c_double), ("rho_f", C.c_double), ("k_n", C.c_double), ("zeta", C.c_double),
                ("kt_over_cn", C.c_double), ("mu_fric", C.c_double), ("c_drag", C.c_double), ("g", C.c_double * 3),
                ("dt_sub", C.c_double), ("dt_fluid", C.c_double), ("virtual_mass", C.c_int32), ("walls", C.c_int32),
                ("sigma", C.c_double), ("bridge_frac", C.c_double), ("moisture", C.c_double),
                ("moisture_peak", C.c_double)]


class GicGranules(C.Structure):
    _fields_ = [("n", C.c_int64), ("cell", C.c_void_p), ("pos", C.c_void_p), ("vel", C.c_void_p), ("id", C.c_void_p),
                ("precision", C.c_int32), ("posf", C.c_void_p)]


class GicProjParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("rho_f", C.c_double), ("alpha_s_max", C.c_double), ("ratio_min", C.c_double),
                ("ratio_max", C.c_double), ("tol", C.c_double), ("inner_tol", C.c_double), ("max_outer", C.c_int32),
                ("max_inner", C.c_int32), ("open", C.c_int32 * 6)]


class GicProjInfo(C.Structure):
    _fields_ = [("outer", C.c_int32 * 2), ("inner", C.c_int32 * 2), ("converged", C.c_int32 * 2),
                ("rel_residual", C.c_double * 2)]


class GicNeighbors(C.Structure):
    _fields_ = [("n", C.c_int64), ("cap", C.c_int32), ("skin", C.c_double), ("list", C.c_void_p),
                ("count", C.c_void_p), ("ref_cell", C.c_void_p), ("ref_pos", C.c_void_p), ("slot", C.c_void_p),
                ("cur", C.c_void_p), ("at", C.c_void_p), ("flags", C.c_void_p)]


_P = C.c_void_p
_SIGS = {
    "gic_workspace_size": [_P, C.c_int64, C.c_int32, _P],
    "gic_cell_table_size": [_P, _P],
    "gic_pack": [_P, C.c_int64, _P, _P, _P, _P, _P, _P],
    "gic_unpack": [_P, _P, _P, _P, _P],
    "gic_unpack_adj": [_P, _P, _P, _P, _P, _P, _P],
    "gic_sort": [_P, _P, _P, _P, _P, _P, C.c_size_t, _P],
    "gic_contact": [_P, _P, _P, _P, _P, _P],
    "gic_g2p_couple": [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "gic_integrate": [_P, _P, _P, _P, _P, _P, _P, _P, _P],
    "gic_p2g": [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "gic_sort_adj": [C.c_int64, C.c_int32, _P, _P, _P, _P, _P, _P],
    "gic_contact_adj": [_P, _P, _P, _P, _P, _P, _P, _P, _P],
    "gic_g2p_couple_adj": [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "gic_integrate_adj": [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "gic_p2g_adj": [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "gic_contact_pairs": [_P, _P, _P, _P, _P, C.c_int64, _P, _P],
    "gic_check_status": [_P, C.c_int32, C.c_int32, _P],
    "gic_sort_static": [_P, _P, _P, _P, _P, _P],
    "gic_contact_verlet": [_P, _P, _P, _P, _P, _P, _P],
    "gic_neighbors_reset": [_P, _P],
    "gic_substep": [_P] * 18,
    "gic_contact_verlet_adj": [_P] * 11,
    "gic_substep_adj": [_P] * 19,
    "gic_step": [_P, _P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "gic_project_workspace_size": [_P, _P],
    "gic_project": [_P] * 16 + [C.c_size_t, _P, _P],
}
# entry points that exist in include/gic.h but are declared optional here
# (added later in the library's life) are looked up lazily
_lib = None


def _debug_wanted() -> bool:
    """GIC_LIBRARY=debug in the environment selects the GIC_DEBUG build
    (device-side index checks) for this process."""
    return os.environ.get("GIC_LIBRARY", "") == "debug"


def lib_path() -> str:
    return _build.DEBUG_LIB if _debug_wanted() else _build.LIB


def lib():
    """Load libgic.so (building it first when the sources are newer)."""
    global _lib
    if _lib is None:
        debug = _debug_wanted()
        path = _build.DEBUG_LIB if debug else _build.LIB
        if not _build.up_to_date(debug):
            try:
                _build.build(debug=debug)
            except Exception as e:  # no nvcc or compile error: fail loudly, never fall back
                raise GicError(f"libgic.so is missing or stale and could not be built: {e}") from e
        if not os.path.exists(path):
            raise GicError(f"libgic.so not found at {path}")
        L = C.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.gic_last_error.restype = C.c_char_p
        L.gic_version.restype = C.c_char_p
        L.gic_launch_count.restype = C.c_int64
        L.gic_sort_static_max_n.restype = C.c_int64
        _lib = L
    return _lib


def last_error() -> str:
    return lib().gic_last_error().decode()


def launch_count() -> int:
    return int(lib().gic_launch_count())


def _check(rc: int, what: str):
    if rc != 0:
        raise GicError(f"{what} failed ({rc}): {last_error()}")


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise GicError("expected a CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def make_grid(g) -> GicGrid:
    """From any object with nx, ny, nz, dx, origin, k_contact."""
    return GicGrid(int(g.nx), int(g.ny), int(g.nz), int(g.k_contact), float(g.dx), (C.c_double * 3)(*g.origin))


def make_params(p) -> GicParams:
    return GicParams(p.rho_s, p.rho_f, p.k_n, p.zeta, p.kt_over_cn, p.mu_fric, p.c_drag, (C.c_double * 3)(*p.g),
                     p.dt_sub, p.dt_fluid, int(p.virtual_mass), int(p.walls), float(getattr(p, "sigma", 0.0)),
                     float(getattr(p, "bridge_frac", 1e-4)), float(getattr(p, "moisture", 0.0)),
                     float(getattr(p, "moisture_peak", 0.3)))


@dataclass
class State:
    """Granule state in device memory (structure of arrays, see include/gic.h)."""
    cell: torch.Tensor  # int32 [n]
    pos: torch.Tensor   # int32 [n, 4] (FP32 path: q bits + radius bits) or float64 [n, 4]
    vel: torch.Tensor   # float32 / float64 [n, 4]
    id: Optional[torch.Tensor]  # int32 [n] or None
    precision: int
    posf: Optional[torch.Tensor] = None  # FP32 path: float32 [n, 4] copy written by gic_sort, or None

    @property
    def n(self) -> int:
        return int(self.cell.shape[0])

    @property
    def real(self):
        return torch.float32 if self.precision == GIC_FP32 else torch.float64

    @staticmethod
    def empty(n: int, precision: int, device="cuda", with_id=True, with_posf=False) -> "State":
        real = torch.float32 if precision == GIC_FP32 else torch.float64
        pos_dtype = torch.int32 if precision == GIC_FP32 else torch.float64
        posf = torch.empty((n, 4), dtype=torch.float32, device=device) if (with_posf and precision == GIC_FP32) \
            else None
        return State(torch.empty(n, dtype=torch.int32, device=device),
                     torch.empty((n, 4), dtype=pos_dtype, device=device),
                     torch.zeros((n, 4), dtype=real, device=device),
                     torch.empty(n, dtype=torch.int32, device=device) if with_id else None, precision, posf)

    def struct(self) -> GicGranules:
        return GicGranules(self.n, _ptr(self.cell), _ptr(self.pos), _ptr(self.vel), _ptr(self.id), self.precision,
                           _ptr(self.posf))

    def clone(self) -> "State":
        return State(self.cell.clone(), self.pos.clone(), self.vel.clone(),
                     None if self.id is None else self.id.clone(), self.precision,
                     None if self.posf is None else self.posf.clone())


def vec4(n: int, precision: int, device="cuda") -> torch.Tensor:
    return torch.zeros((n, 4), dtype=torch.float32 if precision == GIC_FP32 else torch.float64, device=device)


# ---------------------------------------------------------------- sizes

def gic_workspace_size(grid: GicGrid, n: int, precision: int) -> int:
    b = C.c_size_t(0)
    _check(lib().gic_workspace_size(C.byref(grid), n, precision, C.byref(b)), "gic_workspace_size")
    return int(b.value)


def gic_cell_table_size(grid: GicGrid) -> int:
    b = C.c_size_t(0)
    _check(lib().gic_cell_table_size(C.byref(grid), C.byref(b)), "gic_cell_table_size")
    return int(b.value)


def new_workspace(grid: GicGrid, n: int, precision: int, device="cuda") -> torch.Tensor:
    return torch.empty(max(gic_workspace_size(grid, n, precision), 256), dtype=torch.uint8, device=device)


def new_cell_table(grid: GicGrid, device="cuda") -> torch.Tensor:
    return torch.zeros(gic_cell_table_size(grid) // 4, dtype=torch.int32, device=device)


# ---------------------------------------------------------------- conversion

def gic_pack(grid: GicGrid, cell_xyz, q, r, v, out: State, stream=None):
    s = out.struct()
    _check(lib().gic_pack(C.byref(grid), out.n, _ptr(cell_xyz), _ptr(q), _ptr(r), _ptr(v), C.byref(s),
                          _stream(stream)), "gic_pack")


def gic_unpack(grid: GicGrid, st: State, x=None, v=None, stream=None):
    s = st.struct()
    _check(lib().gic_unpack(C.byref(grid), C.byref(s), _ptr(x), _ptr(v), _stream(stream)), "gic_unpack")


def gic_unpack_adj(grid: GicGrid, st: State, gx, gv, g_pos, g_vel, stream=None):
    s = st.struct()
    _check(lib().gic_unpack_adj(C.byref(grid), C.byref(s), _ptr(gx), _ptr(gv), _ptr(g_pos), _ptr(g_vel),
                                _stream(stream)), "gic_unpack_adj")


# ---------------------------------------------------------------- forward

def gic_sort(grid: GicGrid, st_in: State, st_out: State, perm, cell_table, ws, stream=None):
    a, b = st_in.struct(), st_out.struct()
    _check(lib().gic_sort(C.byref(grid), C.byref(a), C.byref(b), _ptr(perm), _ptr(cell_table), _ptr(ws),
                          ws.numel() * ws.element_size(), _stream(stream)), "gic_sort")


def gic_sort_static(grid: GicGrid, st_in: State, st_out: State, perm, cell_table, stream=None):
    """gic_sort with the library's static scratch instead of a workspace."""
    a, b = st_in.struct(), st_out.struct()
    _check(lib().gic_sort_static(C.byref(grid), C.byref(a), C.byref(b), _ptr(perm), _ptr(cell_table),
                                 _stream(stream)), "gic_sort_static")


def gic_sort_static_max_n() -> int:
    return int(lib().gic_sort_static_max_n())


def gic_contact(grid: GicGrid, params: GicParams, st: State, cell_table, F_c, stream=None):
    s = st.struct()
    _check(lib().gic_contact(C.byref(grid), C.byref(params), C.byref(s), _ptr(cell_table), _ptr(F_c),
                             _stream(stream)), "gic_contact")


class Neighbors:
    """Device arrays of a GicNeighbors (Verlet lists kept by granule id)."""

    def __init__(self, n: int, precision: int, cap: int = 48, skin: float = 0.0, device="cuda"):
        self.n, self.cap, self.skin, self.precision = n, cap, float(skin), precision
        i32 = dict(dtype=torch.int32, device=device)
        self.list = torch.empty(max(n * cap, 1), **i32)
        self.count = torch.zeros(max(n, 1), **i32)
        self.ref_cell = torch.zeros(max(n, 1), **i32)
        real = torch.int32 if precision == GIC_FP32 else torch.float64
        self.ref_pos = torch.zeros((max(n, 1), 4), dtype=real, device=device)
        self.slot = torch.zeros(max(n, 1), **i32)
        self.cur = torch.zeros(max(n, 1), **i32)
        self.at = torch.zeros(max(n, 1), **i32)
        self.flags = torch.zeros(8, **i32)

    def struct(self) -> GicNeighbors:
        return GicNeighbors(self.n, self.cap, self.skin, _ptr(self.list), _ptr(self.count), _ptr(self.ref_cell),
                            _ptr(self.ref_pos), _ptr(self.slot), _ptr(self.cur), _ptr(self.at), _ptr(self.flags))

    def builds(self) -> int:
        return int(self.flags[4].item())

    def overflowed(self) -> bool:
        return bool(int(self.flags[1].item()) & 2)


def gic_contact_verlet(grid: GicGrid, params: GicParams, st: State, cell_table, nb: Neighbors, F_c, stream=None):
    s, b = st.struct(), nb.struct()
    _check(lib().gic_contact_verlet(C.byref(grid), C.byref(params), C.byref(s), _ptr(cell_table), C.byref(b), _ptr(F_c),
                                    _stream(stream)), "gic_contact_verlet")


def gic_substep(grid: GicGrid, params: GicParams, sorted_: State, cell_table, nb: Neighbors, u, v, w, p, alpha_f,
                next_: State, f_ex=None, alpha_s=None, Fs=(None, None, None), sums2=None, stream=None):
    s, t, b = sorted_.struct(), next_.struct(), nb.struct()
    _check(lib().gic_substep(C.byref(grid), C.byref(params), C.byref(s), _ptr(cell_table), C.byref(b), _ptr(u),
                             _ptr(v), _ptr(w), _ptr(p), _ptr(alpha_f), C.byref(t), _ptr(f_ex),
                             _ptr(alpha_s), _ptr(Fs[0]), _ptr(Fs[1]), _ptr(Fs[2]), _ptr(sums2), _stream(stream)),
           "gic_substep")


def gic_contact_verlet_adj(grid, params, st: State, cell_table, nb: Neighbors, F_c, gF_c, g_pos, g_vel, g_mu,
                           stream=None):
    s, b = st.struct(), nb.struct()
    _check(lib().gic_contact_verlet_adj(C.byref(grid), C.byref(params), C.byref(s), _ptr(cell_table), C.byref(b),
                                        _ptr(F_c), _ptr(gF_c), _ptr(g_pos), _ptr(g_vel), _ptr(g_mu),
                                        _stream(stream)), "gic_contact_verlet_adj")


def gic_substep_adj(grid: GicGrid, params: GicParams, sorted_: State, perm, cell_table, nb: Neighbors, u, v, w, p,
                    alpha_f, g_pos_out, g_vel_out, g_f_ex, g_pos_in, g_vel_in, g_cdrag=None, g_mu=None, stream=None):
    s, b = sorted_.struct(), nb.struct()
    _check(lib().gic_substep_adj(C.byref(grid), C.byref(params), C.byref(s), _ptr(perm), _ptr(cell_table),
                                 C.byref(b), _ptr(u), _ptr(v), _ptr(w), _ptr(p), _ptr(alpha_f), _ptr(g_pos_out),
                                 _ptr(g_vel_out), _ptr(g_f_ex), _ptr(g_pos_in), _ptr(g_vel_in), _ptr(g_cdrag),
                                 _ptr(g_mu), _stream(stream)), "gic_substep_adj")


def gic_step(grid: GicGrid, params: GicParams, state: State, next_: State, sorted_: State, perm, cell_table, ws,
             nb: Neighbors, u, v, w, p, alpha_f, alpha_s=None, Fs=(None, None, None), sums2=None, stream=None):
    a, t, s, b = state.struct(), next_.struct(), sorted_.struct(), nb.struct()
    _check(lib().gic_step(C.byref(grid), C.byref(params), C.byref(a), C.byref(t), C.byref(s), _ptr(perm),
                          _ptr(cell_table), _ptr(ws), ws.numel() * ws.element_size(), C.byref(b), _ptr(u), _ptr(v),
                          _ptr(w), _ptr(p), _ptr(alpha_f), _ptr(alpha_s), _ptr(Fs[0]), _ptr(Fs[1]), _ptr(Fs[2]),
                          _ptr(sums2), _stream(stream)), "gic_step")


def gic_neighbors_reset(nb: Neighbors, stream=None):
    b = nb.struct()
    _check(lib().gic_neighbors_reset(C.byref(b), _stream(stream)), "gic_neighbors_reset")


def gic_neighbors_build(grid: GicGrid, sorted_: State, cell_table, nb: Neighbors, stream=None):
    b = nb.struct()
    s = sorted_.struct()
    _check(lib().gic_neighbors_build(C.byref(grid), C.byref(s), _ptr(cell_table), C.byref(b), _stream(stream)),
           "gic_neighbors_build")


def gic_g2p_couple(grid: GicGrid, params: GicParams, st: State, u, v, w, p, alpha_f, F_fl, a_f, alpha_f_p=None,
                   stream=None):
    s = st.struct()
    _check(lib().gic_g2p_couple(C.byref(grid), C.byref(params), C.byref(s), _ptr(u), _ptr(v), _ptr(w), _ptr(p),
                                _ptr(alpha_f), _ptr(F_fl), _ptr(a_f), _ptr(alpha_f_p), _stream(stream)),
           "gic_g2p_couple")


def gic_integrate(grid: GicGrid, params: GicParams, st_in: State, F_c, F_fl, a_f, st_out: State, f_ex,
                  stream=None):
    a, b = st_in.struct(), st_out.struct()
    _check(lib().gic_integrate(C.byref(grid), C.byref(params), C.byref(a), _ptr(F_c), _ptr(F_fl), _ptr(a_f),
                               C.byref(b), _ptr(f_ex), _stream(stream)), "gic_integrate")


def gic_p2g(grid: GicGrid, params: GicParams, old: State, new: State, f_ex, alpha_s=None, Fs=(None, None, None),
            sums2=None, stream=None):
    a, b = old.struct(), new.struct()
    _check(lib().gic_p2g(C.byref(grid), C.byref(params), C.byref(a), C.byref(b), _ptr(f_ex), _ptr(alpha_s),
                         _ptr(Fs[0]), _ptr(Fs[1]), _ptr(Fs[2]), _ptr(sums2), _stream(stream)), "gic_p2g")


# ---------------------------------------------------------------- adjoints

def gic_sort_adj(n: int, precision: int, perm, g_pos_out, g_vel_out, g_pos_in, g_vel_in, stream=None):
    _check(lib().gic_sort_adj(n, precision, _ptr(perm), _ptr(g_pos_out), _ptr(g_vel_out), _ptr(g_pos_in),
                              _ptr(g_vel_in), _stream(stream)), "gic_sort_adj")


def gic_contact_adj(grid, params, st: State, cell_table, gF_c, g_pos, g_vel, g_mu, stream=None):
    s = st.struct()
    _check(lib().gic_contact_adj(C.byref(grid), C.byref(params), C.byref(s), _ptr(cell_table), _ptr(gF_c),
                                 _ptr(g_pos), _ptr(g_vel), _ptr(g_mu), _stream(stream)), "gic_contact_adj")


def gic_g2p_couple_adj(grid, params, st: State, u, v, w, p, alpha_f, gF_fl, ga_f, galpha_f_p, g_pos, g_vel, g_cdrag,
                       stream=None):
    s = st.struct()
    _check(lib().gic_g2p_couple_adj(C.byref(grid), C.byref(params), C.byref(s), _ptr(u), _ptr(v), _ptr(w), _ptr(p),
                                    _ptr(alpha_f), _ptr(gF_fl), _ptr(ga_f), _ptr(galpha_f_p), _ptr(g_pos),
                                    _ptr(g_vel), _ptr(g_cdrag), _stream(stream)), "gic_g2p_couple_adj")


def gic_integrate_adj(grid, params, st_in: State, g_pos_out, g_vel_out, g_f_ex, g_pos_in, g_vel_in, gF_c, gF_fl,
                      ga_f, stream=None):
    s = st_in.struct()
    _check(lib().gic_integrate_adj(C.byref(grid), C.byref(params), C.byref(s), _ptr(g_pos_out), _ptr(g_vel_out),
                                   _ptr(g_f_ex), _ptr(g_pos_in), _ptr(g_vel_in), _ptr(gF_c), _ptr(gF_fl),
                                   _ptr(ga_f), _stream(stream)), "gic_integrate_adj")


def gic_p2g_adj(grid, params, old: State, new: State, f_ex, g_alpha_s, gFs, g_pos_old, g_pos_new, g_f_ex,
                stream=None):
    a, b = old.struct(), new.struct()
    gFs = gFs if gFs is not None else (None, None, None)
    _check(lib().gic_p2g_adj(C.byref(grid), C.byref(params), C.byref(a), C.byref(b), _ptr(f_ex), _ptr(g_alpha_s),
                             _ptr(gFs[0]), _ptr(gFs[1]), _ptr(gFs[2]), _ptr(g_pos_old), _ptr(g_pos_new),
                             _ptr(g_f_ex), _stream(stream)), "gic_p2g_adj")


# ---------------------------------------------------------------- projection

def make_proj_params(dt: float, rho_f: float, open_sides=(0, 0, 0, 0, 0, 1), alpha_s_max: float = 0.740,
                     ratio_min: float = 0.5, ratio_max: float = 1.5, tol: float = 1e-9, inner_tol: float = 1e-3,
                     max_outer: int = 12, max_inner: int = 4000) -> GicProjParams:
    return GicProjParams(float(dt), float(rho_f), float(alpha_s_max), float(ratio_min), float(ratio_max), float(tol),
                         float(inner_tol), int(max_outer), int(max_inner), (C.c_int32 * 6)(*[int(o) for o in open_sides]))


def gic_project_workspace_size(grid: GicGrid) -> int:
    b = C.c_size_t(0)
    _check(lib().gic_project_workspace_size(C.byref(grid), C.byref(b)), "gic_project_workspace_size")
    return int(b.value)


def gic_project(grid: GicGrid, params: GicProjParams, alpha_s, alpha_star, u, v, w, p1, p2, vel_out=(None, None, None),
                disp_out=(None, None, None), ws=None, stream=None) -> GicProjInfo:
    """Both projections; blocks until they are solved.  Returns the solver's
    counts (GicProjInfo)."""
    if ws is None:
        ws = torch.empty(gic_project_workspace_size(grid), dtype=torch.uint8, device=alpha_s.device)
    info = GicProjInfo()
    _check(lib().gic_project(C.byref(grid), C.byref(params), _ptr(alpha_s), _ptr(alpha_star), _ptr(u), _ptr(v),
                             _ptr(w), _ptr(p1), _ptr(p2), _ptr(vel_out[0]), _ptr(vel_out[1]), _ptr(vel_out[2]),
                             _ptr(disp_out[0]), _ptr(disp_out[1]), _ptr(disp_out[2]), _ptr(ws), ws.numel(),
                             C.byref(info), _stream(stream)), "gic_project")
    return info


# ---------------------------------------------------------------- diagnostics

def gic_contact_pairs(grid, st: State, cell_table, counts=None, pairs=None, n_pairs=None, stream=None):
    s = st.struct()
    max_pairs = 0 if pairs is None else pairs.shape[0]
    _check(lib().gic_contact_pairs(C.byref(grid), C.byref(s), _ptr(cell_table), _ptr(counts), _ptr(pairs), max_pairs,
                                   _ptr(n_pairs), _stream(stream)), "gic_contact_pairs")


def gic_check_status(clear: bool = True, timeout_ms: int = 60000, stream=None) -> int:
    f = C.c_uint32(0)
    _check(lib().gic_check_status(C.byref(f), int(clear), int(timeout_ms), _stream(stream)), "gic_check_status")
    return int(f.value)


def gic_window_forward_host(grid: GicGrid, params: GicParams, precision: int, cell_xyz, q, r, v, u, vf, wf, p,
                            alpha_f, K: int, x_out, v_out, alpha_s, Fs, sums2, ws, stream=None):
    """K substeps on HOST (CPU, ideally pinned) tensors through the C ABI; ws
    is a device workspace of gic_window_host_workspace_size bytes."""
    L = lib()
    f = L.gic_window_forward_host
    f.argtypes = [_P, _P, C.c_int64, C.c_int32] + [_P] * 9 + [C.c_int32] + [_P] * 8 + [C.c_size_t, _P]
    f.restype = C.c_int
    hp = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    Fs = Fs if Fs is not None else (None, None, None)
    _check(f(C.byref(grid), C.byref(params), int(r.shape[0]), precision, hp(cell_xyz), hp(q), hp(r), hp(v), hp(u),
             hp(vf), hp(wf), hp(p), hp(alpha_f), int(K), hp(x_out), hp(v_out), hp(alpha_s), hp(Fs[0]), hp(Fs[1]),
             hp(Fs[2]), hp(sums2), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "gic_window_forward_host")


def gic_window_host_workspace_size(grid: GicGrid, n: int, precision: int) -> int:
    L = lib()
    L.gic_window_host_workspace_size.argtypes = [_P, C.c_int64, C.c_int32, _P]
    b = C.c_size_t(0)
    _check(L.gic_window_host_workspace_size(C.byref(grid), n, precision, C.byref(b)), "gic_window_host_workspace_size")
    return int(b.value)


def gic_version() -> str:
    return lib().gic_version().decode()
