"""Host-side checks of the C ABI library (no GPU needed).

The library loads, exports every entry point include/gic.h declares, and its
host-side argument validation returns the documented error codes before any
device work is enqueued.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gic_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_00745_gb300 import gic
    return gic.lib()


def test_header_declares_the_hot_path():
    names = _declared()
    for need in ["gic_sort", "gic_contact", "gic_g2p_couple", "gic_integrate", "gic_p2g", "gic_sort_adj",
                 "gic_contact_adj", "gic_g2p_couple_adj", "gic_integrate_adj", "gic_p2g_adj"]:
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_launch_counter(lib):
    from paper_2504_00745_gb300 import gic
    assert "sm_103a" in gic.gic_version()
    assert gic.launch_count() >= 0


def test_grid_validation_codes():
    from paper_2504_00745_gb300 import gic
    bad = [gic.GicGrid(1, 4, 4, 1, 0.1, (C.c_double * 3)(0, 0, 0)),       # < 2 cells
           gic.GicGrid(4, 4, 4, 0, 0.1, (C.c_double * 3)(0, 0, 0)),       # k < 1
           gic.GicGrid(4, 4, 4, 1, -0.1, (C.c_double * 3)(0, 0, 0)),      # dx <= 0
           gic.GicGrid(600, 4, 4, 2, 0.1, (C.c_double * 3)(0, 0, 0))]     # > 1024 contact cells
    for g in bad:
        b = C.c_size_t(0)
        assert gic.lib().gic_workspace_size(C.byref(g), 10, 0, C.byref(b)) == -1
        assert "grid" in gic.last_error() or "cells" in gic.last_error() or "dx" in gic.last_error() \
            or "k_contact" in gic.last_error()


def test_sizes():
    from paper_2504_00745_gb300 import gic
    g = gic.GicGrid(32, 16, 8, 3, 1 / 32, (C.c_double * 3)(0, 0, 0))
    assert gic.gic_cell_table_size(g) == 16 * (1 + 96 * 48 * 24)
    a = gic.gic_workspace_size(g, 1000, 0)
    b = gic.gic_workspace_size(g, 100000, 0)
    assert 0 < a < b
    assert b >= 4 * 4 * 100000  # two ping-pong (key, value) pairs


def test_null_arguments_are_rejected_on_the_host():
    from paper_2504_00745_gb300 import gic
    L = gic.lib()
    g = gic.GicGrid(8, 8, 8, 1, 1 / 8, (C.c_double * 3)(0, 0, 0))
    p = gic.GicParams(2650, 1000, 1e5, 0.3, 1, 0.5, 0.22, (C.c_double * 3)(0, 0, -9.8), 1e-5, 1e-4, 1, 1)
    s = gic.GicGranules(10, None, None, None, None, 0)
    assert L.gic_contact(C.byref(g), C.byref(p), C.byref(s), None, None, None) == -1
    assert L.gic_sort(C.byref(g), C.byref(s), C.byref(s), None, None, None, 0, None) == -1
    s2 = gic.GicGranules(10, None, None, None, None, 7)
    assert L.gic_integrate(C.byref(g), C.byref(p), C.byref(s2), None, None, None, C.byref(s2), None, None) == -1
    assert "precision" in gic.last_error()
    bad_p = gic.GicParams(-1, 1000, 1e5, 0.3, 1, 0.5, 0.22, (C.c_double * 3)(0, 0, -9.8), 1e-5, 1e-4, 1, 1)
    empty = gic.GicGranules(0, None, None, None, None, 0)
    # an empty problem is valid and enqueues nothing
    assert L.gic_contact(C.byref(g), C.byref(bad_p), C.byref(empty), C.c_void_p(16), None, None) == 0
    assert L.gic_sort_adj(0, 0, None, None, None, None, None, None) == 0
    assert L.gic_sort_adj(5, 0, None, None, None, None, None, None) == -1
    # the staged list build wants an FP32 sorted state with ids and float copies
    fake = C.c_void_p(256)  # never dereferenced: the checks come first
    s64 = gic.GicGranules(10, fake, fake, fake, fake, 1, None)
    assert L.gic_neighbors_build(C.byref(g), C.byref(s64), fake, None, None) == -1
    assert "FP32" in gic.last_error()
    s32 = gic.GicGranules(10, fake, fake, fake, fake, 0, None)
    assert L.gic_neighbors_build(C.byref(g), C.byref(s32), fake, None, None) == -1
    assert L.gic_neighbors_build(C.byref(g), C.byref(s), fake, None, None) == -1  # no arrays


def test_projection_validation_on_the_host():
    """gic_project rejects bad grids, parameters, missing arrays and a short
    workspace before any device work (fake non-null pointers are never
    dereferenced on these paths)."""
    from paper_2504_00745_gb300 import gic
    L = gic.lib()
    g = gic.GicGrid(6, 5, 4, 1, 0.1, (C.c_double * 3)(0, 0, 0))
    one = gic.GicGrid(1, 1, 3, 1, 0.1, (C.c_double * 3)(0, 0, 0))  # a one-cell-wide column is a valid grid
    a = gic.gic_project_workspace_size(g)
    assert 0 < a < gic.gic_project_workspace_size(gic.GicGrid(60, 50, 40, 1, 0.1, (C.c_double * 3)(0, 0, 0)))
    assert gic.gic_project_workspace_size(one) > 0
    fake = C.c_void_p(1 << 20)
    arrays = [fake] * 7 + [None] * 6

    def call(grid, pp, arr=arrays, ws=fake, nbytes=a):
        return L.gic_project(C.byref(grid), C.byref(pp), *arr, ws, nbytes, None, None)

    good = gic.make_proj_params(2e-3, 1000.0)
    assert call(gic.GicGrid(0, 5, 4, 1, 0.1, (C.c_double * 3)(0, 0, 0)), good) == -1
    assert call(gic.GicGrid(6, 5, 4, 1, 0.0, (C.c_double * 3)(0, 0, 0)), good) == -1
    for bad in (gic.make_proj_params(0.0, 1000.0), gic.make_proj_params(2e-3, 1000.0, alpha_s_max=1.0),
                gic.make_proj_params(2e-3, 1000.0, ratio_min=1.2), gic.make_proj_params(2e-3, 1000.0, tol=0.0),
                gic.make_proj_params(2e-3, 1000.0, inner_tol=1.0), gic.make_proj_params(2e-3, 1000.0, max_inner=0)):
        assert call(g, bad) == -1
    assert call(g, gic.make_proj_params(2e-3, 1000.0, open_sides=(0, 0, 0, 0, 0, 0))) == -1
    assert "open" in gic.last_error()
    assert call(g, good, arr=[fake] * 6 + [None] + [None] * 6) == -1  # p2 missing
    assert call(g, good, arr=[fake] * 7 + [fake, None, None] + [None] * 3) == -1
    assert "all three" in gic.last_error()
    assert call(g, good, nbytes=a - 1) == -3
    assert call(g, good, ws=C.c_void_p((1 << 20) + 64)) == -4
    huge = gic.GicGrid(1024, 1024, 1024, 1, 0.1, (C.c_double * 3)(0, 0, 0))  # 2^30 cells: 32-bit indices
    assert call(huge, good) == -1 and "2^30" in gic.last_error()


def test_capillary_parameters_and_scope_on_the_host():
    """The capillary force (sigma > 0, Sec. 5.4) is evaluated by the fused
    entry points only: the separate contact entry points refuse it before
    any device work, and the fused ones validate its parameters (checked
    here on an empty problem, which enqueues nothing)."""
    from paper_2504_00745_gb300 import gic
    L = gic.lib()
    g = gic.GicGrid(8, 8, 8, 1, 1 / 8, (C.c_double * 3)(0, 0, 0))
    wet = gic.GicParams(2650, 1000, 1e5, 0.3, 1, 0.5, 0.22, (C.c_double * 3)(0, 0, -9.8), 1e-5, 1e-4, 1, 1,
                        0.07, 1e-4, 0.0, 0.3)
    empty = gic.GicGranules(0, None, None, None, None, 0)
    for name, args in (("gic_contact", (C.byref(g), C.byref(wet), C.byref(empty), C.c_void_p(16), None, None)),
                       ("gic_contact_verlet", (C.byref(g), C.byref(wet), C.byref(empty), C.c_void_p(16), None, None,
                                               None))):
        assert getattr(L, name)(*args) == -1, name
        assert "capillary" in gic.last_error()
    # the fused substep validates the capillary parameters
    bad = gic.GicParams(2650, 1000, 1e5, 0.3, 1, 0.5, 0.22, (C.c_double * 3)(0, 0, -9.8), 1e-5, 1e-4, 1, 1,
                        0.07, 1e-4, 0.0, 0.9)  # peak outside [1/4, 3/4]
    nb = gic.GicNeighbors(0, 48, 0.0, *([C.c_void_p(256)] * 8))
    rc = L.gic_substep(C.byref(g), C.byref(bad), C.byref(empty), C.c_void_p(16), C.byref(nb), *([C.c_void_p(256)] * 5),
                       C.byref(empty), None, None, None, None, None, None, None)
    assert rc == -1 and "moisture_peak" in gic.last_error()


def test_debug_build_compiles_and_exports_the_same_symbols():
    """The GIC_DEBUG variant (device-side index checks that flag
    GIC_STATUS_DEBUG_INDEX and skip the access) builds for sm_103a and has the
    release library's interface."""
    import subprocess

    from paper_2504_00745_gb300 import build as b
    path = b.build(debug=True)
    syms = lambda p: {ln.split()[-1] for ln in subprocess.run(["nm", "-D", "--defined-only", p], capture_output=True,
                                                             text=True).stdout.splitlines() if " T gic_" in ln}
    assert syms(path) == syms(b.build()) and "gic_step" in syms(path)
