"""gic_sort_static: the sort variant for callers that cannot allocate device
memory (its scratch is a static array inside the library).

It must give bit-for-bit the results of gic_sort with a caller workspace, on
consecutive calls with different inputs (the shared array keeps the previous
call's contents), and refuse inputs beyond its fixed capacity.  This file is
collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import gic_inputs as gi
from gpu_util import FP32, FP64, shuffled, subset
from paper_2504_00745_gb300 import gic
from paper_2504_00745_gb300.window import Simulator

pytestmark = pytest.mark.gpu


def _sorted_both_ways(prob, prec):
    sim = Simulator.from_problem(prob, prec)
    # reference: the workspace variant into its own buffers and table
    B_ref = gic.State.empty(prob.n, prec)
    perm_ref = torch.empty(prob.n, dtype=torch.int32, device="cuda")
    table_ref = gic.new_cell_table(sim.grid)
    gic.gic_sort(sim.grid, sim.A, B_ref, perm_ref, table_ref, sim.ws)
    # the static-scratch variant, straight through the C ABI
    table = gic.new_cell_table(sim.grid)
    a, b = sim.A.struct(), sim.B.struct()
    rc = gic.lib().gic_sort_static(C.byref(sim.grid), C.byref(a), C.byref(b), C.c_void_p(sim.perm.data_ptr()),
                                   C.c_void_p(table.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, gic.last_error()
    torch.cuda.synchronize()
    return (perm_ref, B_ref, table_ref), (sim.perm, sim.B, table)


def _assert_same(ref, got):
    (p0, B0, t0), (p1, B1, t1) = ref, got
    assert torch.equal(p0, p1)
    assert torch.equal(B0.cell, B1.cell)
    assert torch.equal(B0.pos, B1.pos)
    assert torch.equal(B0.vel, B1.vel)
    assert torch.equal(B0.id, B1.id)
    assert torch.equal(t0, t1)


def test_static_sort_matches_workspace_sort_on_consecutive_calls():
    first = shuffled(gi.make("dense_block"), seed=1)                  # 2,048 granules
    second = shuffled(gi.make("diff_window_100k"), seed=2)            # 100,000 granules, other grid
    third = subset(shuffled(gi.make("dense_block"), seed=3), 1500)    # smaller again: stale scratch beyond n
    for prob, prec in ((first, FP32), (second, FP32), (third, FP64)):
        ref, got = _sorted_both_ways(prob, prec)
        _assert_same(ref, got)
    assert gic.gic_check_status() == 0


def test_static_sort_allocates_no_device_memory():
    """What the entry point exists for: once the library is loaded on the
    device (the first call), further calls -- other sizes, other grids, both
    precisions -- leave the device's free memory and torch's allocator
    exactly where they were.  Every input is allocated before the first
    reading."""
    cases = [(shuffled(gi.make("dense_block"), seed=4), FP32), (shuffled(gi.make("diff_window_100k"), seed=5), FP32),
             (subset(shuffled(gi.make("dense_block"), seed=6), 700), FP64)]
    prepared = []
    for prob, prec in cases:
        sim = Simulator.from_problem(prob, prec)
        table = gic.new_cell_table(sim.grid)
        prepared.append((sim, table))
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(sim, table):
        a, b = sim.A.struct(), sim.B.struct()
        rc = gic.lib().gic_sort_static(C.byref(sim.grid), C.byref(a), C.byref(b), C.c_void_p(sim.perm.data_ptr()),
                                       C.c_void_p(table.data_ptr()), stream)
        assert rc == 0, gic.last_error()

    call(*prepared[0])  # module loading, if this is the first call in the process
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    for _ in range(2):
        for sim, table in prepared:
            call(sim, table)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0
    assert gic.gic_check_status() == 0


def test_static_sort_rejects_more_than_its_capacity():
    nmax = gic.gic_sort_static_max_n()
    assert nmax == 262144
    prob = gi.make("dense_block")
    grid = gic.make_grid(prob.grid)
    n = nmax + 1
    A = gic.State.empty(n, FP32)
    B = gic.State.empty(n, FP32)
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    table = gic.new_cell_table(grid)
    launches = gic.launch_count()
    with pytest.raises(gic.GicError, match="exceed"):
        gic.gic_sort_static(grid, A, B, perm, table)
    assert gic.launch_count() == launches
