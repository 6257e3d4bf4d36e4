"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Every rank runs an independent replica; the job throughput is all ranks'
units over the slowest rank's time.  The ranks here report different times
and must agree on the maximum."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench

    class A:
        pass

    ws_, rank_, local_ = bench.dist_setup(A())
    assert (ws_, rank_) == (ws, rank)
    bench.barrier(ws_)
    ms_here = 10.0 * (rank + 1)  # rank 1 is the slowest
    value, ms = bench.job_throughput(1000, ms_here, ws_, device="cpu")
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_two_rank_replica_timing_uses_the_slowest_rank():
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
    for r in range(ws):
        value, ms = out[r]
        assert ms == 20.0
        assert abs(value - ws * 1000 / 0.020) < 1e-6


def test_single_rank_is_unchanged():
    import bench

    value, ms = bench.job_throughput(500, 5.0, 1)
    assert ms == 5.0 and abs(value - 500 / 0.005) < 1e-9
