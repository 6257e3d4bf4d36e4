"""Benchmark of the granule-grid coupling substep on GB300.

One step = one window of K substeps of Alg. 2 (sort, contact, G2P couple,
integrate, P2G with FP64 volume fraction and conservation sums) over the
1,000,000-granule dam-break column on a 128^3 grid (100 substeps of 2e-5 s,
FP32 state with FP64 alpha_s accumulation), starting every step from the same
seeded initial packing.  The metric is granule-substeps per second.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "granule-substeps/s fwd & adjoint, FP32 vs FP64 on 1 GB300; % HBM roofline"
UNIT = "granule-substeps/s"
# algorithmic bytes per granule-substep of each step (FP32 path): what the
# method must move, 12 B per 3-vector, state = 36 B.  P2G scatters F_s from
# the old positions every substep (cell + pos 20 B, f_ex 12 B) and alpha_s
# from the new ones once per fluid step (20 B more on the last substep).
# The fused substep (contact, G2P, integrate, P2G after the sort) reads the
# sorted state and writes the next one: 36 + 36 B.
ALGO_BYTES = {"gic_sort": 88, "gic_contact": 48, "gic_g2p_couple": 65, "gic_integrate": 120, "gic_p2g": 32,
              "gic_substep": 72, "gic_step": 72}
P2G_ALPHA_BYTES = 20
# DRAM bytes (read + write) of one call of the dominant entry point on a
# substep that keeps its Verlet lists (the gic_step graph: the decision
# kernel + k_substep), from an ncu capture of the current kernels on the same
# workload, the graph profiled as one unit (ncu flushes the caches first)
NCU_TRAFFIC = {("dam_break_1m", "gic_step"): 197.0e6}


def algo_bytes(name, K):
    """Algorithmic bytes per granule of one call of `name`, averaged over a
    K-substep window."""
    return ALGO_BYTES[name] + (P2G_ALPHA_BYTES / K if name in ("gic_p2g", "gic_substep", "gic_step") else 0.0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="dam_break_1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the FP64 and adjoint variants")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--profile-substeps", type=int, default=0,
                    help="run this many substeps of the workload once, untimed, and exit (for ncu captures)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"], help="precision of --profile-substeps")
    ap.add_argument("--profile-projection", action="store_true",
                    help="with --profile-substeps: then one gic_project call on the window's alpha_s (tol 1e-9)")
    ap.add_argument("--profile-window", action="store_true",
                    help="with --profile-substeps: the differentiable window (forward + backward) instead")
    ap.add_argument("--profile-direct", action="store_true",
                    help="with --profile-substeps: gic_sort + gic_substep every substep (no CUDA graph), so that "
                         "a profiler sees each kernel")
    return ap.parse_args()


# --------------------------------------------------------------------------- distributed plumbing

def dist_setup(args):
    """One process per GPU (torchrun env).  The ranks run independent replicas
    of the workload: the only communication is the barrier and the timing
    reduction (NCCL with GPUs, gloo otherwise)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, ws, device="cuda"):
    """Largest value over the ranks (the slowest rank's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, ms_per_rank, ws, device="cuda"):
    """Whole-job units per second: all ranks' units over the slowest rank's
    time (weak scaling of independent replicas)."""
    ms = max_over_ranks(ms_per_rank, ws, device)
    return ws * units_per_rank / (ms / 1000.0), ms


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- CPU oracle sample

def oracle_sample(prob, target_s, K_full):
    """Time the FP64 oracle on a bounded sample of the workload: the first m
    granules (the bottom of the column, contacts and walls included) for
    K_s substeps, sized for about target_s seconds."""
    import dataclasses

    import oracle

    def sub(m):
        return dataclasses.replace(prob, cell=prob.cell[:m], q=prob.q[:m], r=prob.r[:m], v=prob.v[:m])

    # calibrate on a small sample
    m = min(prob.n, 20000)
    t0 = time.perf_counter()
    oracle.run(sub(m), K=2)
    per = (time.perf_counter() - t0) / (2 * m)
    K_s = K_full
    m = int(min(prob.n, max(1000, target_s / (per * K_s))))
    if m < 1000:
        K_s = max(1, int(target_s / (per * 1000)))
        m = 1000
    t0 = time.perf_counter()
    oracle.run(sub(m), K=K_s)
    dt = time.perf_counter() - t0
    return {"value": m * K_s / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {m} granules of the {prob.n}-granule workload, {K_s} substeps, single-threaded FP64 C",
            "seconds": dt}


def run_reference(args, ws, rank):
    """--impl reference: the oracle is the reference arm (rank 0 only)."""
    if rank != 0:
        return
    import gic_inputs as gi

    prob = gi.make(args.workload)
    import dataclasses

    import oracle

    # bounded sample per step so W + K steps finish within a few minutes
    per_step_s = min(20.0, 150.0 / max(1, args.steps + args.warmup))
    m = min(prob.n, 20000)
    t0 = time.perf_counter()
    oracle.run(dataclasses.replace(prob, cell=prob.cell[:m], q=prob.q[:m], r=prob.r[:m], v=prob.v[:m]), K=2)
    per = (time.perf_counter() - t0) / (2 * m)
    K_s = prob.K
    m = int(min(prob.n, max(1000, per_step_s / (per * K_s))))
    sub = dataclasses.replace(prob, cell=prob.cell[:m], q=prob.q[:m], r=prob.r[:m], v=prob.v[:m])
    for _ in range(args.warmup):
        oracle.run(sub, K=1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(sub, K=K_s)
        times.append(time.perf_counter() - t0)
    ms = 1000 * statistics.mean(times)
    value = m * K_s / (ms / 1000)
    sample = f"first {m} granules of {prob.n}, {K_s} substeps per step, single-threaded FP64 C oracle"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": prob.name, "granules": prob.n, "grid": [prob.grid.nx, prob.grid.ny, prob.grid.nz],
                       "substeps_per_step": prob.K, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU arm

def run_gpu(args, ws, rank, local):
    import numpy as np
    import torch

    import gic_inputs as gi
    from paper_2504_00745_gb300 import gic
    from paper_2504_00745_gb300.window import Simulator

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob = gi.make(args.workload)
    n, K = prob.n, prob.K
    sim = Simulator.from_problem(prob, gic.GIC_FP32, dev)
    init = sim.A.clone()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2

    names = list(ALGO_BYTES)
    ev_acc = {k: [] for k in names}

    def one_step(probe=False):
        sim.load_state(init)  # the window's first substep builds the lists
        flush.zero_()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        sim.zero_transfer()
        for s in range(K):  # alpha_s at the final positions only (Alg. 1), F_s every substep (Alg. 2)
            last = s == K - 1
            if probe:
                sim.substep_probe(ev_acc, stream=stream, alpha=last)
            else:
                sim.substep(alpha=last, sums=last)
        end.record(stream)
        return start, end

    gic.gic_check_status(clear=True)
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    l0 = gic.launch_count()
    t_wall = time.perf_counter()
    evs = [one_step(probe=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - t_wall
    launches = gic.launch_count() - l0
    clk = clocks.stop()
    status = gic.gic_check_status(clear=True)
    ms = statistics.mean(s.elapsed_time(e) for s, e in evs)
    value, ms = job_throughput(n * K, ms, ws, dev)

    # per-entry-point durations inside the timed region -> roofline of the dominant one
    per_call = {k: statistics.mean(a.elapsed_time(b) for a, b in ev_acc[k]) for k in names if ev_acc[k]}
    dom = max(per_call, key=per_call.get)
    import math

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = algo_bytes(dom, K) * n / (per_call[dom] / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": NCU_TRAFFIC.get((prob.name, dom)), "kernel": dom,
                "peak_source": "measured" if peaks else "fallback",
                "per_call_ms": per_call,
                "per_call_frac": {k: algo_bytes(k, K) * n / (v / 1000.0) / 1e9 / hbm for k, v in per_call.items()},
                "algo_bytes_per_granule": {k: algo_bytes(k, K) for k in per_call}}

    # e2e through the C ABI with host buffers (copies inside the timed region)
    e2e = run_e2e(prob, sim, gic, torch, np, dev, stream, max(1, min(args.steps, 3)))

    variants = {}
    if not args.no_variants:
        # the consumer of this window's alpha_s: both projections on the 128^3 grid
        for tol in (1e-6, 1e-9):
            variants[f"projection_{prob.name}_tol{tol:g}"] = run_projection(prob, sim, gic, torch, dev, stream, tol)
        variants["fp64_fwd"] = run_fwd(prob, gic.GIC_FP64, gic, torch, dev, stream)
        for prec_name, prec in (("fp32", gic.GIC_FP32), ("fp64", gic.GIC_FP64)):
            variants[f"{prec_name}_adjoint_dam_break"] = run_adjoint(prob, prec, torch, dev)
            wprob = gi.make("diff_window_100k")
            variants[f"{prec_name}_adjoint_diff_window"] = run_adjoint(wprob, prec, torch, dev)
        del sim, init, flush
        torch.cuda.empty_cache()
        for wname in ("polydisperse_bed_8m", "scale_sweep_16m"):
            wp = gi.make(wname)
            for prec_name, prec in (("fp32", gic.GIC_FP32), ("fp64", gic.GIC_FP64)):
                variants[f"{prec_name}_fwd_{wname}"] = run_fwd(wp, prec, gic, torch, dev, stream)
            del wp

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (fixed-point positions, f64 alpha_s)", "data": "synthetic",
            "config": {"workload": prob.name, "granules": n, "grid": [prob.grid.nx, prob.grid.ny, prob.grid.nz],
                       "substeps_per_step": K, "dt_sub": prob.params.dt_sub, "precision": "fp32",
                       "schedule": "one fluid step: K gic_step calls (Morton sort only when the Verlet lists, skin "
                                   "0.15 r_max, are rebuilt; fused contact, G2P couple, integrate, P2G of F_s); "
                                   "alpha_s and sums at the final positions",
                       "l2": "flushed between steps (512 MB write), state reset to the initial packing",
                       "wall_s": wall},
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "device_status": status, "variants": variants}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(prob, args.cpu_seconds, K)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_e2e(prob, sim, gic, torch, np, dev, stream, steps):
    """The K-substep window through gic_window_forward_host: pinned host
    inputs -> device -> K substeps -> host outputs, per step."""
    n, K = prob.n, prob.K
    G, P = sim.grid, sim.params
    wsb = C.c_size_t(0)
    L = gic.lib()
    L.gic_window_host_workspace_size.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]
    rc = L.gic_window_host_workspace_size(C.byref(G), n, 0, C.byref(wsb))
    assert rc == 0, gic.last_error()
    ws = torch.empty(wsb.value, dtype=torch.uint8, device=dev)
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
    h_cell = pin(prob.cell, torch.int32)
    h_q = pin(prob.q.astype(np.int64), torch.int32)
    h_r = pin(prob.r, torch.float32)
    h_v = pin(prob.v, torch.float32)
    fields = [pin(a, torch.float32) for a in (prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)]
    nx, ny, nz = prob.grid.nx, prob.grid.ny, prob.grid.nz
    o_x = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    o_v = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    o_a = torch.empty(nx * ny * nz, dtype=torch.float64).pin_memory()
    o_fs = [torch.empty(m, dtype=torch.float32).pin_memory()
            for m in ((nx + 1) * ny * nz, nx * (ny + 1) * nz, nx * ny * (nz + 1))]
    o_s = torch.empty(2, dtype=torch.float64).pin_memory()
    fn = L.gic_window_forward_host
    fn.argtypes = [C.c_void_p] * 2 + [C.c_int64, C.c_int32] + [C.c_void_p] * 9 + [C.c_int32] + [C.c_void_p] * 8 + \
        [C.c_size_t, C.c_void_p]
    p = lambda t: C.c_void_p(t.data_ptr())

    def call():
        rc = fn(C.byref(G), C.byref(P), n, 0, p(h_cell), p(h_q), p(h_r), p(h_v), *[p(f) for f in fields], K, p(o_x),
                p(o_v), p(o_a), *[p(f) for f in o_fs], p(o_s), p(ws), ws.numel(), C.c_void_p(stream.cuda_stream))
        assert rc == 0, gic.last_error()

    call()  # warm-up
    times = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        call()
        times.append(time.perf_counter() - t0)
    h2d = sum(t.numel() * t.element_size() for t in [h_cell, h_q, h_r, h_v, *fields])
    d2h = sum(t.numel() * t.element_size() for t in [o_x, o_v, o_a, *o_fs, o_s])
    sec = statistics.mean(times)
    return {"value": n * K / sec, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": 1000 * sec, "api": "gic_window_forward_host (C ABI, pinned host buffers)"}


def run_adjoint(prob, prec, torch, dev, ckpt=10):
    """Forward window + backward (recompute from checkpoints every `ckpt`
    substeps + the adjoint kernels) of L = mean |x_K - target|^2, w.r.t. the
    initial velocities, c_drag and mu.  Reported per granule-substep."""
    import numpy as np

    from paper_2504_00745_gb300.window import GicWindow, Simulator

    if prob.target is None:
        rng = np.random.default_rng(7)
        prob.target = prob.positions() + rng.normal(0.0, 0.5 * float(prob.r.mean()), size=(prob.n, 3))
    sim = Simulator.from_problem(prob, prec, dev)
    init = sim.A.clone()
    target = torch.as_tensor(prob.target, dtype=torch.float64, device=dev)
    K = prob.K
    res = []
    for it in range(2):
        v0 = torch.tensor(prob.v, dtype=torch.float64, device=dev, requires_grad=True)
        c = torch.tensor(float(prob.params.c_drag), dtype=torch.float64, device=dev, requires_grad=True)
        mu = torch.tensor(float(prob.params.mu_fric), dtype=torch.float64, device=dev, requires_grad=True)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record()
        x = GicWindow.apply(v0, c, mu, sim, init, K, ckpt)
        loss = ((x - target) ** 2).sum(dim=1).mean()
        e1.record()
        loss.backward()
        e2.record()
        torch.cuda.synchronize()
        if it > 0:
            res.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
    fwd_ms, bwd_ms = res[-1]
    units = prob.n * K
    return {"value": units / (bwd_ms / 1000), "unit": UNIT, "what": "backward incl. recompute",
            "fwd_ms": fwd_ms, "bwd_ms": bwd_ms, "fwd_plus_bwd_value": units / ((fwd_ms + bwd_ms) / 1000),
            "workload": prob.name, "granules": prob.n, "substeps": K, "ckpt_every": ckpt,
            "dtype": "f32" if prec == 0 else "f64"}


def run_fwd(prob, prec, gic, torch, dev, stream, steps=2, warmup=1):
    """The forward window of a workload on one precision path, `warmup`
    untimed and `steps` timed windows, each from the initial packing after a
    512 MB L2 flush; per-entry-point mean durations from events around each
    call."""
    from paper_2504_00745_gb300.window import Simulator

    sim = Simulator.from_problem(prob, prec, dev)
    init = sim.A.clone()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    K = prob.K
    res = []
    ev_acc = {k: [] for k in ALGO_BYTES}
    gic.gic_check_status(clear=True)
    for it in range(warmup + steps):
        sim.load_state(init)  # the window's first substep builds the lists
        flush.zero_()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        sim.zero_transfer()
        for k in range(K):
            last = k == K - 1
            if it >= warmup:
                sim.substep_probe(ev_acc, stream=stream, alpha=last)
            else:
                sim.substep(alpha=last, sums=last)
        e.record(stream)
        torch.cuda.synchronize()
        if it >= warmup:
            res.append(s.elapsed_time(e))
        elif gic.gic_check_status(clear=False):
            # granules left the domain or crossed cells too fast: the timing
            # would not be of this workload
            out = {"skipped": f"device status {gic.gic_check_status(clear=True)} after the warm-up window",
                   "workload": prob.name, "dtype": "f32" if prec == 0 else "f64"}
            del sim, init, flush
            torch.cuda.empty_cache()
            return out
    status = gic.gic_check_status(clear=True)
    ms = statistics.mean(res)
    per_call = {k: statistics.mean(a.elapsed_time(b) for a, b in v) for k, v in ev_acc.items() if v}
    out = {"value": prob.n * K / (ms / 1000), "unit": UNIT, "ms_per_step": ms, "dtype": "f32" if prec == 0 else "f64",
           "workload": prob.name, "granules": prob.n, "substeps": K, "steps": steps, "per_call_ms": per_call,
           "device_status": status}
    del sim, init, flush
    torch.cuda.empty_cache()
    return out


# bytes per fine cell of one multigrid-preconditioned CG iteration of
# gic_project (4 B values, each array read or written once per pass): on the
# fine level four red-black half sweeps (104), the residual restriction (20),
# the interpolation (9), rho = r . z (8), the direction fused with y = A d
# (28) and the updates (24); the coarser levels add about an eighth of the
# fine level's V-cycle passes (19)
PROJ_CG_BYTES = 212


def run_projection(prob, sim, gic, torch, dev, stream, tol, reps=3):
    """gic_project (velocity and density projections, Sec. 5.1) on the
    workload's grid with alpha_s from the simulator's last window (its final
    positions), alpha_f* = the workload's fluid fraction field, v* = its face
    velocities, dt = the fluid step, the top side open.  Time per call (both
    solves) with CUDA events on `stream`, the solver's counts, and the CG
    iterations' bytes over the whole call's time."""
    import ctypes as C

    g = prob.grid
    n = g.nx * g.ny * g.nz
    grid = gic.GicGrid(g.nx, g.ny, g.nz, 1, float(g.dx), (C.c_double * 3)(0, 0, 0))
    star = torch.as_tensor(prob.alpha_f, dtype=torch.float32, device=dev)
    u, v, w = sim.fluid.u, sim.fluid.v, sim.fluid.w
    p1 = torch.empty(n, dtype=torch.float64, device=dev)
    p2 = torch.empty_like(p1)
    vo = [torch.empty_like(f) for f in (u, v, w)]
    do = [torch.empty_like(f) for f in (u, v, w)]
    ws = torch.empty(gic.gic_project_workspace_size(grid), dtype=torch.uint8, device=dev)
    pp = gic.make_proj_params(prob.params.dt_fluid, prob.params.rho_f, (0, 0, 0, 0, 0, 1), tol=tol)
    times, info = [], None
    for rep in range(reps + 1):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        info = gic.gic_project(grid, pp, sim.alpha_s, star, u, v, w, p1, p2, vo, do, ws=ws, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        if rep:
            times.append(a.elapsed_time(b))
    ms = statistics.mean(times) if times else float("nan")
    iters = int(info.inner[0] + info.inner[1])
    gbs = PROJ_CG_BYTES * n * iters / (ms / 1000) / 1e9
    return {"ms_per_call": ms, "cells": n, "tol": tol, "outer": list(info.outer), "inner": list(info.inner),
            "converged": list(info.converged), "rel_residual": [float(x) for x in info.rel_residual],
            "cg_algo_bytes_per_cell_iter": PROJ_CG_BYTES, "cg_achieved_gbs_over_call": gbs,
            "workload": prob.name}


def run_profile(args):
    """N substeps of the workload, nothing else (the command ncu wraps); with
    --profile-window the loss gradient of an N-substep window instead."""
    import numpy as np
    import torch

    import gic_inputs as gi
    from paper_2504_00745_gb300 import gic
    from paper_2504_00745_gb300.window import GicWindow, Simulator

    prob = gi.make(args.workload)
    prec = gic.GIC_FP32 if args.precision == "fp32" else gic.GIC_FP64
    sim = Simulator.from_problem(prob, prec)
    if args.profile_window:
        rng = np.random.default_rng(7)
        target = torch.as_tensor(prob.positions() + rng.normal(0.0, 0.5 * float(prob.r.mean()), size=(prob.n, 3)),
                                 device=sim.device)
        v0 = torch.tensor(prob.v, dtype=torch.float64, device=sim.device, requires_grad=True)
        c = torch.tensor(float(prob.params.c_drag), dtype=torch.float64, device=sim.device, requires_grad=True)
        mu = torch.tensor(float(prob.params.mu_fric), dtype=torch.float64, device=sim.device, requires_grad=True)
        x = GicWindow.apply(v0, c, mu, sim, sim.A.clone(), args.profile_substeps, 10)
        ((x - target) ** 2).sum(dim=1).mean().backward()
    else:
        sim.run(args.profile_substeps, sort_every=args.profile_direct)
    extra = {}
    if args.profile_projection:
        out = run_projection(prob, sim, gic, torch, sim.device, torch.cuda.current_stream(), 1e-9, reps=0)
        extra = {"projection_outer": out["outer"], "projection_inner": out["inner"]}
    torch.cuda.synchronize()
    st = gic.gic_check_status()
    print(json.dumps({"profile_substeps": args.profile_substeps, "workload": prob.name, "precision": args.precision,
                      "device_status": st, "launches": gic.launch_count(), **extra}))


def main():
    args = parse()
    if args.profile_substeps > 0:
        run_profile(args)
        return
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_gpu(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
