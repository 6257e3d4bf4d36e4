"""Benchmark of the granule-grid coupling substep on GB300.

One step = one fluid step: a window of K substeps of Alg. 2 (Morton sort on
Verlet-list rebuilds, fused contact + G2P couple + integrate + P2G of F_s,
alpha_s and the conservation sums at the final positions) over the largest
single-GPU workload: the 16,000,000-granule precision and scale sweep on a
384^3 grid (20 substeps of 1e-5 s, FP32 state with exact fixed-point alpha_s),
starting every step from the same seeded packing.  The metric is
granule-substeps per second.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead, on all host cores, on bounded sub-boxes of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "granule-substeps/s fwd & adjoint, FP32 vs FP64 on 1 GB300; % HBM roofline"
UNIT = "granule-substeps/s"
# algorithmic bytes per granule-substep of each entry point (FP32 path):
# what the method must move, 12 B per 3-vector, state = 36 B.  P2G scatters
# F_s from the old positions every substep (cell + pos 20 B, f_ex 12 B) and
# alpha_s from the new ones once per fluid step (20 B more on the last
# substep).  The fused substep (contact, G2P, integrate, P2G after the sort)
# is charged 90 B, the per-unit figure for a fused single-pass substep:
# the sorted state in and the next state out
# (72 B) plus the granule's share of the fluid samples and F_s deposits it
# touches.  The FP64 path moves twice the floats of every record (2x); the
# adjoint of the fused substep reads the state and the upstream position and
# velocity gradients and writes the downstream ones (36 + 32 + 32 = 100 B).
ALGO_BYTES = {"gic_sort": 88, "gic_contact": 48, "gic_g2p_couple": 65, "gic_integrate": 120, "gic_p2g": 32,
              "gic_substep": 90, "gic_step": 90, "gic_substep_adj": 100}
P2G_ALPHA_BYTES = 20
# DRAM bytes (read + write) of one call of the dominant entry point, averaged
# over the window's calls as the duration is: on the sweep 1 call that sorts
# and rebuilds the lists (7.08 GB), 18 that keep them (2.41 GB each: the
# decision kernel + k_substep) and the last, which also forms alpha_s (3.76
# GB), from a graph-level ncu capture of the current kernels (ncu flushes the
# caches first); per workload (None where no capture of the current kernels
# exists)
NCU_TRAFFIC = {("scale_sweep_16m", "gic_step"): (7.077e9 + 18 * 2.409e9 + 3.760e9) / 20}


def algo_bytes(name, K, fp64=False):
    """Algorithmic bytes per granule of one call of `name`, averaged over a
    K-substep window (FP64 path: twice the FP32 figure)."""
    b = ALGO_BYTES[name] + (P2G_ALPHA_BYTES / K if name in ("gic_p2g", "gic_substep", "gic_step") else 0.0)
    return 2.0 * b if fp64 else b


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="scale_sweep_16m")
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
    ap.add_argument("--profile-granules", type=int, default=0,
                    help="with --profile-substeps: the workload's generator at this many granules (the same lattice "
                         "and grid, a thinner bed), for captures that must stay small")
    ap.add_argument("--profile-build", action="store_true",
                    help="with --profile-substeps: instead of substeps, that many list builds of the sorted state "
                         "(gic_sort + gic_neighbors_build), for a capture of the staged build")
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

def crop(prob, start, m):
    """Granules start .. start + m - 1 of a workload as a problem of its own
    on the smallest block of the workload's MAC grid that holds them with two
    cells to spare (same dx, origin moved, fields cut out): the oracle then
    spends its time on these granules, not on zeroing the full grid."""
    import dataclasses

    import gic_inputs as gi

    g = prob.grid
    k = g.k_contact
    cell = prob.cell[start:start + m]
    mac = cell // k
    lo = np.maximum(mac.min(0) - 2, 0)
    hi = np.minimum(mac.max(0) + 3, np.array([g.nx, g.ny, g.nz]))
    n3 = hi - lo
    sub = gi.Grid(int(n3[0]), int(n3[1]), int(n3[2]), g.dx,
                  tuple(float(g.origin[a] + lo[a] * g.dx) for a in range(3)), k)

    def cut(f, ext):  # MAC array with ext extra samples per axis, x fastest
        a = np.asarray(f).reshape(g.nz + ext[2], g.ny + ext[1], g.nx + ext[0])
        return np.ascontiguousarray(a[lo[2]:hi[2] + ext[2], lo[1]:hi[1] + ext[1], lo[0]:hi[0] + ext[0]]).ravel()

    return dataclasses.replace(prob, grid=sub, cell=(cell - lo * k).astype(prob.cell.dtype), q=prob.q[start:start + m],
                               r=prob.r[start:start + m], v=prob.v[start:start + m], u=cut(prob.u, (1, 0, 0)),
                               vf=cut(prob.vf, (0, 1, 0)), wf=cut(prob.wf, (0, 0, 1)), p=cut(prob.p, (0, 0, 0)),
                               alpha_f=cut(prob.alpha_f, (0, 0, 0)), target=None)


def oracle_rate(prob, target_s, threads):
    """The FP64 oracle (single-threaded C, as it stands) on `threads` host
    threads at once, each running its own cropped sub-box of consecutive
    granules of the workload for the workload's K substeps (the C calls run
    without the interpreter lock), sized so that each takes about target_s
    seconds.  Returns (granule-substeps/s over the wall time, sample text)."""
    import oracle

    K = prob.K
    m0 = min(prob.n, 4000)
    t0 = time.perf_counter()
    oracle.run(crop(prob, 0, m0), K=1)
    per = (time.perf_counter() - t0) / m0  # seconds per granule-substep, small sample
    m = int(min(prob.n // max(1, threads), max(1000, target_s / (per * K))))
    subs = [crop(prob, t * m, m) for t in range(threads)]
    out = [None] * threads

    def work(t):
        out[t] = oracle.run(subs[t], K=K)["status"]

    ths = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
    t0 = time.perf_counter()
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    wall = time.perf_counter() - t0
    sample = (f"{threads} sub-boxes of {m} consecutive granules of the {prob.n}-granule workload (each on its own "
              f"block of the MAC grid), {K} substeps each, one FP64 C oracle per host thread")
    return threads * m * K / wall, sample, wall


def oracle_sample(prob, target_s, others=None):
    """cpu_baseline: the oracle on all host cores, and on one; with `others`
    (problems by workload name), also on the other configurations."""
    cores = os.cpu_count() or 1
    v_all, sample, wall = oracle_rate(prob, target_s, cores)
    v_one, sample1, wall1 = oracle_rate(prob, target_s / 2, 1)
    out = {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample, "seconds": wall,
           "one_core": {"value": v_one, "cores": 1, "sample": sample1, "seconds": wall1}}
    if others is not None:
        out["configs"] = oracle_configs(others, cores)
    return out


# the oracle on the other configurations: (workload, granules timed; None = all)
ORACLE_CONFIGS = (("plain_fp64_8k", None), ("diff_window_100k", None), ("dam_break_1m", 100_000),
                  ("polydisperse_bed_8m", 50_000))


def oracle_split_rate(prob, m, threads):
    """The oracle on the first m granules of a workload (in the generator's
    order), split into `threads` runs of consecutive granules, each on its own
    block of the MAC grid on its own host thread, for the workload's K
    substeps.  Returns (granule-substeps/s over the wall time, wall seconds)."""
    import oracle

    K = prob.K
    chunk = -(-m // threads)
    subs = [crop(prob, t * chunk, min(chunk, m - t * chunk)) for t in range(threads) if t * chunk < m]

    def work(sub):
        oracle.run(sub, K=K)

    ths = [threading.Thread(target=work, args=(sub,)) for sub in subs]
    t0 = time.perf_counter()
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    wall = time.perf_counter() - t0
    return m * K / wall, wall


def oracle_configs(problems, cores):
    """The oracle's rate on each configuration of ORACLE_CONFIGS: the whole
    problem (or its first granules, a block of consecutive ones) on one core,
    and the same granules split over all cores (the runs then miss the
    contacts across their cuts: a timing, not a result)."""
    import gic_inputs as gi

    out = {}
    for name, m in ORACLE_CONFIGS:
        try:
            prob = problems[name] if name in problems else gi.make(name)
            mm = prob.n if m is None else min(m, prob.n)
            one, w1 = oracle_split_rate(prob, mm, 1)
            allc, wa = oracle_split_rate(prob, mm, cores)
            out[name] = {"granules": mm, "of": prob.n, "substeps": prob.K, "one_core": one, "one_core_s": w1,
                         "all_cores": allc, "all_cores_s": wa, "cores": cores,
                         "sample": "the whole problem" if mm == prob.n else
                         f"the first {mm} granules (consecutive in the generator's order) on their block of the grid"}
        except Exception as e:  # a timing leg: never the benchmark line's failure
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    return out


def run_reference(args, ws, rank):
    """--impl reference: the oracle is the reference arm (rank 0 only), on
    all host cores, a bounded sample of the workload per step."""
    if rank != 0:
        return
    import gic_inputs as gi

    prob = gi.make(args.workload)
    cores = os.cpu_count() or 1
    per_step_s = min(20.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_rate(prob, min(2.0, per_step_s), cores)
    vals, walls, sample = [], [], ""
    for _ in range(args.steps):
        v, sample, wall = oracle_rate(prob, per_step_s, cores)
        vals.append(v)
        walls.append(wall)
    value = statistics.mean(vals)
    ms = 1000 * statistics.mean(walls)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": prob.name, "granules": prob.n, "grid": [prob.grid.nx, prob.grid.ny, prob.grid.nz],
                       "substeps_per_step": prob.K, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU arm

def peaks_file():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def roofline_of(per_call_ms, n, K, fp64, hbm, traffic=None, source="measured"):
    """HBM roofline of the dominant entry point of a window: its algorithmic
    bytes per granule x n over its mean call duration."""
    dom = max(per_call_ms, key=per_call_ms.get)
    achieved = algo_bytes(dom, K, fp64) * n / (per_call_ms[dom] / 1000.0) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "kernel": dom, "peak_source": source, "per_call_ms": per_call_ms,
            "per_call_frac": {k: algo_bytes(k, K, fp64) * n / (v / 1000.0) / 1e9 / hbm for k, v in per_call_ms.items()},
            "algo_bytes_per_granule": {k: algo_bytes(k, K, fp64) for k in per_call_ms}}


def run_gpu(args, ws, rank, local):
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
    peaks, peak_source = peaks_file()
    hbm = float(peaks.get("hbm_gbs", 6800.0))

    ev_acc = {k: [] for k in ALGO_BYTES}

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
    per_call = {k: statistics.mean(a.elapsed_time(b) for a, b in v) for k, v in ev_acc.items() if v}
    roofline = roofline_of(per_call, n, K, False, hbm, NCU_TRAFFIC.get((prob.name, "gic_step")), peak_source)

    # e2e through the C ABI with host buffers (copies inside the timed region)
    e2e = run_e2e(prob, sim, gic, torch, np, dev, stream, max(1, min(args.steps, 5)))
    # what the exact alpha_s costs: the same state's alpha_s with fixed-point limbs and with FP64 atomics
    alpha_cost = run_alpha_cost(prob, sim, gic, torch, stream)

    variants = {"alpha_s_exact_vs_fp64_atomics": alpha_cost}
    oracle_probs = {}  # the other configurations' problems, for the oracle's timings after the GPU work
    del sim, init, flush
    torch.cuda.empty_cache()
    if not args.no_variants:
        variants["fma_rate"] = run_fma_probe(gic, torch, dev, stream)
        fp64_flops = variants["fma_rate"]["fp64_tflops"]
        variants[f"fp64_fwd_{prob.name}"] = run_fwd(prob, gic.GIC_FP64, gic, torch, dev, stream, hbm)
        dam = gi.make("dam_break_1m")
        oracle_probs["dam_break_1m"] = dam
        for prec_name, prec in (("fp32", gic.GIC_FP32), ("fp64", gic.GIC_FP64)):
            variants[f"{prec_name}_fwd_dam_break_1m"] = run_fwd(dam, prec, gic, torch, dev, stream, hbm,
                                                               keep_for_projection=(prec == gic.GIC_FP32))
        dsim = variants["fp32_fwd_dam_break_1m"].pop("_sim")
        for tol in (1e-6, 1e-9):
            variants[f"projection_dam_break_1m_tol{tol:g}"] = run_projection(dam, dsim, gic, torch, dev, stream, tol)
        del dsim
        torch.cuda.empty_cache()
        for prec_name, prec in (("fp32", gic.GIC_FP32), ("fp64", gic.GIC_FP64)):
            variants[f"{prec_name}_adjoint_kernel_dam_break_1m"] = run_adjoint_kernel(dam, prec, gic, torch, dev,
                                                                                    stream, hbm)
            variants[f"{prec_name}_adjoint_dam_break_1m"] = run_adjoint(dam, prec, torch, dev)
            wprob = oracle_probs["diff_window_100k"] = gi.make("diff_window_100k")
            variants[f"{prec_name}_adjoint_diff_window_100k"] = run_adjoint(wprob, prec, torch, dev)
        del dam
        wp = oracle_probs["polydisperse_bed_8m"] = gi.make("polydisperse_bed_8m")
        for prec_name, prec in (("fp32", gic.GIC_FP32), ("fp64", gic.GIC_FP64)):
            variants[f"{prec_name}_fwd_polydisperse_bed_8m"] = run_fwd(wp, prec, gic, torch, dev, stream, hbm,
                                                                      contacts=(prec == gic.GIC_FP32))
        del wp
        for key, v in variants.items():  # the FP64 path against the FP64 pipe: its share of the measured FMA rate
            if key.startswith("fp64_fwd") and "value" in v:
                v["fp64_fma_peak_tflops"] = fp64_flops

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (fixed-point positions, exact f64 alpha_s)", "data": "synthetic",
            "config": {"workload": prob.name, "granules": n, "grid": [prob.grid.nx, prob.grid.ny, prob.grid.nz],
                       "substeps_per_step": K, "dt_sub": prob.params.dt_sub, "precision": "fp32",
                       "schedule": "one fluid step: K gic_step calls (Morton sort only when the Verlet lists, skin "
                                   "0.05 r_max, are rebuilt; fused contact, G2P couple, integrate, P2G of F_s); "
                                   "alpha_s and sums at the final positions",
                       "l2": "flushed between steps (512 MB write); the inputs (16M granules, 1.1 GB of fluid fields) "
                             "exceed L2 anyway; state reset to the initial packing",
                       "wall_s": wall},
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "device_status": status, "variants": variants}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(prob, args.cpu_seconds, None if args.no_variants else oracle_probs)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_alpha_cost(prob, sim, gic, torch, stream, reps=5):
    """alpha_s of the simulator's current FP32 state (after the window): the
    library's exact path (gic_p2g with alpha_s only: 64-bit fixed-point
    deposits, integer atomics, the exact totals, the conversion) against
    the same deposits with plain FP64 atomics (gic_p2g_alpha_atomic64); per
    call, CUDA events on the stream; and the largest difference."""
    import ctypes as C

    L = gic.lib()
    L.gic_p2g_alpha_atomic64.argtypes = [C.c_void_p] * 4
    L.gic_p2g_alpha_atomic64.restype = C.c_int
    a64 = torch.empty_like(sim.alpha_s)
    st = sim.A.struct()

    def exact():
        gic.gic_p2g(sim.grid, sim.params, sim.A, sim.A, None, sim.alpha_s, (None, None, None), sim.sums, stream)

    def atomic():
        rc = L.gic_p2g_alpha_atomic64(C.byref(sim.grid), C.byref(st), C.c_void_p(a64.data_ptr()),
                                      C.c_void_p(stream.cuda_stream))
        assert rc == 0, gic.last_error()

    out = {}
    for name, fn in (("exact_fixed_point", exact), ("fp64_atomics", atomic)):
        fn()
        times = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        out[f"{name}_ms"] = statistics.mean(times)
    out["max_abs_diff"] = float((sim.alpha_s - a64).abs().max().item())
    out["exact_over_atomics"] = out["exact_fixed_point_ms"] / out["fp64_atomics_ms"]
    out["workload"] = prob.name
    out["granules"] = prob.n
    out["note"] = "exact: order-independent, sum_c alpha_s = sum_i S_i as integers; atomics: order-dependent"
    return out


def run_fma_probe(gic, torch, dev, stream):
    """FMA rate of this GPU, FP32 and FP64 (gic_probe_fma, CUDA events)."""
    import ctypes as C

    L = gic.lib()
    L.gic_probe_fma.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    L.gic_probe_fma.restype = C.c_int
    blocks = 152 * 8
    sink = torch.empty(blocks * 256, dtype=torch.float64, device=dev)
    out = {}
    for name, prec, iters in (("fp32", gic.GIC_FP32, 8192), ("fp64", gic.GIC_FP64, 512)):
        fm = C.c_int64(0)
        times = []
        for rep in range(4):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rc = L.gic_probe_fma(prec, blocks, iters, C.c_void_p(sink.data_ptr()), C.byref(fm),
                                 C.c_void_p(stream.cuda_stream))
            b.record(stream)
            assert rc == 0, gic.last_error()
            torch.cuda.synchronize()
            if rep:
                times.append(a.elapsed_time(b))
        out[f"{name}_tflops"] = 2.0 * fm.value / (min(times) / 1000.0) / 1e12
        out[f"{name}_ms"] = min(times)
    out["what"] = "8 independent FMA chains per thread, 1216 CTAs of 256 threads; 2 flops per FMA; best of 3"
    return out


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

    for _ in range(2):  # warm-up (graphs instantiated, kernels loaded)
        call()
    times = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        call()
        times.append(time.perf_counter() - t0)
    h2d = sum(t.numel() * t.element_size() for t in [h_cell, h_q, h_r, h_v, *fields])
    d2h = sum(t.numel() * t.element_size() for t in [o_x, o_v, o_a, *o_fs, o_s])
    # the median call: the copies run over the host's memory, which other jobs on the machine share, and single
    # calls have taken 2-3x the others (every call is listed)
    sec = statistics.median(times)
    link = host_link_rates(torch, o_a, dev, stream)
    io_ms = 1e-6 * (h2d / link["h2d_gbs"] + d2h / link["d2h_gbs"])
    link["io_ms_at_link_rate"] = io_ms
    link["what"] = ("one pinned-host <-> device copy of %d MB on the call's stream, best of 3, after the timed calls; "
                    "io_ms_at_link_rate = h2d bytes / h2d rate + d2h bytes / d2h rate" % (o_a.numel() * 8 >> 20))
    return {"value": n * K / sec, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": 1000 * sec, "ms_per_call": [1000 * t for t in times],
            "ms_mean": 1000 * statistics.mean(times), "statistic": "median of the timed calls",
            "api": "gic_window_forward_host (C ABI, pinned host buffers)", "host_link": link}


def host_link_rates(torch, h, dev, stream):
    """Copy rate of the host link in each direction (GB/s): `h` (pinned) to a
    device buffer and back, timed with CUDA events on `stream`."""
    d = torch.empty(h.shape, dtype=h.dtype, device=dev)
    nbytes = h.numel() * h.element_size()
    out = {}
    with torch.cuda.stream(stream):
        for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
            best = float("inf")
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream)
                dst.copy_(src, non_blocking=True)
                b.record(stream)
                b.synchronize()
                best = min(best, a.elapsed_time(b))
            out[name] = nbytes / (best * 1e6)
    del d
    return out


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


def contacts_per_granule(sim, gic, torch):
    """Contact pairs per granule of the simulator's current state (sorted
    into B for the count), i.e. the contact rate per substep."""
    counts = torch.zeros(sim.n, dtype=torch.int32, device=sim.device)
    gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
    gic.gic_contact_pairs(sim.grid, sim.B, sim.table, counts=counts)
    return float(counts.sum().item()) / 2.0 / max(1, sim.n)


def run_fwd(prob, prec, gic, torch, dev, stream, hbm, steps=2, warmup=1, keep_for_projection=False, contacts=False):
    """The forward window of a workload on one precision path, `warmup`
    untimed and `steps` timed windows, each from the initial packing after a
    512 MB L2 flush; per-entry-point mean durations from events around each
    call, and the roofline of the dominant one."""
    from paper_2504_00745_gb300.window import Simulator

    sim = Simulator.from_problem(prob, prec, dev)
    init = sim.A.clone()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    K = prob.K
    res = []
    ev_acc = {k: [] for k in ALGO_BYTES}
    gic.gic_check_status(clear=True)
    c0 = contacts_per_granule(sim, gic, torch) if contacts else None
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
           "workload": prob.name, "granules": prob.n, "substeps": K, "steps": steps,
           "roofline": roofline_of(per_call, prob.n, K, prec != 0, hbm), "device_status": status}
    if contacts:
        out["contacts_per_granule"] = {"initial": c0, "final": contacts_per_granule(sim, gic, torch)}
    if keep_for_projection:
        out["_sim"] = sim
    else:
        del sim
    del init, flush
    torch.cuda.empty_cache()
    return out


def run_adjoint_kernel(prob, prec, gic, torch, dev, stream, hbm, reps=10):
    """gic_substep_adj alone (the fused adjoint: integrate, G2P and contact
    adjoints of one substep over the Verlet lists; with the displacement
    check it runs first) on the workload's state after one substep, random
    upstream gradients; mean call time and its roofline."""
    from paper_2504_00745_gb300.window import Simulator

    sim = Simulator.from_problem(prob, prec, dev)
    sim.substep(alpha=False, transfer=False, sums=False)  # builds the lists; A is in their order
    F = sim.fluid
    g = torch.Generator(device=dev).manual_seed(3)
    real = torch.float32 if prec == 0 else torch.float64
    gpo, gvo = (torch.randn((prob.n, 4), generator=g, device=dev, dtype=real) for _ in range(2))
    gpi, gvi = gic.vec4(prob.n, prec, dev), gic.vec4(prob.n, prec, dev)
    gs = torch.zeros(2, dtype=torch.float64, device=dev)

    def call():
        gic.gic_substep_adj(sim.grid, sim.params, sim.A, None, sim.table, sim.nb, F.u, F.v, F.w, F.p, F.alpha_f, gpo,
                            gvo, None, gpi, gvi, gs[0:1], gs[1:2], stream)

    call()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call()
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    builds = sim.nb.builds()
    status = gic.gic_check_status(clear=True)
    ms = statistics.mean(times)
    out = {"value": prob.n / (ms / 1000), "unit": UNIT, "ms_per_call": ms, "dtype": "f32" if prec == 0 else "f64",
           "workload": prob.name, "granules": prob.n, "list_builds": builds,
           "roofline": roofline_of({"gic_substep_adj": ms}, prob.n, prob.K, prec != 0, hbm), "device_status": status}
    del sim
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

    prob = gi.make(args.workload, **({"n": args.profile_granules} if args.profile_granules else {}))
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
    elif args.profile_build:
        for _ in range(args.profile_substeps):
            gic.gic_sort(sim.grid, sim.A, sim.B, sim.perm, sim.table, sim.ws)
            gic.gic_neighbors_reset(sim.nb)
            gic.gic_neighbors_build(sim.grid, sim.B, sim.table, sim.nb)
    else:
        sim.run(args.profile_substeps, sort_every=args.profile_direct)
    extra = {}
    if args.profile_projection:
        out = run_projection(prob, sim, gic, torch, sim.device, torch.cuda.current_stream(), 1e-9, reps=0)
        extra = {"projection_outer": out["outer"], "projection_inner": out["inner"]}
    torch.cuda.synchronize()
    st = gic.gic_check_status()
    print(json.dumps({"profile_substeps": args.profile_substeps, "workload": prob.name, "granules": prob.n,
                      "precision": args.precision,
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
