"""K-substep windows of the granule-grid coupling (Alg. 2 SandSubstep) on one GPU.

`Simulator` owns the device buffers of one problem and runs substeps through
the C ABI (sort -> contact -> G2P couple -> integrate -> P2G); `GicWindow` is
the torch.autograd.Function that runs a window forward with a checkpoint
every `ckpt` substeps and, backward, recomputes each segment from its
checkpoint and walks the hand-written adjoints in reverse.

Everything numeric runs in libgic.so kernels; torch provides memory and
streams only.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import torch

from . import gic
from .gic import GIC_FP32, GIC_FP64, State


@dataclass
class DeviceFluid:
    u: torch.Tensor
    v: torch.Tensor
    w: torch.Tensor
    p: torch.Tensor
    alpha_f: torch.Tensor


# default Verlet skin in units of the largest radius (measured on the 16M sweep,
# the dam break and the bed: 0.15 -> 0.05 shortens the rows; at 0.03 the sweep
# rebuilds within its fluid step)
SKIN_OVER_RMAX = 0.05


class Simulator:
    """Device buffers + substep loop for one problem.

    grid / params: objects with the fields of GicGrid / GicParams (e.g.
    gic_inputs.Grid / Params).  The initial state comes from the canonical
    encoding (cell int32 [n,3], q uint32 [n,3], r float32 [n], v float32 [n,3])
    as host or device tensors.  verlet_skin (metres): contact through Verlet
    lists with that skin (gic_contact_verlet, cap partners per granule)
    instead of walking the cell table every substep (gic_contact); with
    lists and fused, a substep is one gic_step from A into A2 (sort into B
    only on list rebuilds, then the fused substep), after which A and A2
    swap: A is always the current state.  A state written into A from
    outside goes through load_state (or set_state), which makes the next
    gic_step rebuild the lists.
    """

    def __init__(self, grid, params, n: int, precision: int = GIC_FP32, device="cuda",
                 verlet_skin: Optional[float] = None, verlet_cap: int = 48, fused: bool = True):
        self.grid_obj = grid
        self.params_obj = params
        self.grid = gic.make_grid(grid)
        self.params = gic.make_params(params)
        self.n = int(n)
        self.precision = precision
        self.device = torch.device(device)
        self.real = torch.float32 if precision == GIC_FP32 else torch.float64
        n = self.n
        # FP32 states carry the float position copy that the contact pre-tests read
        self.A = State.empty(n, precision, device, with_posf=True)
        self.A2 = State.empty(n, precision, device, with_posf=True)  # gic_step's next state
        self.B = State.empty(n, precision, device, with_posf=True)  # the sorted state
        self.perm = torch.empty(n, dtype=torch.int32, device=device)
        self.table = gic.new_cell_table(self.grid, device)
        self.ws = gic.new_workspace(self.grid, n, precision, device)
        self.F_c = gic.vec4(n, precision, device)
        self.F_fl = gic.vec4(n, precision, device)
        self.a_f = gic.vec4(n, precision, device)
        self.f_ex = gic.vec4(n, precision, device)
        self.alpha_f_p = torch.zeros(n, dtype=self.real, device=device)
        nx, ny, nz = grid.nx, grid.ny, grid.nz
        self.alpha_s = torch.zeros(nx * ny * nz, dtype=torch.float64, device=device)
        self.Fs = (torch.zeros((nx + 1) * ny * nz, dtype=self.real, device=device),
                   torch.zeros(nx * (ny + 1) * nz, dtype=self.real, device=device),
                   torch.zeros(nx * ny * (nz + 1), dtype=self.real, device=device))
        self.sums = torch.zeros(2, dtype=torch.float64, device=device)
        self.fluid: Optional[DeviceFluid] = None
        self.nb: Optional[gic.Neighbors] = None
        self.fused = fused
        self.lists_current = False  # A is the last gic_step's result and the lists are those it used
        if verlet_skin is not None:
            self.nb = gic.Neighbors(n, precision, cap=verlet_cap, skin=verlet_skin, device=device)
            gic.gic_neighbors_reset(self.nb)

    # ------------------------------------------------------------ inputs
    def set_fluid(self, u, v, w, p, alpha_f):
        conv = lambda a: torch.as_tensor(a).to(device=self.device, dtype=self.real).contiguous()
        self.fluid = DeviceFluid(conv(u), conv(v), conv(w), conv(p), conv(alpha_f))

    def set_state(self, cell_xyz, q, r, v, stream=None):
        dev = lambda a, dt: torch.as_tensor(a).to(device=self.device, dtype=dt).contiguous()
        q64 = torch.as_tensor(q).to(torch.int64)
        qi = q64.to(torch.int32)  # the 30-bit fractions fit in int32
        gic.gic_pack(self.grid, dev(cell_xyz, torch.int32), dev(qi, torch.int32), dev(r, torch.float32),
                     dev(v, torch.float32), self.A, stream)
        if self.nb is not None:  # radii may have changed
            gic.gic_neighbors_reset(self.nb, stream)
        self.lists_current = False

    def load_state(self, src: State):
        """Copies a state (e.g. a saved initial state) into A; the next
        gic_step rebuilds the lists."""
        _copy_state(self.A, src)
        self.lists_current = False

    @classmethod
    def from_problem(cls, prob, precision=GIC_FP32, device="cuda", verlet: bool = True, fused: bool = True,
                     skin: Optional[float] = None):
        """Simulator of a gic_inputs.Problem; verlet: Verlet lists with a skin
        of 0.05 r_max unless given (48 partners per granule, 96 when radii
        vary by more than 1.5x).  The skin only trades list length against
        rebuild frequency -- every granule's displacement is checked against
        skin / 2, so the contacts are exact for any skin; 0.05 r_max keeps one
        build per fluid step on every workload here and the rows short."""
        cap = None
        if verlet and prob.n > 0:
            r = prob.r
            skin = SKIN_OVER_RMAX * float(r.max()) if skin is None else float(skin)
            cap = 48 if float(r.max()) <= 1.5 * float(r.min()) else 96
        else:
            skin = None
        sim = cls(prob.grid, prob.params, prob.n, precision, device, verlet_skin=skin, verlet_cap=cap or 48,
                  fused=fused)
        sim.set_fluid(prob.u, prob.vf, prob.wf, prob.p, prob.alpha_f)
        sim.set_state(prob.cell, prob.q, prob.r, prob.v)
        return sim

    # ------------------------------------------------------------ substeps
    def substep(self, alpha: bool = True, transfer: bool = True, sums: bool = True, stream=None,
                sort_every: bool = False):
        """One SandSubstep: A (current) -> sort -> B -> forces -> A (next).
        With Verlet lists and the fused path the sort runs only when the
        lists are rebuilt, unless sort_every (then B is the sorted A every
        substep, as the adjoint's recomputation needs)."""
        F = self.fluid
        if self.nb is not None and self.fused and not sort_every:  # sorts only when the lists are rebuilt
            if not self.lists_current:
                gic.gic_neighbors_reset(self.nb, stream)
            gic.gic_step(self.grid, self.params, self.A, self.A2, self.B, self.perm, self.table, self.ws, self.nb,
                         F.u, F.v, F.w, F.p, F.alpha_f, self.alpha_s if alpha else None,
                         self.Fs if transfer else (None, None, None), self.sums if (sums and alpha) else None,
                         stream)
            self.A, self.A2 = self.A2, self.A
            self.lists_current = True
            return
        self.lists_current = False
        gic.gic_sort(self.grid, self.A, self.B, self.perm, self.table, self.ws, stream)
        if self.nb is not None and self.fused:
            self.fused_rest(alpha, transfer, sums, stream)
            return
        self.contact(stream)
        gic.gic_g2p_couple(self.grid, self.params, self.B, F.u, F.v, F.w, F.p, F.alpha_f, self.F_fl, self.a_f,
                           self.alpha_f_p, stream)
        gic.gic_integrate(self.grid, self.params, self.B, self.F_c, self.F_fl, self.a_f, self.A, self.f_ex, stream)
        gic.gic_p2g(self.grid, self.params, self.B, self.A, self.f_ex, self.alpha_s if alpha else None,
                    self.Fs if transfer else (None, None, None), self.sums if (sums and alpha) else None, stream)

    def fused_rest(self, alpha: bool, transfer: bool, sums: bool, stream=None):
        """Everything after the sort as one gic_substep: B -> A."""
        F = self.fluid
        self.lists_current = False
        gic.gic_substep(self.grid, self.params, self.B, self.table, self.nb, F.u, F.v, F.w, F.p, F.alpha_f, self.A,
                        None, self.alpha_s if alpha else None,
                        self.Fs if transfer else (None, None, None), self.sums if (sums and alpha) else None, stream)

    def contact(self, stream=None):
        """a2 on the sorted state B: Verlet lists when configured, else the
        cell-table walk."""
        self.lists_current = False
        if self.nb is not None:
            gic.gic_contact_verlet(self.grid, self.params, self.B, self.table, self.nb, self.F_c, stream)
        else:
            gic.gic_contact(self.grid, self.params, self.B, self.table, self.F_c, stream)

    def substep_probe(self, acc, stream=None, alpha: bool = True):
        """substep() with CUDA events around every entry point: appends
        (start, end) event pairs to acc[name] (timing only)."""
        s = torch.cuda.current_stream() if stream is None else stream
        F = self.fluid

        def timed(name, fn):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            acc.setdefault(name, []).append((a, b))

        if self.nb is not None and self.fused:
            if not self.lists_current:
                gic.gic_neighbors_reset(self.nb, s)
            timed("gic_step", lambda: gic.gic_step(self.grid, self.params, self.A, self.A2, self.B, self.perm,
                                                   self.table, self.ws, self.nb, F.u, F.v, F.w, F.p, F.alpha_f,
                                                   self.alpha_s if alpha else None, self.Fs,
                                                   self.sums if alpha else None, s))
            self.A, self.A2 = self.A2, self.A
            self.lists_current = True
            return
        self.lists_current = False
        timed("gic_sort", lambda: gic.gic_sort(self.grid, self.A, self.B, self.perm, self.table, self.ws, s))
        timed("gic_contact", lambda: self.contact(s))
        timed("gic_g2p_couple", lambda: gic.gic_g2p_couple(self.grid, self.params, self.B, F.u, F.v, F.w, F.p,
                                                            F.alpha_f, self.F_fl, self.a_f, self.alpha_f_p, s))
        timed("gic_integrate", lambda: gic.gic_integrate(self.grid, self.params, self.B, self.F_c, self.F_fl,
                                                          self.a_f, self.A, self.f_ex, s))
        timed("gic_p2g", lambda: gic.gic_p2g(self.grid, self.params, self.B, self.A, self.f_ex,
                                              self.alpha_s if alpha else None, self.Fs,
                                              self.sums if alpha else None, s))

    def zero_transfer(self):
        for f in self.Fs:
            f.zero_()

    def run(self, K: int, stream=None, alpha_every: bool = False, sort_every: bool = False):
        """K substeps (one fluid step); F_s accumulates from zero over them
        (Alg. 2); alpha_s and sums are computed at the final positions only
        (Alg. 1 CalTargetFraction), or after every substep if alpha_every.
        sort_every: as in substep()."""
        self.zero_transfer()
        for s in range(K):
            last = s == K - 1
            self.substep(alpha=alpha_every or last, sums=alpha_every or last, stream=stream, sort_every=sort_every)

    # ------------------------------------------------------------ outputs
    def positions(self, state: Optional[State] = None):
        """(x, v) FP64 [n, 3] in original granule order."""
        st = self.A if state is None else state
        x = torch.empty((self.n, 3), dtype=torch.float64, device=self.device)
        v = torch.empty((self.n, 3), dtype=torch.float64, device=self.device)
        gic.gic_unpack(self.grid, st, x, v)
        return x, v

    def status(self, clear=True) -> int:
        return gic.gic_check_status(clear=clear)

    # ------------------------------------------------------------ checkpoint / resume
    def save(self, path, step: int = 0, meta: Optional[dict] = None, stream=None):
        """Writes the current state (A) and this simulator's grid to `path`
        (see save_checkpoint).  The copy to the host waits for `stream` (the
        stream the substeps ran on; default: torch's current stream) and for
        torch's current stream, so a save after substeps on a side stream
        sees their results."""
        if stream is not None:
            stream.synchronize()
        torch.cuda.current_stream(self.device).synchronize()
        save_checkpoint(path, self.A, step, meta, grid=self.grid_obj)

    def resume(self, path) -> Tuple[int, dict]:
        """Loads a state written by save() into A (the next substep rebuilds
        the Verlet lists); returns (step, meta).  The file must hold a state of
        this simulator's size, precision and grid (positions are stored
        relative to the contact cells of that grid: on another grid they
        would mean other places)."""
        st, step, meta = load_checkpoint(path, self.device, grid=self.grid_obj)
        if st.n != self.n or st.precision != self.precision:
            raise ValueError(f"checkpoint holds {st.n} granules of precision {st.precision}, "
                             f"the simulator {self.n} of precision {self.precision}")
        self.load_state(st)
        return step, meta


# ---------------------------------------------------------------------------
# checkpoint files
# ---------------------------------------------------------------------------

CHECKPOINT_FORMAT = "gic-state-1"


def grid_record(grid) -> dict:
    """The fields of a grid that give a stored state its meaning (positions
    are contact-cell ids plus offsets in units of h_c = dx / k_contact)."""
    return {"nx": int(grid.nx), "ny": int(grid.ny), "nz": int(grid.nz), "dx": float(grid.dx),
            "origin": [float(o) for o in grid.origin], "k_contact": int(grid.k_contact)}


def save_checkpoint(path, state: State, step: int = 0, meta: Optional[dict] = None, grid=None):
    """Writes a granule state to a file with torch.save: the raw arrays in the
    library's layout (cell, pos, vel, id, posf; moved to the host, bit for
    bit), the precision, the grid the positions refer to (any object with
    nx, ny, nz, dx, origin, k_contact; recommended: without it the file can
    only be loaded without a grid check), a step counter and a dict of plain
    metadata (numbers, strings, lists: e.g. the workload's name and
    parameters), so that a long run can stop and resume exactly.  The state
    is copied with .cpu(), which waits for torch's current stream only: after
    work on another stream, synchronise that stream first (Simulator.save
    does)."""
    d = {"format": CHECKPOINT_FORMAT, "precision": int(state.precision), "step": int(step),
         "grid": None if grid is None else grid_record(grid),
         "meta": dict(meta or {}), "cell": state.cell.detach().cpu(), "pos": state.pos.detach().cpu(),
         "vel": state.vel.detach().cpu(), "id": None if state.id is None else state.id.detach().cpu(),
         "posf": None if state.posf is None else state.posf.detach().cpu()}
    torch.save(d, path)


def load_checkpoint(path, device="cuda", grid=None) -> Tuple[State, int, dict]:
    """Reads a file written by save_checkpoint: (state on `device`, step,
    meta).  Raises ValueError for a file of another format, with arrays
    whose shapes or types do not form a state, or -- when `grid` is given --
    for a file saved on another grid or without a grid record."""
    d = torch.load(path, map_location="cpu", weights_only=True)
    if not isinstance(d, dict) or d.get("format") != CHECKPOINT_FORMAT:
        raise ValueError(f"{path}: not a {CHECKPOINT_FORMAT} checkpoint")
    if grid is not None:
        saved = d.get("grid")
        if saved is None:
            raise ValueError(f"{path}: the checkpoint records no grid, so its positions cannot be checked")
        if saved != grid_record(grid):
            raise ValueError(f"{path}: saved on grid {saved}, not on {grid_record(grid)}")
    prec = int(d["precision"])
    if prec not in (GIC_FP32, GIC_FP64):
        raise ValueError(f"{path}: unknown precision {prec}")
    cell, pos, vel, ids, posf = d["cell"], d["pos"], d["vel"], d["id"], d["posf"]
    n = int(cell.shape[0])
    real = torch.float32 if prec == GIC_FP32 else torch.float64
    pos_dtype = torch.int32 if prec == GIC_FP32 else torch.float64
    ok = (cell.dtype == torch.int32 and cell.shape == (n,) and pos.dtype == pos_dtype and tuple(pos.shape) == (n, 4)
          and vel.dtype == real and tuple(vel.shape) == (n, 4)
          and (ids is None or (ids.dtype == torch.int32 and tuple(ids.shape) == (n,)))
          and (posf is None or (prec == GIC_FP32 and posf.dtype == torch.float32 and tuple(posf.shape) == (n, 4))))
    if not ok:
        raise ValueError(f"{path}: arrays do not form a granule state of precision {prec}")
    dev = lambda t: None if t is None else t.to(device).contiguous()
    return State(dev(cell), dev(pos), dev(vel), dev(ids), prec, dev(posf)), int(d["step"]), dict(d["meta"])


# ---------------------------------------------------------------------------
# differentiable window
# ---------------------------------------------------------------------------

def _copy_state(dst: State, src: State):
    dst.cell.copy_(src.cell)
    dst.pos.copy_(src.pos)
    dst.vel.copy_(src.vel)
    if dst.id is not None and src.id is not None:
        dst.id.copy_(src.id)
    if dst.posf is not None and src.posf is not None:  # a gic_step that keeps its lists reads it
        dst.posf.copy_(src.posf)


class GicWindow(torch.autograd.Function):
    """x_K = window(v0, c_drag, mu): K substeps from the simulator's initial
    state with initial velocities v0 (FP64 [n, 3], original order), drag
    coefficient c_drag and friction coefficient mu (0-d tensors).  Returns the
    final absolute positions (FP64 [n, 3], original order).

    Backward: the window is cut into segments of `ckpt` substeps; the state at
    the start of each segment is kept from the forward pass and every segment
    is recomputed from it, in reverse order.

    With Verlet lists and the fused path, forward and recomputation run
    gic_step (the sort only on list rebuilds).  The window opens with a list
    build, and every checkpoint also keeps the lists as they stand (a new
    copy only after a build), so the recomputation from it repeats the
    forward pass exactly.  The recomputation keeps the state before every
    substep and notes which substeps rebuilt the lists; going back, the
    lists each substep used are restored (from the checkpoint, or by sort +
    build from the state of the substep that built them), and each
    substep's adjoint is one gic_substep_adj: on the substep's state, or on
    its sorted copy with the sort's permutation where the substep sorted.

    Otherwise forward and recomputation sort every substep, and each
    substep's adjoint re-sorts its state and runs gic_integrate_adj,
    gic_g2p_couple_adj, gic_contact_adj (through the Verlet lists when the
    simulator has them) and gic_sort_adj.
    """

    @staticmethod
    def forward(ctx, v0, c_drag, mu, sim: "Simulator", init: State, K: int, ckpt: int):
        sim.params.c_drag = float(c_drag)
        sim.params.mu_fric = float(mu)
        sim.load_state(init)
        vel = sim.A.vel
        vel[:, :3] = v0.detach().to(vel.dtype)  # init is in original order (id = 0..n-1)
        vel[:, 3] = 0
        stepped = sim.nb is not None and sim.fused
        if stepped:  # the lists left by earlier calls do not enter the result: the first substep builds
            gic.gic_neighbors_reset(sim.nb)
            sim.lists_current = True
        ckpts, lists = [], []
        log = torch.zeros(K + 1, dtype=torch.int32, device=sim.device) if stepped else None
        if stepped:
            log[0:1].copy_(sim.nb.flags[4:5])
        for s in range(K):
            if s % ckpt == 0:
                ckpts.append(sim.A.clone())
                if stepped:
                    lists.append(_lists_snapshot(sim.nb))
            sim.substep(alpha=False, transfer=False, sums=False, sort_every=not stepped)
            if stepped:
                log[s + 1:s + 2].copy_(sim.nb.flags[4:5])  # list builds so far (device copy, no wait)
        x, _ = sim.positions()
        ctx.sim, ctx.K, ctx.ckpt, ctx.stepped = sim, K, ckpt, stepped
        ctx.ckpts, ctx.lists = ckpts, lists
        # the window's build record, read once: the recomputation from each
        # checkpoint repeats the forward pass exactly, builds included
        ctx.build_log = log.tolist() if stepped else None
        ctx.final = sim.A.clone()
        return x

    @staticmethod
    def backward(ctx, g_x):
        sim = ctx.sim
        n, prec, dev = sim.n, sim.precision, sim.device
        g_pos = gic.vec4(n, prec, dev)
        g_vel = gic.vec4(n, prec, dev)
        gic.gic_unpack_adj(sim.grid, ctx.final, g_x.contiguous().to(torch.float64), None, g_pos, None)
        g_scalars = torch.zeros(2, dtype=torch.float64, device=dev)  # [c_drag, mu]
        if ctx.stepped:
            g_vel = _backward_stepped(ctx, g_pos, g_vel, g_scalars)
        else:
            g_vel = _backward_sorted(ctx, g_pos, g_vel, g_scalars)
        g_v0 = g_vel[:, :3].to(torch.float64)
        return g_v0, g_scalars[0].clone(), g_scalars[1].clone(), None, None, None, None


def _segments(K: int, ckpt: int):
    """(s0, s1) of every checkpoint segment, last first."""
    return [(m * ckpt, min(K, (m + 1) * ckpt)) for m in reversed(range((K + ckpt - 1) // ckpt))]


_NB_ARRAYS = ("list", "count", "ref_cell", "ref_pos", "slot")


def _lists_snapshot(nb: gic.Neighbors) -> dict:
    """The Verlet lists as they stand, copied on the device without waiting
    for them: the flag words (among them the decision for the next gic_step
    and the build count) and the rows and reference entries (`cur` and `at`
    follow from them at the next check).  When a build is pending the rows
    are not used: restoring the flags makes the next call rebuild."""
    return {"flags": nb.flags.clone(), "arrays": {a: getattr(nb, a).clone() for a in _NB_ARRAYS}}


def _lists_restore(nb: gic.Neighbors, snap: dict):
    nb.flags.copy_(snap["flags"])
    if snap["arrays"] is not None:
        for a, t in snap["arrays"].items():
            getattr(nb, a).copy_(t)


def _backward_stepped(ctx, g_pos, g_vel, g_scalars):
    sim, nb, F = ctx.sim, ctx.sim.nb, ctx.sim.fluid
    n, prec, dev = sim.n, sim.precision, sim.device
    g_pos_n = gic.vec4(n, prec, dev)
    g_vel_n = gic.vec4(n, prec, dev)
    ends, expected = [], []

    def sort_and_build(st: State):
        """st sorted into B (perm, cell table) and the lists built from B
        (with the capillary force on, by a fused substep into the scratch
        state A2, whose list build covers the bridge reach)."""
        gic.gic_sort(sim.grid, st, sim.B, sim.perm, sim.table, sim.ws)
        gic.gic_neighbors_reset(nb)
        if sim.params.sigma > 0.0:
            gic.gic_substep(sim.grid, sim.params, sim.B, sim.table, nb, F.u, F.v, F.w, F.p, F.alpha_f, sim.A2, None,
                            None, (None, None, None), None)
        else:
            gic.gic_contact_verlet(sim.grid, sim.params, sim.B, sim.table, nb, sim.F_c)

    for m, (s0, s1) in zip(reversed(range(len(ctx.ckpts))), _segments(ctx.K, ctx.ckpt)):
        L = s1 - s0
        # recompute the segment from its checkpoint and lists, keeping the state before every substep
        _copy_state(sim.A, ctx.ckpts[m])
        _lists_restore(nb, ctx.lists[m])
        sim.lists_current = True
        states = []
        for k in range(L):
            states.append(sim.A.clone())
            sim.substep(alpha=False, transfer=False, sums=False)
        counts = ctx.build_log[s0:s1 + 1]  # the forward pass's record: the recomputation repeats it
        built = [counts[k + 1] != counts[k] for k in range(L)]
        # the substep whose build made the lists substep k walked (-1: the checkpoint's)
        last_build = [max([j for j in range(k + 1) if built[j]], default=-1) for k in range(L)]
        lists_of, count_now = last_build[L - 1], counts[L]
        for k in reversed(range(L)):
            b = last_build[k]
            if b != lists_of and b != k:  # restore the lists substep k walked
                if b < 0:
                    _lists_restore(nb, ctx.lists[m])
                    count_now = ctx.build_log[s0]
                else:
                    sort_and_build(states[b])
                    count_now = 1  # a reset clears the build count
                lists_of = b
            if built[k]:  # substep k sorted its state and built the lists from it: the adjoint runs there
                if lists_of != k:
                    sort_and_build(states[k])
                    lists_of, count_now = k, 1
                else:
                    gic.gic_sort(sim.grid, states[k], sim.B, sim.perm, sim.table, sim.ws)
                acted, perm = sim.B, sim.perm
            else:  # substep k ran on its state as it was, and its result kept the order
                acted, perm = states[k], None
            gic.gic_substep_adj(sim.grid, sim.params, acted, perm, sim.table, nb, F.u, F.v, F.w, F.p, F.alpha_f,
                                g_pos, g_vel, None, g_pos_n, g_vel_n, g_scalars[0:1], g_scalars[1:2])
            g_pos, g_pos_n = g_pos_n, g_pos
            g_vel, g_vel_n = g_vel_n, g_vel
        ends.append(nb.flags[4:5].clone())
        expected.append(count_now)
    sim.lists_current = False
    # every adjoint walked the lists its forward substep used: no build of its own
    got = torch.cat(ends).tolist()
    if got != expected:
        raise RuntimeError(f"Verlet lists were rebuilt inside the adjoint (builds {got}, expected {expected})")
    return g_vel


def _backward_sorted(ctx, g_pos, g_vel, g_scalars):
    sim, K, ckpt, F = ctx.sim, ctx.K, ctx.ckpt, ctx.sim.fluid
    n, prec, dev = sim.n, sim.precision, sim.device
    g_pos_b = gic.vec4(n, prec, dev)
    g_vel_b = gic.vec4(n, prec, dev)
    gFc = gic.vec4(n, prec, dev)
    gFfl = gic.vec4(n, prec, dev)
    gaf = gic.vec4(n, prec, dev)
    for m, (s0, s1) in zip(reversed(range(len(ctx.ckpts))), _segments(K, ckpt)):
        # recompute the segment, keeping the state before every substep
        _copy_state(sim.A, ctx.ckpts[m])
        pre = []
        for s in range(s0, s1):
            pre.append(sim.A.clone())
            if s < s1 - 1:
                sim.substep(alpha=False, transfer=False, sums=False, sort_every=True)
        for s in reversed(range(s0, s1)):
            S = pre[s - s0]
            gic.gic_sort(sim.grid, S, sim.B, sim.perm, sim.table, sim.ws)
            gic.gic_integrate_adj(sim.grid, sim.params, sim.B, g_pos, g_vel, None, g_pos_b, g_vel_b, gFc, gFfl, gaf)
            gic.gic_g2p_couple_adj(sim.grid, sim.params, sim.B, F.u, F.v, F.w, F.p, F.alpha_f, gFfl, gaf, None,
                                   g_pos_b, g_vel_b, g_scalars[0:1])
            if sim.nb is not None:
                gic.gic_contact_verlet_adj(sim.grid, sim.params, sim.B, sim.table, sim.nb, sim.F_c, gFc, g_pos_b,
                                           g_vel_b, g_scalars[1:2])
            else:
                gic.gic_contact_adj(sim.grid, sim.params, sim.B, sim.table, gFc, g_pos_b, g_vel_b, g_scalars[1:2])
            gic.gic_sort_adj(n, prec, sim.perm, g_pos_b, g_vel_b, g_pos, g_vel)
    return g_vel


def window_loss_and_grads(prob, precision=GIC_FP32, K=None, ckpt=10, device="cuda", **sim_kw):
    """Loss = mean |x_K - target|^2 of a problem with a target cloud, and its
    gradients w.r.t. the initial velocities, c_drag and mu (FP64 tensors).
    sim_kw go to Simulator.from_problem."""
    sim = Simulator.from_problem(prob, precision, device, **sim_kw)
    init = sim.A.clone()
    K = prob.K if K is None else K
    v0 = torch.tensor(prob.v, dtype=torch.float64, device=device, requires_grad=True)
    c = torch.tensor(float(prob.params.c_drag), dtype=torch.float64, device=device, requires_grad=True)
    mu = torch.tensor(float(prob.params.mu_fric), dtype=torch.float64, device=device, requires_grad=True)
    x = GicWindow.apply(v0, c, mu, sim, init, K, ckpt)
    target = torch.as_tensor(prob.target, dtype=torch.float64, device=device)
    loss = ((x - target) ** 2).sum(dim=1).mean()
    loss.backward()
    return loss.detach(), v0.grad, c.grad, mu.grad, sim
