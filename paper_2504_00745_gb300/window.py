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
from typing import List, Optional

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


class Simulator:
    """Device buffers + substep loop for one problem.

    grid / params: objects with the fields of GicGrid / GicParams (e.g.
    gic_inputs.Grid / Params).  The initial state comes from the canonical
    encoding (cell int32 [n,3], q uint32 [n,3], r float32 [n], v float32 [n,3])
    as host or device tensors.  verlet_skin (metres): contact through Verlet
    lists with that skin (gic_contact_verlet, cap partners per granule)
    instead of walking the cell table every substep (gic_contact); with
    lists and fused, a substep is one gic_step (sort only on list rebuilds,
    then the fused gic_substep).
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
        self.A = State.empty(n, precision, device)
        self.B = State.empty(n, precision, device, with_posf=True)  # sorted state: float position copy (FP32)
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

    @classmethod
    def from_problem(cls, prob, precision=GIC_FP32, device="cuda", verlet: bool = True, fused: bool = True):
        """Simulator of a gic_inputs.Problem; verlet: Verlet lists with a skin
        of 0.15 r_max (48 partners per granule, 96 when radii vary by more
        than 1.5x)."""
        skin = cap = None
        if verlet and prob.n > 0:
            r = prob.r
            skin = 0.15 * float(r.max())
            cap = 48 if float(r.max()) <= 1.5 * float(r.min()) else 96
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
            gic.gic_step(self.grid, self.params, self.A, self.B, self.perm, self.table, self.ws, self.nb, F.u, F.v,
                         F.w, F.p, F.alpha_f, self.alpha_s if alpha else None,
                         self.Fs if transfer else (None, None, None), self.sums if (sums and alpha) else None,
                         stream)
            return
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
        gic.gic_substep(self.grid, self.params, self.B, self.table, self.nb, F.u, F.v, F.w, F.p, F.alpha_f, self.A,
                        None, self.alpha_s if alpha else None,
                        self.Fs if transfer else (None, None, None), self.sums if (sums and alpha) else None, stream)

    def contact(self, stream=None):
        """a2 on the sorted state B: Verlet lists when configured, else the
        cell-table walk."""
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
            timed("gic_step", lambda: gic.gic_step(self.grid, self.params, self.A, self.B, self.perm, self.table,
                                                   self.ws, self.nb, F.u, F.v, F.w, F.p, F.alpha_f,
                                                   self.alpha_s if alpha else None, self.Fs,
                                                   self.sums if alpha else None, s))
            return
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

    def run(self, K: int, stream=None, alpha_every: bool = False):
        """K substeps (one fluid step); F_s accumulates from zero over them
        (Alg. 2); alpha_s and sums are computed at the final positions only
        (Alg. 1 CalTargetFraction), or after every substep if alpha_every."""
        self.zero_transfer()
        for s in range(K):
            last = s == K - 1
            self.substep(alpha=alpha_every or last, sums=alpha_every or last, stream=stream)

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


# ---------------------------------------------------------------------------
# differentiable window
# ---------------------------------------------------------------------------

def _copy_state(dst: State, src: State):
    dst.cell.copy_(src.cell)
    dst.pos.copy_(src.pos)
    dst.vel.copy_(src.vel)
    if dst.id is not None and src.id is not None:
        dst.id.copy_(src.id)


class GicWindow(torch.autograd.Function):
    """x_K = window(v0, c_drag, mu): K substeps from the simulator's initial
    state with initial velocities v0 (FP64 [n, 3], original order), drag
    coefficient c_drag and friction coefficient mu (0-d tensors).  Returns the
    final absolute positions (FP64 [n, 3], original order).

    Backward: the window is cut into segments of `ckpt` substeps; the state at
    the start of each segment is kept from the forward pass, every segment is
    recomputed from it in reverse order (forward and recomputation sort every
    substep, so each substep's sorted order is the one its adjoint re-sorts
    to), and each substep's adjoint runs
    gic_integrate_adj, gic_g2p_couple_adj, gic_contact_adj (through the
    Verlet lists when the simulator has them) and gic_sort_adj.
    """

    @staticmethod
    def forward(ctx, v0, c_drag, mu, sim: "Simulator", init: State, K: int, ckpt: int):
        sim.params.c_drag = float(c_drag)
        sim.params.mu_fric = float(mu)
        _copy_state(sim.A, init)
        vel = sim.A.vel
        vel[:, :3] = v0.detach().to(vel.dtype)  # init is in original order (id = 0..n-1)
        vel[:, 3] = 0
        ckpts = []
        for s in range(K):
            if s % ckpt == 0:
                ckpts.append(sim.A.clone())
            sim.substep(alpha=False, transfer=False, sums=False, sort_every=True)
        x, _ = sim.positions()
        ctx.sim, ctx.K, ctx.ckpt = sim, K, ckpt
        ctx.ckpts = ckpts
        ctx.final = sim.A.clone()
        return x

    @staticmethod
    def backward(ctx, g_x):
        sim, K, ckpt = ctx.sim, ctx.K, ctx.ckpt
        n, prec = sim.n, sim.precision
        dev = sim.device
        g_pos = gic.vec4(n, prec, dev)
        g_vel = gic.vec4(n, prec, dev)
        gic.gic_unpack_adj(sim.grid, ctx.final, g_x.contiguous().to(torch.float64), None, g_pos, None)
        g_pos_b = gic.vec4(n, prec, dev)
        g_vel_b = gic.vec4(n, prec, dev)
        gFc = gic.vec4(n, prec, dev)
        gFfl = gic.vec4(n, prec, dev)
        gaf = gic.vec4(n, prec, dev)
        g_scalars = torch.zeros(2, dtype=torch.float64, device=dev)  # [c_drag, mu]
        F = sim.fluid
        n_seg = len(ctx.ckpts)
        for m in reversed(range(n_seg)):
            s0 = m * ckpt
            s1 = min(K, s0 + ckpt)
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
                gic.gic_integrate_adj(sim.grid, sim.params, sim.B, g_pos, g_vel, None, g_pos_b, g_vel_b, gFc, gFfl,
                                      gaf)
                gic.gic_g2p_couple_adj(sim.grid, sim.params, sim.B, F.u, F.v, F.w, F.p, F.alpha_f, gFfl, gaf, None,
                                       g_pos_b, g_vel_b, g_scalars[0:1])
                if sim.nb is not None:
                    gic.gic_contact_verlet_adj(sim.grid, sim.params, sim.B, sim.table, sim.nb, sim.F_c, gFc, g_pos_b,
                                               g_vel_b, g_scalars[1:2])
                else:
                    gic.gic_contact_adj(sim.grid, sim.params, sim.B, sim.table, gFc, g_pos_b, g_vel_b,
                                        g_scalars[1:2])
                gic.gic_sort_adj(n, prec, sim.perm, g_pos_b, g_vel_b, g_pos, g_vel)
        g_v0 = g_vel[:, :3].to(torch.float64)
        return g_v0, g_scalars[0].clone(), g_scalars[1].clone(), None, None, None, None


def window_loss_and_grads(prob, precision=GIC_FP32, K=None, ckpt=10, device="cuda"):
    """Loss = mean |x_K - target|^2 of a problem with a target cloud, and its
    gradients w.r.t. the initial velocities, c_drag and mu (FP64 tensors)."""
    sim = Simulator.from_problem(prob, precision, device)
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
