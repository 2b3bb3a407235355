"""Hierarchical kick-drift-kick time stepping of one system on the GPU
(paper Sec. 7.1-7.3), around the force path.

Every tick of the power-of-two hierarchy: all particles drift
(``tpm_drift``), the particles due are selected on the device
(``tpm_active_set``, with their previous |a|), the tree is built anew from
all particles' positions (``tpm_build_tree``, Sec. 3.1: one build per local
step), the forces on the particles due are computed (``tpm_compute_forces``;
the first evaluation with the geometric criterion, later ones with the
relative criterion against each particle's last |a|; periodic systems add the
PM long-range force, recomputed after each build), and their steps are
closed and reopened with new bins (``tpm_kick``).  Positions and velocities
stay on the device in FP64.  This module only sequences library calls.
"""
from __future__ import annotations

from dataclasses import replace

from . import CRIT_RELATIVE, BuildParams, Context, ForceParams, StepParams, active_set, drift, kick


class Integrator:
    """State of one system: ``pos``, ``vel`` (n x 3 FP64), ``mass`` (n FP32),
    ``bins`` (n int8), ``amag`` (n FP32, |a| of each particle's last force) as
    device tensors, and the tick counter.  ``fp_first`` is the criterion of
    the first evaluation (normally geometric), ``fp`` the one of later ticks
    (normally relative).  ``shift(tick)`` gives the root shift of each build
    (a fixed one if None)."""

    def __init__(self, ctx: Context, pos, vel, mass, bp: BuildParams, sp: StepParams, fp_first: ForceParams,
                 fp: ForceParams, shift=None, stream=None):
        import torch

        self.torch = torch
        self.ctx, self.bp, self.sp, self.fp_first, self.fp = ctx, bp, sp, fp_first, fp
        self.shift = shift
        self.stream = stream
        dev = torch.device("cuda", ctx.device)
        as_dev = lambda x, dt: torch.as_tensor(x, dtype=dt).to(dev).contiguous().clone()
        self.pos = as_dev(pos, torch.float64)
        self.vel = as_dev(vel, torch.float64)
        self.mass = as_dev(mass, torch.float32)
        n = self.n = int(self.pos.shape[0])
        self.bins = torch.zeros(n, dtype=torch.int8, device=dev)
        self.amag = torch.zeros(n, dtype=torch.float32, device=dev)
        self.ids = torch.arange(n, dtype=torch.int32, device=dev)
        self.a_old = torch.empty(n, dtype=torch.float32, device=dev)
        self.acc = torch.empty((n, 3), dtype=torch.float32, device=dev)
        self.pot = torch.empty(n, dtype=torch.float32, device=dev)
        self.nint = torch.empty(n, dtype=torch.int32, device=dev)
        self.tick = 0
        self.n_forces = 0
        self._forces(n, first=True)
        kick(ctx, self.ids, n, self.acc, self.vel, self.bins, self.amag, 0, sp, first=True, stream=stream)

    def _forces(self, n_act: int, first: bool):
        bp = self.bp if self.shift is None else replace(self.bp, shift=tuple(self.shift(self.tick)))
        s = self.ctx.build_tree(self.pos, self.mass, bp, stream=self.stream)
        try:
            fp = self.fp_first if first else self.fp
            if fp.treepm:
                s.pm_long_range(fp, stream=self.stream)
            a_old = self.a_old[:n_act] if fp.crit == CRIT_RELATIVE else None
            s.compute_forces(active_ids=self.ids[:n_act], a_old=a_old, fp=fp, acc=self.acc[:n_act],
                             pot=self.pot[:n_act], n_int=self.nint[:n_act], stream=self.stream)
        finally:
            s.release()
        self.n_forces += n_act

    def advance(self) -> int:
        """One tick; returns the number of particles that were due."""
        bp = self.bp
        drift(self.ctx, self.pos, self.vel, self.sp.dt_tick, bp.periodic, bp.box, stream=self.stream)
        self.tick += 1
        n_act = active_set(self.ctx, self.bins, self.tick, self.sp.nbins, self.ids, amag=self.amag,
                           a_old=self.a_old, stream=self.stream)
        if n_act:
            self._forces(n_act, first=False)
            kick(self.ctx, self.ids, n_act, self.acc[:n_act], self.vel, self.bins, self.amag, self.tick, self.sp,
                 stream=self.stream)
        return n_act

    def run_cycle(self) -> int:
        """Advances to the end of the current cycle of 2^(nbins-1) ticks (where
        every bin is due again); returns the number of forces computed."""
        before = self.n_forces
        cycle = 1 << (self.sp.nbins - 1)
        while True:
            self.advance()
            if self.tick % cycle == 0:
                return self.n_forces - before
