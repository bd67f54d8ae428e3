"""Gradients of a probe loss through the PIC run, as a torch.autograd.Function.

The forward pass runs the CUDA step with checkpoints (``bp_forward_ckpt``) and
returns the recorded probe samples; the backward pass is the library's
hand-written discrete adjoint (``bp_backward``): transposed Yee, reversed
Boris push and modified-Coulomb force, gather and deposit used as each
other's transposes, recomputation from the checkpoints, FP64 reductions.
Parameters: the bound-electron natural frequency of every parameter index
(e.g. one per column) and the lattice-site positions (each site's ions move
rigidly with it).
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from . import binding as B


class SiteProblem:
    """A two-body species whose ions sit at fixed offsets from lattice sites.

    x_ion = sites[site_of_ion] + offset_ion; omega_b[param_idx[ion]].
    """

    def __init__(self, ctx: B.Context, sid: int, pid: int, site_of_ion: np.ndarray, offsets: np.ndarray,
                 param_idx: np.ndarray, steps: int, K: int, u: Optional[np.ndarray] = None):
        self.ctx = ctx
        self.sid = sid
        self.pid = pid
        self.site_of_ion = np.ascontiguousarray(site_of_ion, dtype=np.int32)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.float64)
        self.param_idx = np.ascontiguousarray(param_idx, dtype=np.int32)
        self.steps = steps
        self.K = K
        self.u = u
        self.n_sites = int(self.site_of_ion.max()) + 1 if len(self.site_of_ion) else 0

    def run(self, omega_b: np.ndarray, sites: np.ndarray) -> np.ndarray:
        c = self.ctx
        c.reset()
        c.set_omega(self.sid, omega_b)
        x = sites[self.site_of_ion] + self.offsets
        c.load_particles(self.sid, x, self.u, self.param_idx)
        c.forward_ckpt(self.steps, self.K)
        c.sync()
        return c.read_probe(self.pid)

    def gradients(self, dl_dprobe: np.ndarray, n_omega: int):
        return self.ctx.backward(self.pid, dl_dprobe, self.sid, n_omega, self.site_of_ion, self.n_sites)


class PICProbe(torch.autograd.Function):
    """probe = PICProbe.apply(omega_b, sites, problem)

    omega_b: float64 [n_omega]; sites: float64 [n_sites, dims].  Returns the
    probe samples [steps, npts] (float64 view of the FP32 record)."""

    @staticmethod
    def forward(ctx, omega_b: torch.Tensor, sites: torch.Tensor, problem: SiteProblem):
        probe = problem.run(omega_b.detach().cpu().double().numpy(), sites.detach().cpu().double().numpy())
        ctx.problem = problem
        ctx.n_omega = omega_b.numel()
        ctx.dtype_o = omega_b.dtype
        ctx.dtype_s = sites.dtype
        return torch.from_numpy(probe.astype(np.float64))

    @staticmethod
    def backward(ctx, grad_probe: torch.Tensor):
        g = grad_probe.detach().cpu().float().numpy()
        go, gs = ctx.problem.gradients(g, ctx.n_omega)
        return (torch.from_numpy(go).to(ctx.dtype_o), torch.from_numpy(np.ascontiguousarray(gs)).to(ctx.dtype_s),
                None)
