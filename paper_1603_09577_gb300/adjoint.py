"""Differentiable runs: phi_N = run(phi0, K(x), u) as a torch.autograd.Function.

The forward pass advances the lattice with liblbm's fused step and keeps a
checkpoint of the state every `ckpt_every` steps. The backward pass walks the
segments from last to first: it restores the segment's checkpoint, recomputes
and keeps the segment's states, then runs liblbm's reverse steps over them
(FP64 gradient accumulation in the kernels) and finishes at the initial
condition. Built for the linear family with periodic walls (see lbm.h).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as C
from .solver import Solver, _prec_of, _ptr, _stream


class LBMRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, K, u, nsteps, ckpt_every, prec, s_rates):
        ny, nx = phi0.shape
        dev = phi0.device
        solver = Solver(nx, ny, prec=prec, per_cell_K=True, device=dev)
        uu = [float(v) for v in u.detach().cpu().tolist()]
        solver.set_coeffs(conv=0, u=uu, diff=0, K=(0.0, 0.0, 0.0), s=s_rates)
        solver.set_K_field(K.detach())
        phi0c = phi0.detach().contiguous()
        solver.set_phi(phi0c)
        ckpts = [solver.save()]
        done = 0
        while done < nsteps:
            n = min(ckpt_every, nsteps - done)
            solver.step(n)
            done += n
            if done < nsteps:
                ckpts.append(solver.save())
        out = solver.phi(torch.float64)
        ctx.solver, ctx.ckpts, ctx.phi0 = solver, ckpts, phi0c
        ctx.nsteps, ctx.ckpt_every = nsteps, ckpt_every
        return out

    @staticmethod
    def backward(ctx, grad_out):
        s, nsteps, L = ctx.solver, ctx.nsteps, ctx.ckpt_every
        lib = s.lib
        st = _stream()
        size = ctypes.c_size_t()
        C.check(lib.lbm_adjoint_workspace_size(s.h, ctypes.byref(size)))
        ws = torch.empty(size.value, dtype=torch.uint8, device=s.device)
        g = grad_out.detach().to(torch.float64).contiguous()
        C.check(lib.lbm_adjoint_begin(s.h, _ptr(ws), size.value, _ptr(g), C.LBM_F64, st))
        nseg = len(ctx.ckpts)
        nb = s.state_bytes()
        scratch = torch.empty(max(1, min(L, nsteps) - 1) * nb, dtype=torch.uint8, device=s.device)
        for seg in range(nseg - 1, -1, -1):
            t0 = seg * L
            t1 = min(t0 + L, nsteps)
            # recompute the segment's states from its checkpoint and walk them back
            C.check(lib.lbm_adjoint_segment(s.h, _ptr(ctx.ckpts[seg]), t1 - t0, _ptr(scratch),
                                            scratch.numel(), st))
        ny, nx = ctx.phi0.shape
        dphi0 = torch.empty((ny, nx), dtype=torch.float64, device=s.device)
        dK = torch.empty((3, ny, nx), dtype=torch.float64, device=s.device)
        du = torch.empty(2, dtype=torch.float64, device=s.device)
        C.check(lib.lbm_adjoint_end(s.h, _ptr(ctx.phi0), _prec_of(ctx.phi0), _ptr(dphi0), _ptr(dK), _ptr(du), st))
        return dphi0, dK, du, None, None, None, None


def run(phi0: torch.Tensor, K: torch.Tensor, u: torch.Tensor, nsteps: int, ckpt_every: int = 50,
        prec: str = "f32", s_rates=(1.0, 1.2, 1.2, 0.0, 1.0, 0.0, 1.0, 1.1, 1.1)) -> torch.Tensor:
    """phi(t_N) of the linear anisotropic CDE with per-node tensor K (3, ny, nx),
    differentiable with respect to phi0, K and u (2,)."""
    return LBMRun.apply(phi0, K, u, int(nsteps), int(ckpt_every), prec, tuple(s_rates))
