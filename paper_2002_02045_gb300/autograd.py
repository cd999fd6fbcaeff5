"""torch.autograd functions over the collision integral and RK4 stepping.

Argument marshalling only: the forward values come from ``pgb_collision`` /
``pgb_step_rk4`` and the derivatives from ``pgb_collision_vjp`` /
``pgb_rk4_adjoint`` (reverse-mode derivatives written by hand in the CUDA
library, with checkpointed recomputation of the RK4 states).  Autograd keeps
only f (or f0) between forward and backward.

|g|^2 of the list entries is an input like f: a float32 CUDA tensor in the
entry order of the list the context holds.  When a call sees a different
tensor than the previous call (another storage, or an in-place change), the
context's list is updated with ``pgb_collision_set_g2`` first.
"""
from __future__ import annotations

import torch

from .native import Context


class CollisionList:
    """The scattering list built in ``ctx`` and the |g|^2 tensor it currently holds."""

    def __init__(self, ctx: Context, g2: torch.Tensor):
        self.ctx = ctx
        self.nstates = ctx.pgb_collision_energies()
        self.nnz = int(g2.numel())
        self._key = None
        self.sync(g2)

    def sync(self, g2: torch.Tensor):
        if g2.dtype != torch.float32 or g2.numel() != self.nnz:
            raise ValueError("g2 must be a float32 tensor with one value per list entry")
        key = (g2.data_ptr(), g2._version)
        if key != self._key:
            self.ctx.pgb_collision_set_g2(g2.detach().contiguous())
            self._key = key


class _Collision(torch.autograd.Function):
    @staticmethod
    def forward(actx, f, g2, lst):
        lst.sync(g2)
        f = f.detach().contiguous()
        out = torch.empty_like(f)
        lst.ctx.pgb_collision(f, out)
        actx.save_for_backward(f)
        actx.lst = lst
        return out

    @staticmethod
    def backward(actx, grad):
        (f,) = actx.saved_tensors
        lst = actx.lst
        vf = torch.empty_like(f)
        vg = torch.empty(lst.nnz, dtype=torch.float64, device=f.device) if actx.needs_input_grad[1] else None
        lst.ctx.pgb_collision_vjp(f, grad.detach().to(torch.float64).contiguous(), vf, vg)
        return vf, (vg.to(torch.float32) if vg is not None else None), None


class _RK4(torch.autograd.Function):
    @staticmethod
    def forward(actx, f0, g2, lst, dt_fs, nsteps, checkpoint):
        lst.sync(g2)
        f0 = f0.detach().contiguous()
        f = f0.clone()
        lst.ctx.pgb_step_rk4(f, dt_fs, nsteps)
        actx.save_for_backward(f0)
        actx.args = (lst, float(dt_fs), int(nsteps), int(checkpoint))
        return f

    @staticmethod
    def backward(actx, grad):
        (f0,) = actx.saved_tensors
        lst, dt_fs, nsteps, checkpoint = actx.args
        lam0 = torch.empty_like(f0)
        dg2 = torch.empty(lst.nnz, dtype=torch.float64, device=f0.device) if actx.needs_input_grad[1] else None
        lst.ctx.pgb_rk4_adjoint(f0, dt_fs, nsteps, checkpoint, grad.detach().to(torch.float64).contiguous(), lam0,
                                dg2)
        return lam0, (dg2.to(torch.float32) if dg2 is not None else None), None, None, None, None


def collision(f: torch.Tensor, g2: torch.Tensor, lst: CollisionList) -> torch.Tensor:
    """I[f] (Eq. e_ph_scattering), differentiable in f (float64) and g2 (float32)."""
    return _Collision.apply(f, g2, lst)


def rk4(f0: torch.Tensor, g2: torch.Tensor, lst: CollisionList, dt_fs: float, nsteps: int,
        checkpoint: int = 50) -> torch.Tensor:
    """f after ``nsteps`` RK4 steps of df/dt = I[f] (Sec. 2.1.1), differentiable in f0 and g2."""
    return _RK4.apply(f0, g2, lst, dt_fs, nsteps, checkpoint)
