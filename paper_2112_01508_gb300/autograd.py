"""Differentiable short-range force and a checkpointed KDK leapfrog.

``ShortRangeAccel`` is a ``torch.autograd.Function`` whose forward runs the
library's sort + pair kernel and whose backward runs its hand-written adjoint
kernel (the vector-Jacobian product of the accelerations with respect to the
positions, derived from Eq. p3m_gravity).  Kick and drift (Section 2.2.2,
operators K and D with a = 1) are Functions over the library's kick/drift
kernels; their adjoints reuse the kick kernel as an axpy.  ``leapfrog`` chains
them into a kick-drift-kick integrator with uniform time step and activation
checkpointing: only the states at segment boundaries are kept, and each
segment's forward is recomputed during the backward pass.

Tensors are (3, n) structure-of-arrays in the caller's particle order; the
sorting into the tile/subtile walk order happens inside each force call.
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint

from .shortrange import ShortRange


class ShortRangeAccel(torch.autograd.Function):
    """a = short-range acceleration(x) for all particles (all active)."""

    @staticmethod
    def forward(ctx, pos: torch.Tensor, sr: ShortRange, precision: int):
        work = pos.detach().clone()
        sr.sort(work)
        sr.build_pairs()
        acc_sorted = sr.forces(work, precision)
        acc = sr.unpermute(acc_sorted)
        ctx.sr = sr
        ctx.precision = precision
        ctx.save_for_backward(pos.detach())
        return acc

    @staticmethod
    def backward(ctx, acc_bar: torch.Tensor):
        (pos,) = ctx.saved_tensors
        sr, precision = ctx.sr, ctx.precision
        dt = torch.float32 if precision == 32 else torch.float64
        work = pos.clone()
        sr.sort(work)  # the context may have been used since the forward
        sr.build_pairs()
        abar_sorted = sr.permute(acc_bar.to(dt).contiguous())
        xbar_sorted = sr.vjp(work, abar_sorted, precision)
        xbar = sr.unpermute(xbar_sorted)
        return xbar.to(pos.dtype), None, None


class Kick(torch.autograd.Function):
    """q' = q + factor * a  (adjoint: qbar = q'bar, abar = factor * q'bar)."""

    @staticmethod
    def forward(ctx, mom: torch.Tensor, acc: torch.Tensor, sr: ShortRange, factor: float):
        out = mom.detach().clone()
        sr.kick(out, acc.detach().contiguous(), [factor])
        ctx.sr, ctx.factor = sr, factor
        ctx.acc_dtype = acc.dtype
        return out

    @staticmethod
    def backward(ctx, gout: torch.Tensor):
        gout = gout.contiguous()
        gacc = torch.zeros(gout.shape, dtype=ctx.acc_dtype, device=gout.device)
        ctx.sr.kick(gacc, gout, [ctx.factor])
        return gout, gacc, None, None


class Drift(torch.autograd.Function):
    """x' = wrap(x + factor * q)  (adjoint: xbar = x'bar, qbar = factor * x'bar)."""

    @staticmethod
    def forward(ctx, pos: torch.Tensor, mom: torch.Tensor, sr: ShortRange, factor: float):
        out = pos.detach().clone()
        sr.drift(out, mom.detach().contiguous(), factor)
        ctx.sr, ctx.factor = sr, factor
        ctx.mom_dtype = mom.dtype
        return out

    @staticmethod
    def backward(ctx, gout: torch.Tensor):
        gout = gout.contiguous()
        gmom = torch.zeros(gout.shape, dtype=ctx.mom_dtype, device=gout.device)
        ctx.sr.kick(gmom, gout, [ctx.factor])
        return gout, gmom, None, None


def short_range_accel(pos: torch.Tensor, sr: ShortRange, precision: int = 64) -> torch.Tensor:
    return ShortRangeAccel.apply(pos, sr, precision)


def _kdk_segment(sr: ShortRange, dt: float, n_steps: int, precision: int):
    def run(x, q, a):
        for _ in range(n_steps):
            q = Kick.apply(q, a, sr, 0.5 * dt)
            x = Drift.apply(x, q, sr, dt)
            a = ShortRangeAccel.apply(x, sr, precision)
            q = Kick.apply(q, a, sr, 0.5 * dt)
        return x, q, a

    return run


def leapfrog(pos: torch.Tensor, mom: torch.Tensor, sr: ShortRange, dt: float, n_steps: int = 16,
             checkpoint_every: int = 4, precision: int = 64):
    """Kick-drift-kick leapfrog (Section 2.2.2) with activation checkpointing.

    Returns (positions, momenta) after n_steps steps of size dt.  With
    checkpoint_every = k, the autograd graph keeps only the state every k steps
    and recomputes each k-step segment (forces included) in the backward pass.
    """
    x, q = pos, mom
    a = ShortRangeAccel.apply(x, sr, precision)
    done = 0
    while done < n_steps:
        k = min(checkpoint_every, n_steps - done) if checkpoint_every else n_steps - done
        seg = _kdk_segment(sr, dt, k, precision)
        if checkpoint_every and torch.is_grad_enabled():
            x, q, a = checkpoint(seg, x, q, a, use_reentrant=False)
        else:
            x, q, a = seg(x, q, a)
        done += k
    return x, q
