"""Differentiable wave modelling for PyTorch (the AD rule of the paper's
section "Wave-equation-based inversion": the pullback of d = F(m) q returns
J' dy with respect to the model and F' dy with respect to the source).

``ForwardModel.apply(vel, wavelet, grid, src_xyz, rec_xyz)`` returns the shot
records; its backward calls libwave's ``wave_jacobian_adjoint`` (checkpointed
or BF16-store adjoint-state gradient, with the chain rule to velocity applied
in the library) and ``wave_adjoint``.  No arithmetic of the method happens in
Python.
"""
from __future__ import annotations

import torch

from . import wave


class ForwardModel(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vel, wavelet, grid, src_xyz, rec_xyz, store=wave.STORE_CHECKPOINT, nsnap=64):
        vel = vel.contiguous()
        wavelet = wavelet.contiguous()
        ctx.save_for_backward(vel, wavelet)
        ctx.meta = (grid, src_xyz, rec_xyz, store, nsnap)
        return wave.wave_forward(grid, vel, src_xyz, wavelet, rec_xyz)

    @staticmethod
    def backward(ctx, dy):
        vel, wavelet = ctx.saved_tensors
        grid, src, rec, store, nsnap = ctx.meta
        dy = dy.contiguous()
        g_vel = g_wav = None
        if ctx.needs_input_grad[0]:
            g_vel = wave.wave_jacobian_adjoint(grid, vel, src, wavelet, rec, dy, store=store, nsnap=nsnap,
                                               wrt=wave.WRT_VELOCITY)
        if ctx.needs_input_grad[1]:
            g_wav = wave.wave_adjoint(grid, vel, src, rec, dy)
        return g_vel, g_wav, None, None, None, None, None


def forward_model(vel, wavelet, grid, src_xyz, rec_xyz, store=wave.STORE_CHECKPOINT, nsnap=64):
    """Shot records with autograd support for vel and wavelet."""
    return ForwardModel.apply(vel, wavelet, grid, src_xyz, rec_xyz, store, nsnap)


class BatchMisfit(torch.autograd.Function):
    """Misfits of an uneven batch of problems as a differentiable function of
    their velocity models: forward runs wave_gradient_batch once (both sweeps)
    and keeps the velocity gradients for the backward pass."""

    @staticmethod
    def forward(ctx, problems, store, use_graph, *vels):
        misfits, grads = wave.wave_gradient_batch(problems, store=store, wrt=wave.WRT_VELOCITY, use_graph=use_graph)
        ctx.grads = grads
        return torch.tensor(misfits, dtype=torch.float64, device=vels[0].device)

    @staticmethod
    def backward(ctx, gout):
        return (None, None, None) + tuple(g * gout[i].to(g.dtype) for i, g in enumerate(ctx.grads))


def batch_misfit(problems, store=wave.STORE_BF16, use_graph=True):
    """Per-problem misfits [nprob] with gradients flowing to each problem's vel."""
    return BatchMisfit.apply(problems, store, use_graph, *[p.vel for p in problems])
