"""Least-squares reverse-time migration on the GPU.

Fits a squared-slowness perturbation dm to data dd through the Born operator
J = judiJacobian(F, q) of the paper (section "Wave-equation-based
inversion"): min 1/2 ||J dm - dd||^2, by conjugate gradients on the normal
equations J'J dm = J' dd (the least-squares form CGLS, from dm = 0).  J runs
as ``wave_born`` and J' as ``wave_jacobian_adjoint``; the vector updates and
dot products are libwave kernels (``wave_axpy``, ``wave_axpby``,
``wave_dot``); only the two scalar ratios of each iteration are formed on
the host from the dot products.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import wave


@dataclass
class LsrtmHistory:
    rnorm: list = field(default_factory=list)  # ||dd - J dm_k||, k = 0..niter
    iterates: list = field(default_factory=list)  # dm_1 .. dm_niter (when kept)


def _dot(x: torch.Tensor, y: torch.Tensor, buf: torch.Tensor) -> float:
    return float(wave.wave_dot(x, y, out=buf)[0].item())


def lsrtm_cgls(grid: wave.Grid, vel: torch.Tensor, src, wavelet: torch.Tensor, rec, dd: torch.Tensor, niter: int,
               store: int = wave.STORE_CHECKPOINT, nsnap: int = 64, keep_iterates: bool = False):
    """CGLS for least-squares RTM.  vel [nz][nx] (device), dd [nshot][nt][nrec]
    (device).  Returns (dm [phys shape], LsrtmHistory)."""
    buf = torch.empty(1 + wave.DOT_PARTIALS, dtype=torch.float64, device=vel.device)
    x = torch.zeros(grid.phys_shape, dtype=torch.float32, device=vel.device)
    r = dd.detach().clone().contiguous()
    s = wave.wave_jacobian_adjoint(grid, vel, src, wavelet, rec, r, store=store, nsnap=nsnap)
    p = s.clone()
    gamma = _dot(s, s, buf)
    hist = LsrtmHistory(rnorm=[_dot(r, r, buf) ** 0.5])
    for _ in range(niter):
        q = wave.wave_born(grid, vel, src, wavelet, rec, p)
        qq = _dot(q, q, buf)
        if qq == 0.0 or gamma == 0.0:
            break
        alpha = gamma / qq
        wave.wave_axpy(alpha, p, x)
        wave.wave_axpy(-alpha, q, r)
        wave.wave_jacobian_adjoint(grid, vel, src, wavelet, rec, r, store=store, nsnap=nsnap, grad=s)
        gamma_new = _dot(s, s, buf)
        wave.wave_axpby(1.0, s, gamma_new / gamma, p)  # p = s + beta p
        gamma = gamma_new
        hist.rnorm.append(_dot(r, r, buf) ** 0.5)
        if keep_iterates:
            hist.iterates.append(x.clone())
    return x, hist
