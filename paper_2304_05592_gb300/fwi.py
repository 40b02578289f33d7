"""FWI outer loops on the batched solver.

* ``fwi_subsampled``: gradient descent where each iteration uses a few shots
  drawn at random with replacement, which is how the paper keeps the count of
  wave-equation solves down (arxiv 2304.05592, section "Putting it all together":
  four random shots per iteration, 200 iterations, about 25 passes through the
  data); the step along the subset gradient is found by a line search on the
  subset misfit, and models stay within velocity bounds.
* ``timelapse_gradients``: the block-diagonal time-lapse operator
  F(v) = diag(F^i(v^i) q^i) of the same section: each vintage has its own
  model (and may have its own wavelet); all (vintage, shot) pairs run in one
  uneven batch (two persistent sweeps), and the shot gradients of each vintage
  are summed on the device.

Wave solves, misfits and model updates run in libwave's kernels; this module
draws the shot indices and sequences the calls.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import wave
from .precond import Acquisition, Misfit, line_search
from .wave import BatchProblem


@dataclass
class FWIHistory:
    shots: list = field(default_factory=list)        # shot indices of each iteration
    subset_misfit: list = field(default_factory=list)
    step: list = field(default_factory=list)         # accepted step (m/s RMS over the grid), 0 = none
    full_misfit: list = field(default_factory=list)  # (iteration, misfit over all shots)
    solves: int = 0


def _subset(acq: Acquisition, d_obs: torch.Tensor, shots: np.ndarray):
    idx = torch.from_numpy(shots).to(d_obs.device)
    sub = Acquisition(acq.grid, acq.src[shots], acq.rec[shots], acq.wavelet.index_select(0, idx).contiguous())
    return sub, d_obs.index_select(0, idx).contiguous()


def fwi_subsampled(acq: Acquisition, d_obs: torch.Tensor, v0: torch.Tensor, iters: int, nsub: int = 4,
                   seed: int = 0, first_len: float = 50.0, vmin: float = 1400.0, vmax: float = 5000.0,
                   full_every: int = 0):
    """Returns (model, history).  full_every > 0 also records the misfit over
    all shots every that many iterations (and at the start and the end)."""
    rng = np.random.default_rng(seed)
    nshot = acq.src.shape[0]
    v = v0.clone()
    h = FWIHistory()
    full = Misfit(acq, d_obs)
    if full_every:
        h.full_misfit.append((0, full.value(v)))
    for it in range(iters):
        shots = rng.integers(0, nshot, nsub)
        sub, dsub = _subset(acq, d_obs, shots)
        M = Misfit(sub, dsub)
        phi, g = M.gradient(v)
        v, phi, taken, _ = line_search(M, v, phi, g, first_len, vmin, vmax)
        h.shots.append(shots.tolist())
        h.subset_misfit.append(phi)
        h.step.append(taken)
        h.solves += M.solves
        if full_every and ((it + 1) % full_every == 0 or it + 1 == iters):
            h.full_misfit.append((it + 1, full.value(v)))
    h.solves += full.solves
    return v, h


def timelapse_gradients(grid: wave.Grid, models, src, rec, wavelets, d_obs, store: int = wave.STORE_BF16,
                        wrt: int = wave.WRT_VELOCITY, batched: bool = True):
    """Misfit and gradient of every vintage of a time-lapse survey.

    models: list of nv velocity models [nz][nx] (device); src, rec: [nshot][n][2]
    host coordinates shared by the vintages; wavelets: [nshot][nt][nsrc] (shared)
    or a list of nv of them; d_obs: list of nv records [nshot][nt][nrec].
    Returns (misfits [nv], gradients [nv] of [nz][nx])."""
    nv = len(models)
    ws = wavelets if isinstance(wavelets, (list, tuple)) else [wavelets] * nv
    nshot = src.shape[0]
    if not batched:
        out = [wave.wave_gradient(grid, models[i], src, ws[i], rec, d_obs[i], store=store, wrt=wrt)
               for i in range(nv)]
        return [o[0] for o in out], [o[1] for o in out]
    probs = [BatchProblem(grid, models[i], src[s], ws[i][s].contiguous(), rec[s], d_obs[i][s].contiguous())
             for i in range(nv) for s in range(nshot)]
    misfits, grads = wave.wave_gradient_batch(probs, store=store, wrt=wrt)
    g_out, m_out = [], []
    for i in range(nv):
        acc = grads[i * nshot].clone()
        for s in range(1, nshot):
            wave.wave_axpy(1.0, grads[i * nshot + s], acc)
        g_out.append(acc)
        m_out.append(float(sum(misfits[i * nshot:(i + 1) * nshot])))
    return m_out, g_out
