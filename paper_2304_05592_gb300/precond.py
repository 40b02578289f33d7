"""Learned preconditioner for FWI: an FNO that maps the RTM gradient of a
baseline model to the velocity perturbation that produced the data.

Pieces (every wave solve and every network step runs in libwave's kernels):

* ``make_pairs``: for each (baseline, perturbation) model pair, observed data
  F(v0 + dv) q and the velocity gradient of the misfit at v0, both from the
  plain solver (``wave_forward`` / ``wave_gradient``); the network input is the
  gradient divided by its RMS plus two coordinate channels, the target dv / 100
  m/s.
* ``train``: Adam on the mean squared error over shuffled mini-batches.
* ``fwi``: gradient-descent FWI where each iteration either takes the FNO
  update (accepted only if the data misfit drops, tried at full and half
  length) or falls back to the plain step: the depth-weighted gradient
  (``depth_weights``) with a safeguarded quadratic line search
  (``line_search``); the plain solver's misfit judges every update.  With
  ``net=None`` it is the plain method.

The paper runs FWI with stochastic shot subsampling and learned components
(arxiv 2304.05592, sections "Wave-equation-based inversion" and "Fourier neural
operator surrogates"); this module is that outer loop on the batched solver.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch

from . import fno, synth, wave

SCALE = 100.0  # m/s per unit of network output


@dataclass
class Acquisition:
    grid: wave.Grid
    src: np.ndarray
    rec: np.ndarray
    wavelet: torch.Tensor   # [nshot][nt][1]

    @staticmethod
    def of(p: synth.Problem, device="cuda") -> "Acquisition":
        q = wave.wave_ricker(p.f0, p.dt, p.nt, device=device)
        return Acquisition(wave.Grid.of(p), p.src, p.rec, q[None, :, None].repeat(p.nshot, 1, 1).contiguous())


class Misfit:
    """Data misfit 1/2 ||F(v) q - d||^2 and its velocity gradient."""

    def __init__(self, acq: Acquisition, d_obs: torch.Tensor):
        self.acq, self.d_obs = acq, d_obs
        dev = d_obs.device
        self._loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self._work = torch.zeros(1024, dtype=torch.float64, device=dev)
        self.solves = 0

    def value(self, v: torch.Tensor) -> float:
        a = self.acq
        d = wave.wave_forward(a.grid, v, a.src, a.wavelet, a.rec)
        fno.fno_mse(d, self.d_obs, None, self._loss, self._work)
        self.solves += 1
        return 0.5 * float(self._loss.item()) * d.numel()

    def gradient(self, v: torch.Tensor):
        a = self.acq
        phi, g, _ = wave.wave_gradient(a.grid, v, a.src, a.wavelet, a.rec, self.d_obs, store=wave.STORE_BF16,
                                       wrt=wave.WRT_VELOCITY)
        self.solves += 2
        return float(phi), g


def features(g: torch.Tensor) -> torch.Tensor:
    """Network input [1][3][nz][nx]: gradient / RMS(gradient) (scaled by a
    libwave kernel), z and x in [0, 1]."""
    nz, nx = g.shape
    out = torch.zeros((1, 3, nz, nx), dtype=torch.float32, device=g.device)
    rms = max((_dot(g, g) / g.numel()) ** 0.5, 1e-30)
    wave.wave_axpy(1.0 / rms, g.contiguous(), out[0, 0])
    out[0, 1] = torch.linspace(0, 1, nz, device=g.device)[:, None]
    out[0, 2] = torch.linspace(0, 1, nx, device=g.device)[None, :]
    return out


def make_pairs(seeds, acq: Acquisition, model=synth.plume_model, device="cuda", log=None):
    """Training pairs for the model seeds: (features of the gradient at the
    baseline, dv / SCALE), stacked as [n][3][nz][nx] and [n][1][nz][nx]."""
    g0 = acq.grid
    X, Y = [], []
    t0 = time.perf_counter()
    for k, s in enumerate(seeds):
        base, dv = model(int(s), nx=g0.nx, nz=g0.nz, h=g0.h)
        vb = torch.from_numpy(base).to(device)
        vt = torch.from_numpy(base + dv).to(device)
        d_obs = wave.wave_forward(g0, vt, acq.src, acq.wavelet, acq.rec)
        _, g = Misfit(acq, d_obs).gradient(vb)
        X.append(features(g))
        Y.append(torch.from_numpy(dv / SCALE).to(device)[None, None])
        if log and (k + 1) % 200 == 0:
            log(f"pairs {k + 1}/{len(seeds)} ({time.perf_counter() - t0:.1f} s)")
    return torch.cat(X), torch.cat(Y)


def train(net: fno.FNO2d, X: torch.Tensor, Y: torch.Tensor, epochs: int, batch: int, lr: float, seed: int = 0,
          log=None):
    """Adam on shuffled mini-batches with the learning rate halved at 50 % and
    75 % of the epochs; returns the mean loss of every epoch."""
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    hist = []
    for ep in range(epochs):
        f = 0.5 ** ((ep >= epochs // 2) + (ep >= 3 * epochs // 4))
        perm = rng.permutation(n)
        losses = []
        for i in range(0, n - batch + 1, batch):
            idx = torch.from_numpy(perm[i:i + batch]).to(X.device)
            losses.append(net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr * f))
        hist.append(float(torch.stack(losses).mean().item()))
        if log:
            log(f"epoch {ep + 1}/{epochs} loss {hist[-1]:.4e}")
    return hist


def _dot(x: torch.Tensor, y: torch.Tensor) -> float:
    return float(wave.wave_dot(x, y)[0].item())


def _trial(M: Misfit, v: torch.Tensor, a: float, d: torch.Tensor, vmin: float, vmax: float):
    """The model v + a d clamped to [vmin, vmax] (libwave kernels) and its misfit."""
    cand = v.clone()
    wave.wave_axpy(a, d, cand)
    wave.wave_clamp(cand, vmin, vmax)
    return cand, M.value(cand)


def depth_weights(nz: int, nx: int, device="cuda") -> torch.Tensor:
    """Depth preconditioner of the velocity gradient, w(z) = (z + 1) / nz: the
    standard compensation for the geometric spreading that makes the gradient
    of a surface survey decay with depth (an input table, built once)."""
    w = (torch.arange(nz, dtype=torch.float32, device=device) + 1.0) / nz
    return w[:, None].expand(nz, nx).contiguous()


def line_search(M: Misfit, v: torch.Tensor, phi: float, g: torch.Tensor, first_len: float = 50.0,
                vmin: float = 1400.0, vmax: float = 5000.0, max_evals: int = 6, weights: torch.Tensor = None):
    """Step along d = -g (or -w .* g with diagonal weights w) with a
    safeguarded quadratic line search on the misfit (interpolation as in
    Nocedal and Wright, ch. 3).  The first trial is the step that would zero
    a misfit falling linearly at slope <g, d>, a = phi / |<g, d>|, kept
    between 1 m/s and 4 first_len m/s in RMS over the grid (so neither a
    gradient that peaks at a few cells next to the sources nor a tiny
    residual sets its scale); the parabola through phi(0), the slope and
    phi(a) gives the next trial -- beyond a after a decrease (at most 4 a),
    within [0.1 a, 0.5 a] after an increase -- and at most max_evals misfits
    are evaluated.  Returns (model, misfit, step length in m/s RMS,
    evaluations); the old model and 0 if no trial reduced the misfit."""
    p = g if weights is None else wave.wave_mul(weights, g.clone())  # search along -p
    gp = _dot(g, p)
    if not gp > 0.0:
        return v, phi, 0.0, 0
    rms = (_dot(p, p) / p.numel()) ** 0.5
    slope = -gp
    a = min(max(phi / gp, 1.0 / rms), 4.0 * first_len / rms)
    best_v, best_phi, best_a = v, phi, 0.0
    cand, pa = _trial(M, v, -a, p, vmin, vmax)
    evals = 1
    if pa < phi:
        best_v, best_phi, best_a = cand, pa, a
    while evals < max_evals:
        curv = pa - phi - slope * a
        aq = -slope * a * a / (2.0 * curv) if curv > 0.0 else 4.0 * a
        if best_a > 0.0:
            # a decrease at a: one more trial at the parabola's minimum (or further out)
            nxt = min(max(aq, 0.1 * a), 4.0 * a)
            if abs(nxt - a) < 0.05 * a:
                break
            cand, pn = _trial(M, v, -nxt, p, vmin, vmax)
            evals += 1
            if pn < best_phi:
                best_v, best_phi, best_a = cand, pn, nxt
            break
        a = min(max(aq, 0.1 * a), 0.5 * a)
        cand, pa = _trial(M, v, -a, p, vmin, vmax)
        evals += 1
        if pa < phi:
            best_v, best_phi, best_a = cand, pa, a
    return best_v, best_phi, best_a * rms, evals


def plain_step(M: Misfit, v, phi, g, first_len: float = 50.0, vmin=1400.0, vmax=5000.0, weights=None):
    """The plain method's update: the line search along the (depth-weighted)
    negative gradient; returns the new model, its misfit and "plain" (or the
    old ones and "none" if no trial reduced the misfit)."""
    nv, nphi, step, _ = line_search(M, v, phi, g, first_len, vmin, vmax, weights=weights)
    return nv, nphi, ("plain" if step > 0.0 else "none")


def fwi(M: Misfit, v0: torch.Tensor, iters: int, net: fno.FNO2d = None, vmin=1400.0, vmax=5000.0, weights=None):
    """FWI from v0; returns misfits after 0..iters iterations and the step
    kinds.  weights: diagonal preconditioner of the plain step (None: the
    raw gradient)."""
    v = v0.clone()
    phi, g = M.gradient(v)
    hist, kinds = [phi], []
    for _ in range(iters):
        done = False
        if net is not None:
            upd = net.forward(features(g), train=False)[0, 0].contiguous()
            for a in (1.0, 0.5):
                cand, pc = _trial(M, v, a * SCALE, upd, vmin, vmax)
                if pc < phi:
                    v, phi, done = cand, pc, True
                    kinds.append("fno" if a == 1.0 else "fno/2")
                    break
        if not done:
            v, phi, kind = plain_step(M, v, phi, g, vmin=vmin, vmax=vmax, weights=weights)
            kinds.append(kind)
        hist.append(phi)
        # keep phi as evaluated for the accepted model (the gradient call's own
        # misfit sums in another order and may differ in the last bits)
        _, g = M.gradient(v)
    return hist, kinds, v


# A model whose plume changes the records by less than this fraction of their
# energy carries no plume signal within the record (the reflection arrives
# after it ends): its residual is FP32 rounding, and it is left out of the
# FWI comparison.
MIN_SIGNAL = 1e-9


def evaluate(seeds, acq: Acquisition, net: fno.FNO2d, iters: int, model=synth.plume_model, device="cuda",
             depth_weighting: bool = True):
    """Misfit and model error after each iteration, plain vs preconditioned,
    on held-out model seeds (both normalised by the starting values).  The
    plain method (and the FNO runs' fallback) steps along the depth-weighted
    gradient unless depth_weighting is off.  Seeds whose plume leaves no
    signal in the records (MIN_SIGNAL) are listed in "no_signal" and skipped."""
    g0 = acq.grid
    W = depth_weights(g0.nz, g0.nx, device) if depth_weighting else None
    out = {"plain": [], "fno": [], "err_plain": [], "err_fno": [], "kinds": [], "kinds_plain": [], "no_signal": []}
    for s in seeds:
        base, dv = model(int(s), nx=g0.nx, nz=g0.nz, h=g0.h)
        vb = torch.from_numpy(base).to(device)
        vt = torch.from_numpy(base + dv).to(device)
        d_obs = wave.wave_forward(g0, vt, acq.src, acq.wavelet, acq.rec)
        M = Misfit(acq, d_obs)
        if M.value(vb) < MIN_SIGNAL * 0.5 * _dot(d_obs, d_obs):
            out["no_signal"].append(int(s))
            continue
        e0 = float(torch.linalg.vector_norm(vb - vt))
        hp, kinds_p, vp = fwi(M, vb, iters, weights=W)
        hf, kinds, vf = fwi(M, vb, iters, net, weights=W)
        out["kinds_plain"].append(kinds_p)
        out["plain"].append(np.array(hp) / hp[0])
        out["fno"].append(np.array(hf) / hf[0])
        out["err_plain"].append(float(torch.linalg.vector_norm(vp - vt)) / e0)
        out["err_fno"].append(float(torch.linalg.vector_norm(vf - vt)) / e0)
        out["kinds"].append(kinds)
    return out


def run(npairs: int = 2000, nheld: int = 200, nfwi: int = 32, iters: int = 3, epochs: int = 30, batch: int = 8,
        lr: float = 1e-3, nt: int = 2000, nshot: int = 8, log=print) -> dict:
    """The full learned-preconditioner workload: plume models on a 512 x 256
    grid at 10 m (baselines with 2-8 % patchy velocity drops), 8 surface shots
    with a 15 Hz Ricker over nt steps of 0.8 ms, npairs (gradient, dv) pairs
    from the plain solver (the last nheld held out), the 4-layer width-32
    16x16-mode FNO trained in FP32 and run with BF16 activations, and FWI
    with and without it on nfwi held-out models."""
    dev = "cuda"
    p = synth.plume_acquisition(nx=512, nz=256, h=10.0, nshot=nshot, nt=nt)
    acq = Acquisition.of(p, dev)
    res = {"grid": "512x256 at 10 m", "nshot": nshot, "nt": nt, "pairs": npairs, "held_out": nheld}
    t = time.perf_counter()
    X, Y = make_pairs(range(npairs), acq, device=dev, log=log)
    torch.cuda.synchronize()
    res["pair_generation_s"] = time.perf_counter() - t
    ntr = npairs - nheld
    net = fno.FNO2d(fno.FNOConfig(), 256, 512, dev, seed=0)
    t = time.perf_counter()
    hist = train(net, X[:ntr], Y[:ntr], epochs, batch, lr, log=log)
    torch.cuda.synchronize()
    res["train_s"] = time.perf_counter() - t
    res["train_samples_per_s"] = epochs * (ntr // batch) * batch / res["train_s"]
    res["loss_history"] = hist
    Xh, Yh = X[ntr:].contiguous(), Y[ntr:].contiguous()
    res["heldout_loss_fp32"] = float(np.mean([net.loss(Xh[i:i + batch].contiguous(), Yh[i:i + batch].contiguous())
                                              for i in range(0, nheld, batch)]))
    res["heldout_loss_bf16"] = float(np.mean([net.loss(Xh[i:i + batch].contiguous(), Yh[i:i + batch].contiguous(),
                                                       bf16=True) for i in range(0, nheld, batch)]))
    res["target_variance"] = float((Yh.double() ** 2).mean())
    for name, bf in (("fp32", False), ("bf16", True)):
        xb = Xh[:batch].contiguous()
        for _ in range(3):
            net.forward(xb, train=False, bf16=bf)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(10):
            net.forward(xb, train=False, bf16=bf)
        torch.cuda.synchronize()
        res[f"inference_samples_per_s_{name}"] = 10 * batch / (time.perf_counter() - t)
    t = time.perf_counter()
    ev = evaluate(range(ntr, ntr + nfwi), acq, net, iters, device=dev)
    res["fwi_s"] = time.perf_counter() - t
    res["fwi_models"] = nfwi - len(ev["no_signal"])
    res["fwi_models_without_plume_signal"] = ev["no_signal"]
    res["misfit_plain"] = np.mean(ev["plain"], axis=0).tolist()
    res["misfit_fno"] = np.mean(ev["fno"], axis=0).tolist()
    res["model_error_plain"] = float(np.mean(ev["err_plain"]))
    res["model_error_fno"] = float(np.mean(ev["err_fno"]))
    kinds = [k for ks in ev["kinds"] for k in ks]
    res["step_kinds"] = {k: kinds.count(k) for k in sorted(set(kinds))}
    kp = [k for ks in ev["kinds_plain"] for k in ks]
    res["step_kinds_plain"] = {k: kp.count(k) for k in sorted(set(kp))}
    res["plain_descent_rate"] = kp.count("plain") / max(len(kp), 1)
    return res


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="train and evaluate the FNO preconditioner on plume models")
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--held", type=int, default=200)
    ap.add_argument("--fwi", type=int, default=32)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--out", default=None, help="write the result JSON here")
    a = ap.parse_args()
    r = run(a.pairs, a.held, a.fwi, a.iters, a.epochs, log=lambda m: print(m, flush=True))
    print(json.dumps(r))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
