"""Fourier neural operator (Li et al. 2020) on libwave's FNO kernels
(``include/fno.h``), used as a learned preconditioner: it maps a normalised
RTM gradient to a velocity update.  The paper trains FNOs as learned
surrogates with reverse-mode AD (arxiv 2304.05592, section "Fourier neural
operator surrogates"); here forward, backward, loss and optimiser steps are
the library's CUDA kernels and this module only sequences them and marshals
pointers (no CPU path: a missing library or a CPU tensor raises).

Network (width W, hidden H, L layers, mz x mx modes):
    v = P x + p
    v = act(W_l v + b_l + S(R_l * T(v)))   l = 0..L-1, act = GELU except l = L-1
    out = Q2 GELU(Q1 v + q1) + q2
with T / S the truncated DFT and its real inverse and R_l * X the per-mode
complex channel mix.  Parameters live in one flat float32 buffer (complex
weights as interleaved re/im pairs), so Adam runs as one kernel.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import wave

ACT_NONE, ACT_GELU = 0, 1
_BOUND = False


def _lib():
    global _BOUND
    lib = wave._lib()
    if not _BOUND:
        P, I, L, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        sig = {
            "fno_tables": [I, I, I, I, P, P, P, P, P, P],
            "fno_dft_x": [L, I, I, P, I, P, P, P],
            "fno_dft_z": [I, I, I, I, P, P, P, P],
            "fno_idft_z": [I, I, I, I, P, P, P, P],
            "fno_mix": [I, I, I, I, P, P, P, P],
            "fno_mix_backward": [I, I, I, I, P, P, P, P, P, P],
            "fno_mix_idft_z": [I, I, I, I, I, I, P, P, P, P, P],
            "fno_combine": [I, I, I, I, I, I, P, I, P, I, P, P, P, I, P, P, I, P],
            "fno_project": [I, I, I, I, I, P, I, P, P, P, P, P, P],
            "fno_wgrad": [I, I, I, L, P, P, P, P, P, P],
            "fno_gelu_backward": [L, P, P, P, P],
            "fno_mse": [L, P, P, P, P, P, P],
            "fno_adam": [L, P, P, P, P, D, D, D, D, I, P],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = I
        lib.fno_set_tensor_cores.argtypes = [I]
        lib.fno_set_tensor_cores.restype = I
        lib.fno_tensor_core_status.argtypes = []
        lib.fno_tensor_core_status.restype = I
        lib.fno_wgrad_work_floats.argtypes = [I, I, I, L]
        lib.fno_wgrad_work_floats.restype = ctypes.c_size_t
        _BOUND = True
    return lib


def _p(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("FNO kernels take CUDA tensors (there is no CPU path)")
    if not t.is_contiguous():
        raise TypeError("FNO kernels take contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _call(name: str, *args):
    st = getattr(_lib(), name)(*args)
    if st:
        raise wave.WaveError(st, name)


def _s(stream):
    return wave._stream(stream)


# --- C ABI, one Python function per entry point ------------------------------------

def fno_tables(Nz, Nx, mz, mx, device="cuda", stream=None):
    """The x tables (fwd, inv, bwd, adj; [Nx][mx][2] each) and the z table."""
    tx = [torch.empty((Nx, mx, 2), dtype=torch.float32, device=device) for _ in range(4)]
    tz = torch.empty((Nz, 2 * mz, 2), dtype=torch.float32, device=device)
    _call("fno_tables", Nz, Nx, mz, mx, *[_p(t) for t in tx], _p(tz), _s(stream))
    return tx, tz


def fno_dft_x(inp, mx, table, out=None, stream=None):
    Nx = inp.shape[-1]
    rows = inp.numel() // Nx
    if out is None:
        out = torch.empty((rows, mx, 2), dtype=torch.float32, device=inp.device)
    _call("fno_dft_x", rows, Nx, mx, _p(inp), int(inp.dtype == torch.bfloat16), _p(table), _p(out), _s(stream))
    return out


def fno_dft_z(inp, nb, Nz, mz, mx, tz, out=None, stream=None):
    if out is None:
        out = torch.empty((nb, 2 * mz, mx, 2), dtype=torch.float32, device=inp.device)
    _call("fno_dft_z", nb, Nz, mz, mx, _p(inp), _p(tz), _p(out), _s(stream))
    return out


def fno_idft_z(inp, nb, Nz, mz, mx, tz, out=None, stream=None):
    if out is None:
        out = torch.empty((nb, Nz, mx, 2), dtype=torch.float32, device=inp.device)
    _call("fno_idft_z", nb, Nz, mz, mx, _p(inp), _p(tz), _p(out), _s(stream))
    return out


def fno_mix(X, R, B, Ci, Co, nmode, out=None, stream=None):
    if out is None:
        out = torch.empty((B, Co, nmode, 2), dtype=torch.float32, device=X.device)
    _call("fno_mix", B, Ci, Co, nmode, _p(X), _p(R), _p(out), _s(stream))
    return out


def fno_mix_idft_z(X, R, B, Ci, Co, Nz, mz, mx, tz, out=None, stream=None):
    """fno_mix then fno_idft_z in one pass: [B][Co][Nz][mx][2] from X [B][Ci][2mz][mx][2]."""
    if out is None:
        out = torch.empty((B * Co, Nz, mx, 2), dtype=torch.float32, device=X.device)
    _call("fno_mix_idft_z", B, Ci, Co, Nz, mz, mx, _p(X), _p(R), _p(tz), _p(out), _s(stream))
    return out


def fno_mix_backward(X, R, dY, B, Ci, Co, nmode, dX=None, dR=None, stream=None):
    _call("fno_mix_backward", B, Ci, Co, nmode, _p(X), _p(R), _p(dY), _p(dX), _p(dR), _s(stream))
    return dX, dR


def fno_combine(inp, M, Co, m_trans=False, bias=None, T=None, table=None, mx=1, act=ACT_NONE, pre=None, out=None,
                out_dtype=torch.float32, stream=None):
    B, Ci, Nz, Nx = inp.shape
    if out is None:
        out = torch.empty((B, Co, Nz, Nx), dtype=out_dtype, device=inp.device)
    _call("fno_combine", B, Ci, Co, Nz, Nx, mx, _p(inp), int(inp.dtype == torch.bfloat16), _p(M), int(m_trans),
          _p(bias), _p(T), _p(table), act, _p(pre), _p(out), int(out.dtype == torch.bfloat16), _s(stream))
    return out


def fno_project(inp, Q1, q1, Q2, q2, out=None, stream=None):
    """out = q2 + Q2 GELU(Q1 inp + q1) per pixel, the hidden channels kept on chip."""
    B, Ci, Nz, Nx = inp.shape
    H = Q1.shape[0]
    if out is None:
        out = torch.empty((B, 1, Nz, Nx), dtype=torch.float32, device=inp.device)
    _call("fno_project", B, Ci, H, Nz, Nx, _p(inp), int(inp.dtype == torch.bfloat16), _p(Q1), _p(q1), _p(Q2), _p(q2),
          _p(out), _s(stream))
    return out


def fno_set_tensor_cores(on: bool):
    """Allow (the default) or forbid the tcgen05 path of fno_combine's BF16 inference."""
    _call("fno_set_tensor_cores", int(bool(on)))


def fno_tensor_core_status() -> int:
    """0, or 6 (WAVE_ERR_TIMEOUT) if a tensor-core launch gave up since the last call."""
    return int(_lib().fno_tensor_core_status())


def fno_wgrad_work_floats(B, Ci, Co, npix) -> int:
    return int(_lib().fno_wgrad_work_floats(B, Ci, Co, npix))


def fno_wgrad(dU, inp, dM, dbias, work, stream=None):
    B, Co = dU.shape[0], dU.shape[1]
    Ci = inp.shape[1]
    npix = dU[0, 0].numel()
    _call("fno_wgrad", B, Ci, Co, npix, _p(dU), _p(inp), _p(dM), _p(dbias), _p(work), _s(stream))


def fno_gelu_backward(dout, pre, out=None, stream=None):
    if out is None:
        out = torch.empty_like(pre)
    _call("fno_gelu_backward", pre.numel(), _p(dout), _p(pre), _p(out), _s(stream))
    return out


def fno_mse(pred, target, dpred, loss, work, stream=None):
    _call("fno_mse", pred.numel(), _p(pred), _p(target), _p(dpred), _p(loss), _p(work), _s(stream))


def fno_adam(p, g, m, v, lr, t, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    _call("fno_adam", p.numel(), _p(p), _p(g), _p(m), _p(v), lr, b1, b2, eps, t, _s(stream))


# --- the network ------------------------------------------------------------------------

@dataclass(frozen=True)
class FNOConfig:
    cin: int = 3       # input channels: normalised gradient, z, x
    width: int = 32
    hidden: int = 64
    layers: int = 4
    mz: int = 16
    mx: int = 16


class FNO2d:
    """FNO on a fixed Nz x Nx grid; all arithmetic in libwave's kernels."""

    def __init__(self, cfg: FNOConfig, Nz: int, Nx: int, device="cuda", seed: int = 0):
        self.cfg, self.Nz, self.Nx = cfg, Nz, Nx
        self.device = torch.device(device)
        W, H, KZ = cfg.width, cfg.hidden, 2 * cfg.mz
        shapes = [("P", (W, cfg.cin)), ("p", (W,))]
        for l in range(cfg.layers):
            shapes += [(f"W{l}", (W, W)), (f"b{l}", (W,)), (f"R{l}", (W, W, KZ, cfg.mx, 2))]
        shapes += [("Q1", (H, W)), ("q1", (H,)), ("Q2", (1, H)), ("q2", (1,))]
        self.offsets = {}
        n = 0
        for name, shp in shapes:
            self.offsets[name] = (n, shp)
            n += (math.prod(shp) + 3) // 4 * 4  # 16-byte aligned views
        self.nparam = n
        self.params = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        (self.tx_fwd, self.tx_inv, self.tx_bwd, self.tx_adj), self.tz = fno_tables(Nz, Nx, cfg.mz, cfg.mx, self.device)
        self._loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        self._mse_work = torch.zeros(1024, dtype=torch.float64, device=self.device)
        self._init(seed)
        self._cache = None

    # parameter views
    def view(self, name: str, which: torch.Tensor = None) -> torch.Tensor:
        off, shp = self.offsets[name]
        buf = self.params if which is None else which
        return buf[off:off + math.prod(shp)].view(shp)

    def grad(self, name: str) -> torch.Tensor:
        return self.view(name, self.grads)

    def _init(self, seed: int):
        """Seeded initial weights: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for the
        pointwise layers and (1/W^2) U(0,1) re/im for the spectral weights."""
        rng = np.random.default_rng(seed)
        cfg = self.cfg
        for name, (off, shp) in self.offsets.items():
            if name.startswith("R"):
                a = rng.uniform(0, 1, shp) / (cfg.width * cfg.width)
            else:
                fan = shp[1] if len(shp) == 2 else {"p": cfg.cin, "q1": cfg.width, "q2": cfg.hidden}.get(
                    name, cfg.width)
                k = 1.0 / math.sqrt(fan)
                a = rng.uniform(-k, k, shp)
            self.view(name).copy_(torch.from_numpy(a.astype(np.float32)))

    def load(self, params: dict):
        """Copies a dict of numpy arrays (complex spectral weights) into the buffer."""
        for name, (off, shp) in self.offsets.items():
            a = np.asarray(params[name])
            if np.iscomplexobj(a):
                a = np.stack([a.real, a.imag], axis=-1)
            self.view(name).copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).reshape(shp))

    def export(self, grads: bool = False) -> dict:
        out = {}
        for name, (off, shp) in self.offsets.items():
            a = (self.grad(name) if grads else self.view(name)).detach().cpu().numpy().astype(np.float64)
            out[name] = a[..., 0] + 1j * a[..., 1] if name.startswith("R") else a
        return out

    def _work(self, B):
        cfg = self.cfg
        npix = self.Nz * self.Nx
        need = max(fno_wgrad_work_floats(B, ci, co, npix) for ci, co in
                   ((cfg.hidden, 1), (cfg.width, cfg.hidden), (cfg.width, cfg.width), (cfg.cin, cfg.width)))
        if getattr(self, "_wg", None) is None or self._wg.numel() < need:
            self._wg = torch.empty(need, dtype=torch.float32, device=self.device)
        return self._wg

    # forward / backward
    def forward(self, x: torch.Tensor, train: bool = True, bf16: bool = False) -> torch.Tensor:
        """x[B][cin][Nz][Nx] (float32) -> out[B][1][Nz][Nx] (float32).  With
        bf16, activations are stored in bfloat16 (inference only)."""
        cfg, Nz, Nx = self.cfg, self.Nz, self.Nx
        if x.shape[1:] != (cfg.cin, Nz, Nx):
            raise ValueError(f"input must be [B][{cfg.cin}][{Nz}][{Nx}], got {tuple(x.shape)}")
        if bf16 and train:
            raise ValueError("bf16 activations are for inference only")
        B, W, KZ, mz, mx = x.shape[0], cfg.width, 2 * cfg.mz, cfg.mz, cfg.mx
        adt = torch.bfloat16 if bf16 else torch.float32
        v = fno_combine(x, self.view("P"), W, bias=self.view("p"), out_dtype=adt)
        layers = []
        for l in range(cfg.layers):
            last = l == cfg.layers - 1
            T1 = fno_dft_x(v, mx, self.tx_fwd)
            X = fno_dft_z(T1, B * W, Nz, mz, mx, self.tz)
            T2 = fno_mix_idft_z(X, self.view(f"R{l}"), B, W, W, Nz, mz, mx, self.tz)
            pre = torch.empty((B, W, Nz, Nx), dtype=torch.float32, device=x.device) if (train and not last) else None
            vn = fno_combine(v, self.view(f"W{l}"), W, bias=self.view(f"b{l}"), T=T2, table=self.tx_inv, mx=mx,
                             act=ACT_NONE if last else ACT_GELU, pre=pre, out_dtype=adt)
            if train:
                layers.append((v, X, pre if not last else vn))
            v = vn
        if not train:
            self._cache = None
            return fno_project(v, self.view("Q1"), self.view("q1"), self.view("Q2"),
                               self.view("q2"))
        hpre = torch.empty((B, cfg.hidden, Nz, Nx), dtype=torch.float32, device=x.device)
        h = fno_combine(v, self.view("Q1"), cfg.hidden, bias=self.view("q1"), act=ACT_GELU, pre=hpre, out_dtype=adt)
        out = fno_combine(h, self.view("Q2"), 1, bias=self.view("q2"))
        self._cache = dict(x=x, layers=layers, v=v, hpre=hpre, h=h)
        return out

    def backward(self, dout: torch.Tensor):
        """Gradients of sum(dout * out) for the last forward(train=True) into self.grads."""
        if self._cache is None:
            raise RuntimeError("backward needs a preceding forward(train=True)")
        c, cfg, Nz, Nx = self._cache, self.cfg, self.Nz, self.Nx
        B, W, H, mz, mx = dout.shape[0], cfg.width, cfg.hidden, cfg.mz, cfg.mx
        KZ = 2 * mz
        work = self._work(B)
        fno_wgrad(dout, c["h"], self.grad("Q2"), self.grad("q2"), work)
        dh = fno_combine(dout, self.view("Q2"), H, m_trans=True)
        dhpre = fno_gelu_backward(dh, c["hpre"])
        fno_wgrad(dhpre, c["v"], self.grad("Q1"), self.grad("q1"), work)
        dv = fno_combine(dhpre, self.view("Q1"), W, m_trans=True)
        for l in reversed(range(cfg.layers)):
            v, X, u = c["layers"][l]
            du = fno_gelu_backward(dv, u) if l < cfg.layers - 1 else dv
            fno_wgrad(du, v, self.grad(f"W{l}"), self.grad(f"b{l}"), work)
            dT2 = fno_dft_x(du, mx, self.tx_bwd)
            dY = fno_dft_z(dT2, B * W, Nz, mz, mx, self.tz)
            dX = torch.empty_like(X)
            fno_mix_backward(X, self.view(f"R{l}"), dY, B, W, W, KZ * mx, dX=dX, dR=self.grad(f"R{l}"))
            dT1 = fno_idft_z(dX, B * W, Nz, mz, mx, self.tz)
            dv = fno_combine(du, self.view(f"W{l}"), W, m_trans=True, T=dT1, table=self.tx_adj, mx=mx)
        fno_wgrad(dv, c["x"], self.grad("P"), self.grad("p"), work)
        self._cache = None

    def train_step(self, x: torch.Tensor, target: torch.Tensor, lr: float) -> torch.Tensor:
        """One Adam step on the MSE loss; returns the loss (a device scalar)."""
        out = self.forward(x, train=True)
        dout = torch.empty_like(out)
        fno_mse(out, target, dout, self._loss, self._mse_work)
        self.backward(dout)
        self.t += 1
        fno_adam(self.params, self.grads, self.m, self.v, lr, self.t)
        return self._loss.clone()

    def loss(self, x: torch.Tensor, target: torch.Tensor, bf16: bool = False) -> float:
        out = self.forward(x, train=False, bf16=bf16)
        fno_mse(out, target, None, self._loss, self._mse_work)
        return float(self._loss.item())
