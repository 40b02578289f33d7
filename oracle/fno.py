"""FP64 CPU oracle of the Fourier neural operator used as a learned
preconditioner (test infrastructure only; only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it).

The network is the FNO of Li et al. (2020), which the paper cites for its
neural surrogates (section "Fourier neural operator surrogates") and which is
used here to map an RTM gradient to a velocity update.  Architecture:

* lift: v = P x + p (pointwise, Cin -> W channels);
* L Fourier layers: v <- act(W_l v + b_l + K_l v), act = GELU except after the
  last layer, K_l the spectral convolution below;
* projection: out = Q2 GELU(Q1 v + q1) + q2 (W -> H -> 1 channels).

Spectral convolution of a real field v[z, x] (Nz x Nx) with mz, mx modes:

* X = T v, the truncated DFT: X[kz, kx] = sum_{z,x} v[z,x] exp(-i psi), with
  psi = 2 pi (kz z / Nz + kx x / Nx), kz in {0..mz-1} u {Nz-mz..Nz-1} (the
  rows are stored in that order), kx in {0..mx-1};
* Y[o, k] = sum_i X[i, k] R[i, o, k] (complex weights per mode);
* y = S Y, the truncated real inverse: y[z,x] = (1/(Nz Nx)) sum_k w_kx
  Re(Y[k] exp(+i psi)) with w_0 = 1 and w_kx = 2 for kx > 0 (the conjugate
  half of the spectrum).

The DFTs use numpy.fft (a library routine); every adjoint is written out from
its definition.  Complex gradients follow dR = dL/dRr + i dL/dRi, so for
Y = X R: dX = dY conj(R) and dR = conj(X) dY.  GELU is the exact form
x Phi(x).  Pinned by ``tests/test_oracle_fno.py``: brute-force DFT sums,
exact reconstruction of band-limited fields, single-mode sign checks, dot
tests of both adjoints, closed-form GELU values and a finite-difference check
of the full network gradient.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import erf


@dataclass(frozen=True)
class Config:
    cin: int = 3       # input channels (gradient, z, x)
    width: int = 32    # W
    hidden: int = 64   # H, projection
    layers: int = 4    # L
    mz: int = 16
    mx: int = 16


def kz_rows(Nz: int, mz: int) -> np.ndarray:
    """Wavenumber rows kept along z, in storage order."""
    return np.concatenate([np.arange(mz), np.arange(Nz - mz, Nz)])


# --- transforms -------------------------------------------------------------

def dft_trunc(v: np.ndarray, mz: int, mx: int) -> np.ndarray:
    """X = T v for v[..., Nz, Nx] real -> X[..., 2mz, mx] complex."""
    Nz = v.shape[-2]
    full = np.fft.fft2(v, axes=(-2, -1))
    return full[..., kz_rows(Nz, mz), :][..., :mx]


def dft_trunc_adjoint(dX: np.ndarray, Nz: int, Nx: int) -> np.ndarray:
    """T' dX: dv[z,x] = sum_k Re(dX[k] exp(+i psi))."""
    mz2, mx = dX.shape[-2], dX.shape[-1]
    S = np.zeros(dX.shape[:-2] + (Nz, Nx), complex)
    S[..., kz_rows(Nz, mz2 // 2)[:, None], np.arange(mx)[None, :]] = dX
    return np.real(np.fft.ifft2(S, axes=(-2, -1))) * (Nz * Nx)


def idft_trunc(Y: np.ndarray, Nz: int, Nx: int) -> np.ndarray:
    """y = S Y: (1/(Nz Nx)) sum_k w_kx Re(Y[k] exp(+i psi))."""
    mz2, mx = Y.shape[-2], Y.shape[-1]
    w = np.where(np.arange(mx) == 0, 1.0, 2.0)
    S = np.zeros(Y.shape[:-2] + (Nz, Nx), complex)
    S[..., kz_rows(Nz, mz2 // 2)[:, None], np.arange(mx)[None, :]] = Y * w
    return np.real(np.fft.ifft2(S, axes=(-2, -1)))


def idft_trunc_adjoint(dy: np.ndarray, mz: int, mx: int) -> np.ndarray:
    """S' dy: dY[k] = (w_kx / (Nz Nx)) sum_{z,x} dy[z,x] exp(-i psi)."""
    Nz, Nx = dy.shape[-2], dy.shape[-1]
    w = np.where(np.arange(mx) == 0, 1.0, 2.0)
    return dft_trunc(dy, mz, mx) * w / (Nz * Nx)


# --- pointwise pieces ---------------------------------------------------------

def twiddle_tables(Nz: int, Nx: int, mz: int, mx: int):
    """The factors of the separable truncated transforms above, as complex
    arrays: fwd[x, kx] = exp(-i 2 pi kx x / Nx) (the x part of T), inv[x, kx] =
    w_kx / (Nz Nx) exp(+i 2 pi kx x / Nx) (the x part of S), bwd = conj(inv)
    (the x part of S'), adj = conj(fwd) (the x part of T'), and the z factors
    ez[z, a] = exp(+i 2 pi kz_a z / Nz) over the retained rows kz_a."""
    x = np.arange(Nx)[:, None]
    kx = np.arange(mx)[None, :]
    fwd = np.exp(-2j * np.pi * kx * x / Nx)
    w = np.where(kx == 0, 1.0, 2.0) / (Nz * Nx)
    inv = w * np.conj(fwd)
    ez = np.exp(2j * np.pi * np.arange(Nz)[:, None] * kz_rows(Nz, mz)[None, :] / Nz)
    return fwd, inv, np.conj(inv), np.conj(fwd), ez


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def pointwise(M: np.ndarray, b: np.ndarray, v: np.ndarray) -> np.ndarray:
    """out[b, o, ...] = sum_i M[o, i] v[b, i, ...] + b[o]."""
    return np.einsum("oi,bi...->bo...", M, v) + b.reshape((1, -1) + (1,) * (v.ndim - 2))


# --- parameters -----------------------------------------------------------------

def init_params(cfg: Config, seed: int) -> dict:
    """Seeded initial weights: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for the
    pointwise layers, scale * U(0,1) (real and imaginary parts) with
    scale = 1/(W W) for the spectral weights, as in Li et al. (2020)."""
    rng = np.random.default_rng(seed)
    W, H = cfg.width, cfg.hidden

    def lin(o, i):
        k = 1.0 / math.sqrt(i)
        return rng.uniform(-k, k, (o, i)), rng.uniform(-k, k, o)

    p = {}
    p["P"], p["p"] = lin(W, cfg.cin)
    for l in range(cfg.layers):
        p[f"W{l}"], p[f"b{l}"] = lin(W, W)
        s = 1.0 / (W * W)
        p[f"R{l}"] = s * (rng.uniform(0, 1, (W, W, 2 * cfg.mz, cfg.mx))
                          + 1j * rng.uniform(0, 1, (W, W, 2 * cfg.mz, cfg.mx)))
    p["Q1"], p["q1"] = lin(H, W)
    p["Q2"], p["q2"] = lin(1, H)
    return p


# --- network ------------------------------------------------------------------

def forward(p: dict, x: np.ndarray, cfg: Config):
    """x[B, Cin, Nz, Nx] -> out[B, 1, Nz, Nx] and the cache for backward."""
    Nz, Nx = x.shape[-2], x.shape[-1]
    v = pointwise(p["P"], p["p"], x)
    cache = {"x": x, "layers": []}
    for l in range(cfg.layers):
        X = dft_trunc(v, cfg.mz, cfg.mx)
        Y = np.einsum("bikx,iokx->bokx", X, p[f"R{l}"])
        u = pointwise(p[f"W{l}"], p[f"b{l}"], v) + idft_trunc(Y, Nz, Nx)
        cache["layers"].append((v, X, u))
        v = gelu(u) if l < cfg.layers - 1 else u
    hpre = pointwise(p["Q1"], p["q1"], v)
    h = gelu(hpre)
    out = pointwise(p["Q2"], p["q2"], h)
    cache.update(v=v, hpre=hpre, h=h)
    return out, cache


def _wgrad(du: np.ndarray, v: np.ndarray):
    """dM[o, i] = sum_{b, pixels} du[b, o] v[b, i]; db[o] = sum du[b, o]."""
    B = du.shape[0]
    d2, v2 = du.reshape(B, du.shape[1], -1), v.reshape(B, v.shape[1], -1)
    return np.einsum("bon,bin->oi", d2, v2), d2.sum(axis=(0, 2))


def backward(p: dict, cache: dict, dout: np.ndarray, cfg: Config) -> dict:
    """Gradients of sum(dout * out) with respect to every parameter."""
    g = {}
    x = cache["x"]
    Nz, Nx = x.shape[-2], x.shape[-1]
    g["Q2"], g["q2"] = _wgrad(dout, cache["h"])
    dh = np.einsum("oi,bo...->bi...", p["Q2"], dout)
    dhpre = dh * gelu_grad(cache["hpre"])
    g["Q1"], g["q1"] = _wgrad(dhpre, cache["v"])
    dv = np.einsum("oi,bo...->bi...", p["Q1"], dhpre)
    for l in reversed(range(cfg.layers)):
        v, X, u = cache["layers"][l]
        du = dv * gelu_grad(u) if l < cfg.layers - 1 else dv
        g[f"W{l}"], g[f"b{l}"] = _wgrad(du, v)
        dY = idft_trunc_adjoint(du, cfg.mz, cfg.mx)
        g[f"R{l}"] = np.einsum("bikx,bokx->iokx", np.conj(X), dY)
        dX = np.einsum("bokx,iokx->bikx", dY, np.conj(p[f"R{l}"]))
        dv = np.einsum("oi,bo...->bi...", p[f"W{l}"], du) + dft_trunc_adjoint(dX, Nz, Nx)
    g["P"], g["p"] = _wgrad(dv, x)
    return g


def mse(pred: np.ndarray, target: np.ndarray):
    """Loss (1/n) sum (pred - target)^2 and its gradient."""
    r = pred - target
    n = r.size
    return float(np.sum(r * r) / n), 2.0 * r / n


def adam(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, lr: float,
         b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (Kingma and Ba 2015, Algorithm 1) on flat arrays; t >= 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
