"""FP64 CPU oracle for the acoustic FWI path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It shares no code with the CUDA library: the C source
``wave_oracle.c`` is compiled here with gcc and called through ctypes.

Functions follow arxiv 2304.05592, section "Wave-equation-based inversion":
``forward`` is F(m) q = P_r A(m)^{-1} P_s^T q (Eq. eq-fwi), ``gradient`` is the
misfit 1/2||F(m)q - d||^2 with its adjoint-state gradient J'(F(m)q - d) with
respect to the squared slowness m, ``adjoint`` is the pullback F' dy of the AD
rule for F*q, and ``born`` is the Jacobian J applied to dm (judiJacobian).
Shots are independent; every function loops over them.  Parity is pinned by
the tests in ``tests/test_oracle_*.py`` (analytic Green's functions,
reciprocity, energy conservation, dot tests, Taylor test, stencil exactness).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wave_oracle.c")
_OUT = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT, "liboracle.so")

OK, ERR_ARG, ERR_CFL, ERR_GEOMETRY, ERR_OOM = 0, 1, 2, 3, 4


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        names = {1: "ERR_ARG", 2: "ERR_CFL", 3: "ERR_GEOMETRY", 4: "ERR_OOM"}
        super().__init__(f"{what}: oracle status {names.get(code, code)}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP) into oracle/_build."""
    os.makedirs(_OUT, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("nb", ctypes.c_int), ("nt", ctypes.c_int),
                ("h", ctypes.c_double), ("dt", ctypes.c_double), ("vref", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(ctypes.c_double)
        G = ctypes.POINTER(_Grid)
        lib.og_forward.argtypes = [G, P, ctypes.c_int, P, P, ctypes.c_int, P, P, P]
        lib.og_adjoint.argtypes = [G, P, ctypes.c_int, P, ctypes.c_int, P, P, P, P]
        lib.og_gradient.argtypes = [G, P, ctypes.c_int, P, P, ctypes.c_int, P, P, P, P, P]
        lib.og_born.argtypes = [G, P, ctypes.c_int, P, P, ctypes.c_int, P, P, P]
        lib.og_model.argtypes = [G, P, P, P]
        lib.og_laplacian.argtypes = [G, P, P]
        lib.og_ricker.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, P]
        lib.og_ricker.restype = None
        lib.og_padded_points.argtypes = [G]
        lib.og_padded_points.restype = ctypes.c_long
        lib.og_courant_limit.argtypes = [ctypes.c_int]
        lib.og_courant_limit.restype = ctypes.c_double
        lib.og_threads.restype = ctypes.c_int
        lib.og_set_threads.argtypes = [ctypes.c_int]
        lib.og_set_threads.restype = None
        _lib = lib
    return _lib


@dataclass(frozen=True)
class Grid:
    """Physical grid (nx, [ny,] nz points at spacing h), sponge width nb, nt samples
    at step dt, sponge reference velocity vref (0: no damping)."""
    ndim: int
    nx: int
    nz: int
    h: float
    dt: float
    nt: int
    nb: int = 40
    ny: int = 1
    vref: float = 0.0

    def c(self) -> _Grid:
        return _Grid(self.ndim, self.nx, self.ny if self.ndim == 3 else 1, self.nz, self.nb,
                     self.nt, float(self.h), float(self.dt), float(self.vref))

    @property
    def phys_shape(self):
        return (self.nz, self.ny, self.nx) if self.ndim == 3 else (self.nz, self.nx)

    @property
    def pad_shape(self):
        p = 2 * self.nb
        return ((self.nz + p, self.ny + p, self.nx + p) if self.ndim == 3
                else (self.nz + p, self.nx + p))


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(code: int, what: str):
    if code != OK:
        raise OracleError(code, what)


def threads() -> int:
    return int(_load().og_threads())


def set_threads(n: int) -> None:
    """OpenMP threads of later oracle calls (timing only; results do not depend on it)."""
    _load().og_set_threads(int(n))


def courant_limit(ndim: int) -> float:
    return float(_load().og_courant_limit(ndim))


def padded_points(g: Grid) -> int:
    return int(_load().og_padded_points(ctypes.byref(g.c())))


def ricker(f: float, dt: float, nt: int) -> np.ndarray:
    """Ricker wavelet with peak frequency f delayed by 1/f, sampled at n*dt."""
    q = np.zeros(nt)
    _load().og_ricker(float(f), float(dt), int(nt), _ptr(q))
    return q


def model(g: Grid, vel) -> tuple[np.ndarray, np.ndarray]:
    """Padded squared slowness m and sponge damping eta."""
    vel = _f64(vel)
    m = np.zeros(g.pad_shape)
    eta = np.zeros(g.pad_shape)
    _check(_load().og_model(ctypes.byref(g.c()), _ptr(vel), _ptr(m), _ptr(eta)), "model")
    return m, eta


def laplacian(g: Grid, u) -> np.ndarray:
    """8th-order Laplacian of a padded field, zero values outside the padded grid."""
    u = _f64(u)
    out = np.zeros_like(u)
    _check(_load().og_laplacian(ctypes.byref(g.c()), _ptr(u), _ptr(out)), "laplacian")
    return out


def _shots(src, rec, ndim):
    src = _f64(src)
    rec = _f64(rec)
    if src.ndim == 2:
        src = src[None]
    if rec.ndim == 2:
        rec = rec[None]
    assert src.shape[-1] == ndim and rec.shape[-1] == ndim
    return src, rec


def forward(g: Grid, vel, src, wavelet, rec, fields: bool = False):
    """Shot records d[s, n, r] for sources src[s, i, :] firing wavelet[s, n, i]
    and receivers rec[s, r, :].  With fields=True also returns u[s, n, ...]."""
    src, rec = _shots(src, rec, g.ndim)
    wavelet = _f64(wavelet)
    if wavelet.ndim == 2:
        wavelet = wavelet[None]
    vel = _f64(vel)
    ns = src.shape[0]
    data = np.zeros((ns, g.nt, rec.shape[1]))
    U = np.zeros((ns, g.nt) + g.pad_shape) if fields else None
    for s in range(ns):
        d = np.zeros((g.nt, rec.shape[1]))
        w = np.ascontiguousarray(wavelet[s])
        u = np.zeros((g.nt,) + g.pad_shape) if fields else None
        _check(_load().og_forward(ctypes.byref(g.c()), _ptr(vel), src.shape[1],
                                  _ptr(np.ascontiguousarray(src[s])), _ptr(w), rec.shape[1],
                                  _ptr(np.ascontiguousarray(rec[s])), _ptr(d), _ptr(u)), "forward")
        data[s] = d
        if fields:
            U[s] = u
    return (data, U) if fields else data


def adjoint(g: Grid, vel, src, rec, resid, fields: bool = False):
    """F^T r per shot: returns src_grad[s, n, i] (and mu[s, k, ...] with fields=True)."""
    src, rec = _shots(src, rec, g.ndim)
    resid = _f64(resid)
    if resid.ndim == 2:
        resid = resid[None]
    vel = _f64(vel)
    ns = src.shape[0]
    out = np.zeros((ns, g.nt, src.shape[1]))
    MU = np.zeros((ns, g.nt) + g.pad_shape) if fields else None
    for s in range(ns):
        o = np.zeros((g.nt, src.shape[1]))
        mu = np.zeros((g.nt,) + g.pad_shape) if fields else None
        _check(_load().og_adjoint(ctypes.byref(g.c()), _ptr(vel), src.shape[1],
                                  _ptr(np.ascontiguousarray(src[s])), rec.shape[1],
                                  _ptr(np.ascontiguousarray(rec[s])),
                                  _ptr(np.ascontiguousarray(resid[s])), _ptr(o), _ptr(mu)), "adjoint")
        out[s] = o
        if fields:
            MU[s] = mu
    return (out, MU) if fields else out


def gradient(g: Grid, vel, src, wavelet, rec, dobs, per_shot: bool = False):
    """Misfit 1/2 sum ||F q - d||^2 over shots and its gradient w.r.t. the
    physical squared slowness (summed over shots, or per shot)."""
    src, rec = _shots(src, rec, g.ndim)
    wavelet = _f64(wavelet)
    if wavelet.ndim == 2:
        wavelet = wavelet[None]
    dobs = _f64(dobs)
    if dobs.ndim == 2:
        dobs = dobs[None]
    vel = _f64(vel)
    ns = src.shape[0]
    grads = np.zeros((ns,) + g.phys_shape)
    phis = np.zeros(ns)
    for s in range(ns):
        gr = np.zeros(g.phys_shape)
        phi = ctypes.c_double(0.0)
        _check(_load().og_gradient(ctypes.byref(g.c()), _ptr(vel), src.shape[1],
                                   _ptr(np.ascontiguousarray(src[s])),
                                   _ptr(np.ascontiguousarray(wavelet[s])), rec.shape[1],
                                   _ptr(np.ascontiguousarray(rec[s])),
                                   _ptr(np.ascontiguousarray(dobs[s])), _ptr(gr),
                                   ctypes.cast(ctypes.byref(phi), ctypes.POINTER(ctypes.c_double)),
                                   None), "gradient")
        grads[s] = gr
        phis[s] = phi.value
    if per_shot:
        return phis, grads
    return float(phis.sum()), grads.sum(axis=0)


def born(g: Grid, vel, src, wavelet, rec, dm):
    """Linearised data J dm per shot, dm on the physical grid."""
    src, rec = _shots(src, rec, g.ndim)
    wavelet = _f64(wavelet)
    if wavelet.ndim == 2:
        wavelet = wavelet[None]
    vel = _f64(vel)
    dm = _f64(dm)
    ns = src.shape[0]
    out = np.zeros((ns, g.nt, rec.shape[1]))
    for s in range(ns):
        o = np.zeros((g.nt, rec.shape[1]))
        _check(_load().og_born(ctypes.byref(g.c()), _ptr(vel), src.shape[1],
                               _ptr(np.ascontiguousarray(src[s])), _ptr(np.ascontiguousarray(wavelet[s])),
                               rec.shape[1], _ptr(np.ascontiguousarray(rec[s])), _ptr(dm), _ptr(o)),
               "born")
        out[s] = o
    return out
