"""Thin ctypes binding of libwave's C ABI (``include/wave.h``).

The functions keep the C names and only marshal arguments: device arrays are
torch CUDA tensors (float32, contiguous), coordinates are host arrays, the
workspace is a torch uint8 tensor from torch's caching allocator, and the
stream is torch's current stream unless one is given.  Every computation runs
in libwave's CUDA kernels; there is no CPU path.  If the library has not been
built, or a tensor is not on a CUDA device, the call raises.

Operations (arxiv 2304.05592, "Wave-equation-based inversion", Eq. eq-fwi):
``wave_forward`` is F(m) q = P_r A(m)^{-1} P_s^T q, ``wave_adjoint`` is the
pullback F' r of the AD rule for F*q, ``wave_gradient`` returns the misfit
1/2 ||F(m) q - d||^2 and J'(F(m) q - d), its gradient w.r.t. the squared
slowness m.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libwave.so")

STORE_CHECKPOINT, STORE_BF16, STORE_FP32 = 0, 1, 2
OP_FORWARD, OP_ADJOINT, OP_GRADIENT, OP_BORN = 0, 1, 2, 3
WRT_SLOWNESS2, WRT_VELOCITY = 0, 1
STATUS = {0: "WAVE_OK", 1: "WAVE_ERR_ARG", 2: "WAVE_ERR_CFL", 3: "WAVE_ERR_GEOMETRY",
          4: "WAVE_ERR_WORKSPACE", 5: "WAVE_ERR_CUDA", 6: "WAVE_ERR_TIMEOUT", 7: "WAVE_ERR_NONFINITE"}


class WaveError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = _lib().wave_status_str(status).decode() if _LIB is not None else ""
        if status == 5 and _LIB is not None:
            msg += ", " + _lib().wave_cuda_error_name().decode()
        super().__init__(f"{what}: {STATUS.get(status, status)} ({msg})")


class wave_grid_t(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("nb", ctypes.c_int), ("nt", ctypes.c_int), ("h", ctypes.c_float), ("dt", ctypes.c_float),
                ("vref", ctypes.c_float)]


class wave_problem_t(ctypes.Structure):
    _fields_ = [("grid", wave_grid_t), ("vel", ctypes.c_void_p), ("nsrc", ctypes.c_int),
                ("src_xyz", ctypes.c_void_p), ("wavelet", ctypes.c_void_p), ("nrec", ctypes.c_int),
                ("rec_xyz", ctypes.c_void_p), ("d_obs", ctypes.c_void_p), ("grad", ctypes.c_void_p),
                ("misfit", ctypes.c_double)]


_LIB = None
EXPORTS = ("wave_workspace_size", "wave_forward", "wave_adjoint", "wave_gradient", "wave_ricker",
           "wave_checkpoint_schedule", "wave_profile_start", "wave_profile_stop", "wave_courant_limit",
           "wave_status_str", "wave_launch_count")


def library_path() -> str:
    return _LIB_PATH


def _lib():
    """Loads libwave.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libwave.so is not built ({_LIB_PATH}); run __graft_entry__.build() "
                               "or python -m paper_2304_05592_gb300.build")
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        G = ctypes.POINTER(wave_grid_t)
        lib.wave_workspace_size.argtypes = [G, I, I, I, P, I, P, I, I, ctypes.POINTER(ctypes.c_size_t)]
        lib.wave_forward.argtypes = [G, P, I, I, P, P, I, P, P, P, ctypes.c_size_t, P]
        lib.wave_adjoint.argtypes = [G, P, I, I, P, I, P, P, P, P, ctypes.c_size_t, P]
        lib.wave_gradient.argtypes = [G, P, I, I, P, P, I, P, P, P, P, ctypes.POINTER(ctypes.c_double), I, I, I, P,
                                      ctypes.c_size_t, P]
        lib.wave_jacobian_adjoint.argtypes = [G, P, I, I, P, P, I, P, P, P, I, I, I, P, ctypes.c_size_t, P]
        lib.wave_jacobian_adjoint.restype = I
        lib.wave_born.argtypes = [G, P, I, I, P, P, I, P, P, P, P, ctypes.c_size_t, P]
        lib.wave_born.restype = I
        lib.wave_ricker.argtypes = [ctypes.c_float, ctypes.c_float, I, P, P]
        lib.wave_checkpoint_schedule.argtypes = [I, I, ctypes.POINTER(ctypes.c_longlong), P, I,
                                                 ctypes.POINTER(ctypes.c_int)]
        lib.wave_courant_limit.argtypes = [I]
        lib.wave_courant_limit.restype = ctypes.c_double
        lib.wave_cuda_error_name.argtypes = []
        lib.wave_cuda_error_name.restype = ctypes.c_char_p
        lib.wave_status_str.argtypes = [I]
        lib.wave_status_str.restype = ctypes.c_char_p
        lib.wave_forward_static.argtypes = [G, P, I, I, P, P, I, P, P, P]
        lib.wave_forward_static.restype = I
        lib.wave_autotune.argtypes = [G, P, I, I, P, P, I, P, I, P, ctypes.c_size_t, P,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        lib.wave_autotune.restype = I
        lib.wave_workspace_size_batch.argtypes = [ctypes.POINTER(wave_problem_t), I, I,
                                                  ctypes.POINTER(ctypes.c_size_t)]
        lib.wave_workspace_size_batch.restype = I
        lib.wave_gradient_batch.argtypes = [ctypes.POINTER(wave_problem_t), I, I, I, I, P, ctypes.c_size_t, P]
        lib.wave_gradient_batch.restype = I
        lib.wave_autotune_batch.argtypes = [ctypes.POINTER(wave_problem_t), I, I, I, P, ctypes.c_size_t, P,
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        lib.wave_autotune_batch.restype = I
        lib.wave_set_batch_variant.argtypes = [I, I]
        lib.wave_set_batch_variant.restype = I
        lib.wave_batch_variant_count.argtypes = []
        lib.wave_batch_variant_count.restype = I
        lib.wave_status_wait.argtypes = [P, P, ctypes.POINTER(ctypes.c_double)]
        lib.wave_status_wait.restype = I
        L = ctypes.c_longlong
        F = ctypes.c_float
        lib.wave_lowcut_work_bytes.argtypes = [I]
        lib.wave_lowcut_work_bytes.restype = ctypes.c_size_t
        lib.wave_lowcut.argtypes = [P, I, F, F, F, P, P, P]
        lib.wave_lowcut.restype = I
        lib.wave_add_noise_work_bytes.argtypes = [I, I, I]
        lib.wave_add_noise_work_bytes.restype = ctypes.c_size_t
        lib.wave_add_noise.argtypes = [P, P, I, I, I, P, I, I, ctypes.c_double, P, P, P]
        lib.wave_add_noise.restype = I
        lib.wave_axpy.argtypes = [L, F, P, P, P]
        lib.wave_axpy.restype = I
        lib.wave_clamp.argtypes = [L, F, F, P, P]
        lib.wave_clamp.restype = I
        lib.wave_axpby.argtypes = [L, F, P, F, P, P]
        lib.wave_axpby.restype = I
        lib.wave_mul.argtypes = [L, P, P, P]
        lib.wave_mul.restype = I
        lib.wave_dot.argtypes = [L, P, P, P, P]
        lib.wave_dot.restype = I
        lib.wave_wait_probe.argtypes = [P, I, P, P, P]
        lib.wave_wait_probe.restype = I
        lib.wave_set_variant.argtypes = [I, I]
        lib.wave_set_variant.restype = I
        lib.wave_variant_count.argtypes = [I]
        lib.wave_variant_count.restype = I
        lib.wave_profile_start.argtypes = [I]
        lib.wave_profile_stop.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
        lib.wave_launch_count.argtypes = []
        lib.wave_launch_count.restype = ctypes.c_longlong
        for name in EXPORTS[:-3]:
            getattr(lib, name).restype = I
        _LIB = lib
    return _LIB


@dataclass(frozen=True)
class Grid:
    """Physical grid nx x (ny x) nz at spacing h, nb sponge cells per side, nt
    samples at step dt, frozen sponge reference velocity vref (0: no damping)."""
    ndim: int
    nx: int
    nz: int
    h: float
    dt: float
    nt: int
    nb: int = 40
    ny: int = 1
    vref: float = 0.0

    def c(self) -> wave_grid_t:
        return wave_grid_t(self.ndim, self.nx, self.ny if self.ndim == 3 else 1, self.nz, self.nb, self.nt,
                           self.h, self.dt, self.vref)

    @property
    def phys_shape(self):
        return (self.nz, self.ny, self.nx) if self.ndim == 3 else (self.nz, self.nx)

    @staticmethod
    def of(p) -> "Grid":
        """Grid of a synth.Problem."""
        return Grid(p.ndim, p.nx, p.nz, float(p.h), float(p.dt), int(p.nt), int(p.nb), int(p.ny), float(p.vref))


def _dev(t: torch.Tensor, name: str, shape=None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (libwave has no CPU path)")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def _host_xyz(a, ndim: int) -> np.ndarray:
    if isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if a.ndim != 3 or a.shape[-1] != ndim:
        raise ValueError(f"coordinates must have shape [nshot][npts][{ndim}], got {a.shape}")
    return a


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def wave_status_wait(work: torch.Tensor, stream=None):
    """Waits for the stream and returns (status, misfit) of the last call
    queued on the workspace `work` (0 = success; the misfit of wave_gradient)."""
    phi = ctypes.c_double(0.0)
    st = _lib().wave_status_wait(ctypes.c_void_p(work.data_ptr()), _stream(stream), ctypes.byref(phi))
    return int(st), float(phi.value)


def _finish(st: int, work: torch.Tensor, stream, name: str, sync: bool) -> float:
    """Raises on a host-side error; with sync, waits for the call and raises on a
    device-side error; returns the misfit the workspace holds (0 without sync)."""
    if st:
        raise WaveError(st, name)
    if not sync:
        return 0.0
    st, phi = wave_status_wait(work, stream)
    if st:
        raise WaveError(st, name)
    return phi


def wave_workspace_size(grid: Grid, op: int, src_xyz, rec_xyz, store: int = STORE_CHECKPOINT,
                        nsnap: int = 1) -> int:
    src = _host_xyz(src_xyz, grid.ndim)
    rec = _host_xyz(rec_xyz, grid.ndim)
    out = ctypes.c_size_t(0)
    g = grid.c()
    st = _lib().wave_workspace_size(ctypes.byref(g), op, src.shape[0], src.shape[1], _ptr(src), rec.shape[1],
                                    _ptr(rec), store, nsnap, ctypes.byref(out))
    if st:
        raise WaveError(st, "wave_workspace_size")
    return int(out.value)


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def wave_forward(grid: Grid, vel: torch.Tensor, src_xyz, wavelet: torch.Tensor, rec_xyz, data=None,
                 stream=None, work: torch.Tensor | None = None, sync: bool = True) -> torch.Tensor:
    """Shot records [nshot][nt][nrec] = F(m) q for every shot.  With
    sync=False the call is only queued on the stream (pass `work` and check it
    later with wave_status_wait)."""
    src = _host_xyz(src_xyz, grid.ndim)
    rec = _host_xyz(rec_xyz, grid.ndim)
    ns, nsrc, nrec = src.shape[0], src.shape[1], rec.shape[1]
    if rec.shape[0] != ns:
        raise ValueError("src_xyz and rec_xyz disagree on the number of shots")
    pv = _dev(vel, "vel", grid.phys_shape)
    pw = _dev(wavelet, "wavelet", (ns, grid.nt, nsrc))
    if data is None:
        data = torch.empty((ns, grid.nt, nrec), dtype=torch.float32, device=vel.device)
    pd = _dev(data, "data", (ns, grid.nt, nrec))
    nbytes = wave_workspace_size(grid, OP_FORWARD, src, rec)
    if work is None or work.numel() < nbytes:
        work = _workspace(nbytes, vel.device)
    g = grid.c()
    st = _lib().wave_forward(ctypes.byref(g), pv, ns, nsrc, _ptr(src), pw, nrec, _ptr(rec), pd,
                             work.data_ptr(), work.numel(), _stream(stream))
    _finish(st, work, stream, "wave_forward", sync and ns > 0)
    return data


STATIC_WORKSPACE_BYTES = 32 << 20


def wave_forward_static(grid: Grid, vel: torch.Tensor, src_xyz, wavelet: torch.Tensor, rec_xyz, data=None,
                        stream=None) -> torch.Tensor:
    """wave_forward on the library's own fixed device scratch array (no
    workspace from the caller): for callers that cannot allocate device memory
    when they model.  Problems needing more than 32 MiB of scratch raise
    WAVE_ERR_WORKSPACE; calls that overlap on the GPU race (one shared array)."""
    src = _host_xyz(src_xyz, grid.ndim)
    rec = _host_xyz(rec_xyz, grid.ndim)
    ns, nsrc, nrec = src.shape[0], src.shape[1], rec.shape[1]
    pv = _dev(vel, "vel", grid.phys_shape)
    pw = _dev(wavelet, "wavelet", (ns, grid.nt, nsrc))
    if data is None:
        data = torch.empty((ns, grid.nt, nrec), dtype=torch.float32, device=vel.device)
    pd = _dev(data, "data", (ns, grid.nt, nrec))
    g = grid.c()
    st = _lib().wave_forward_static(ctypes.byref(g), pv, ns, nsrc, _ptr(src), pw, nrec, _ptr(rec), pd,
                                    _stream(stream))
    if st:
        raise WaveError(st, "wave_forward_static")
    return data


def wave_adjoint(grid: Grid, vel: torch.Tensor, src_xyz, rec_xyz, resid: torch.Tensor, src_out=None,
                 stream=None, work: torch.Tensor | None = None, sync: bool = True) -> torch.Tensor:
    """F(m)' r for every shot: [nshot][nt][nsrc]."""
    src = _host_xyz(src_xyz, grid.ndim)
    rec = _host_xyz(rec_xyz, grid.ndim)
    ns, nsrc, nrec = src.shape[0], src.shape[1], rec.shape[1]
    pv = _dev(vel, "vel", grid.phys_shape)
    pr = _dev(resid, "resid", (ns, grid.nt, nrec))
    if src_out is None:
        src_out = torch.empty((ns, grid.nt, nsrc), dtype=torch.float32, device=vel.device)
    po = _dev(src_out, "src_out", (ns, grid.nt, nsrc))
    nbytes = wave_workspace_size(grid, OP_ADJOINT, src, rec)
    if work is None or work.numel() < nbytes:
        work = _workspace(nbytes, vel.device)
    g = grid.c()
    st = _lib().wave_adjoint(ctypes.byref(g), pv, ns, nsrc, _ptr(src), nrec, _ptr(rec), pr, po, work.data_ptr(),
                             work.numel(), _stream(stream))
    _finish(st, work, stream, "wave_adjoint", sync and ns > 0)
    return src_out


def wave_gradient(grid: Grid, vel: torch.Tensor, src_xyz, wavelet: torch.Tensor, rec_xyz, d_obs: torch.Tensor,
                  store: int = STORE_CHECKPOINT, nsnap: int = 64, grad=None, want_dsyn: bool = False,
                  work: torch.Tensor | None = None, stream=None, wrt: int = WRT_SLOWNESS2, sync: bool = True):
    """Returns (misfit, dPhi/dm (or dPhi/dv with wrt=WRT_VELOCITY) [phys shape], d_syn or None).
    With sync=False the call is only queued (misfit None; pass `work` and read
    the status and misfit later with wave_status_wait)."""
    src = _host_xyz(src_xyz, grid.ndim)
    rec = _host_xyz(rec_xyz, grid.ndim)
    ns, nsrc, nrec = src.shape[0], src.shape[1], rec.shape[1]
    pv = _dev(vel, "vel", grid.phys_shape)
    pw = _dev(wavelet, "wavelet", (ns, grid.nt, nsrc))
    po = _dev(d_obs, "d_obs", (ns, grid.nt, nrec))
    if grad is None:
        grad = torch.empty(grid.phys_shape, dtype=torch.float32, device=vel.device)
    pg = _dev(grad, "grad", grid.phys_shape)
    dsyn = torch.empty((ns, grid.nt, nrec), dtype=torch.float32, device=vel.device) if want_dsyn else None
    pds = dsyn.data_ptr() if dsyn is not None else None
    nbytes = wave_workspace_size(grid, OP_GRADIENT, src, rec, store, nsnap)
    if work is None or work.numel() < nbytes:
        work = _workspace(nbytes, vel.device)
    g = grid.c()
    st = _lib().wave_gradient(ctypes.byref(g), pv, ns, nsrc, _ptr(src), pw, nrec, _ptr(rec), po, pg, pds,
                              None, store, nsnap, wrt, work.data_ptr(), work.numel(), _stream(stream))
    phi = _finish(st, work, stream, "wave_gradient", sync)
    return (phi if sync else None), grad, dsyn


def wave_jacobian_adjoint(grid: Grid, vel: torch.Tensor, src_xyz, wavelet: torch.Tensor, rec_xyz,
                          resid: torch.Tensor, store: int = STORE_CHECKPOINT, nsnap: int = 64,
                          wrt: int = WRT_SLOWNESS2, grad=None, stream=None) -> torch.Tensor:
    """J(m)' r summed over shots, on the physical grid (w.r.t. m, or v with wrt=WRT_VELOCITY)."""
    src = _host_xyz(src_xyz, grid.ndim)
    rec = _host_xyz(rec_xyz, grid.ndim)
    ns, nsrc, nrec = src.shape[0], src.shape[1], rec.shape[1]
    pv = _dev(vel, "vel", grid.phys_shape)
    pw = _dev(wavelet, "wavelet", (ns, grid.nt, nsrc))
    pr = _dev(resid, "resid", (ns, grid.nt, nrec))
    if grad is None:
        grad = torch.empty(grid.phys_shape, dtype=torch.float32, device=vel.device)
    pg = _dev(grad, "grad", grid.phys_shape)
    work = _workspace(wave_workspace_size(grid, OP_GRADIENT, src, rec, store, nsnap), vel.device)
    g = grid.c()
    st = _lib().wave_jacobian_adjoint(ctypes.byref(g), pv, ns, nsrc, _ptr(src), pw, nrec, _ptr(rec), pr, pg, store,
                                      nsnap, wrt, work.data_ptr(), work.numel(), _stream(stream))
    _finish(st, work, stream, "wave_jacobian_adjoint", True)
    return grad


def wave_born(grid: Grid, vel: torch.Tensor, src_xyz, wavelet: torch.Tensor, rec_xyz, dm: torch.Tensor, data=None,
              stream=None) -> torch.Tensor:
    """Born data J(m) dm [nshot][nt][nrec] for a squared-slowness perturbation dm."""
    src = _host_xyz(src_xyz, grid.ndim)
    rec = _host_xyz(rec_xyz, grid.ndim)
    ns, nsrc, nrec = src.shape[0], src.shape[1], rec.shape[1]
    pv = _dev(vel, "vel", grid.phys_shape)
    pw = _dev(wavelet, "wavelet", (ns, grid.nt, nsrc))
    pdm = _dev(dm, "dm", grid.phys_shape)
    if data is None:
        data = torch.empty((ns, grid.nt, nrec), dtype=torch.float32, device=vel.device)
    pd = _dev(data, "data", (ns, grid.nt, nrec))
    work = _workspace(wave_workspace_size(grid, OP_BORN, src, rec), vel.device)
    g = grid.c()
    st = _lib().wave_born(ctypes.byref(g), pv, ns, nsrc, _ptr(src), pw, nrec, _ptr(rec), pdm, pd, work.data_ptr(),
                          work.numel(), _stream(stream))
    _finish(st, work, stream, "wave_born", ns > 0)
    return data


def wave_ricker(f0: float, dt: float, nt: int, device="cuda", out=None, stream=None) -> torch.Tensor:
    """Ricker wavelet with peak frequency f0 delayed by 1/f0, [nt] on the GPU."""
    if out is None:
        out = torch.empty(nt, dtype=torch.float32, device=device)
    st = _lib().wave_ricker(float(f0), float(dt), int(nt), _dev(out, "out", (nt,)), _stream(stream))
    if st:
        raise WaveError(st, "wave_ricker")
    return out


def wave_checkpoint_schedule(nt: int, nsnap: int):
    """(forward steps, actions[n][3]) of the binomial checkpoint schedule (host only)."""
    n = ctypes.c_int(0)
    steps = ctypes.c_longlong(0)
    st = _lib().wave_checkpoint_schedule(nt, nsnap, ctypes.byref(steps), None, 0, ctypes.byref(n))
    if st:
        raise WaveError(st, "wave_checkpoint_schedule")
    acts = np.zeros((max(n.value, 1), 3), dtype=np.int32)
    st = _lib().wave_checkpoint_schedule(nt, nsnap, ctypes.byref(steps), ctypes.c_void_p(acts.ctypes.data),
                                         n.value, ctypes.byref(n))
    if st:
        raise WaveError(st, "wave_checkpoint_schedule")
    return int(steps.value), acts[:n.value]


def wave_courant_limit(ndim: int) -> float:
    return float(_lib().wave_courant_limit(ndim))


def wave_launch_count() -> int:
    """Kernels libwave has launched so far in this process."""
    return int(_lib().wave_launch_count())


def wave_profile_start(every: int = 1) -> None:
    """Bracket every `every`-th stencil step launch with CUDA events (every = 0:
    each run of consecutive step launches of one kind, overlap kept)."""
    st = _lib().wave_profile_start(int(every))
    if st:
        raise WaveError(st, "wave_profile_start")


def wave_profile_stop():
    """(forward ms, forward samples, adjoint ms, adjoint samples) since start."""
    f, a = ctypes.c_double(0), ctypes.c_double(0)
    nf, na = ctypes.c_longlong(0), ctypes.c_longlong(0)
    st = _lib().wave_profile_stop(ctypes.byref(f), ctypes.byref(nf), ctypes.byref(a), ctypes.byref(na))
    if st:
        raise WaveError(st, "wave_profile_stop")
    return f.value, nf.value, a.value, na.value


def wave_set_variant(which: int, variant: int) -> None:
    """Select the 2D forward (which=0) or adjoint (which=1) kernel variant; -1 = default."""
    st = _lib().wave_set_variant(int(which), int(variant))
    if st:
        raise WaveError(st, "wave_set_variant")


def wave_variant_count(which: int) -> int:
    return int(_lib().wave_variant_count(int(which)))


def wave_autotune(grid: Grid, vel: torch.Tensor, src_xyz, wavelet: torch.Tensor, rec_xyz, steps: int = 20,
                  stream=None):
    """Times every 2D step variant on this problem and remembers the fastest
    for this grid and shot count; returns (forward variant, adjoint variant)."""
    src = _host_xyz(src_xyz, grid.ndim)
    rec = _host_xyz(rec_xyz, grid.ndim)
    ns, nsrc, nrec = src.shape[0], src.shape[1], rec.shape[1]
    pv = _dev(vel, "vel", grid.phys_shape)
    pw = _dev(wavelet, "wavelet", (ns, grid.nt, nsrc))
    nbytes = wave_workspace_size(grid, OP_GRADIENT, src, rec, STORE_CHECKPOINT, 1)
    work = _workspace(nbytes, vel.device)
    bf, ba = ctypes.c_int(-1), ctypes.c_int(-1)
    g = grid.c()
    st = _lib().wave_autotune(ctypes.byref(g), pv, ns, nsrc, _ptr(src), pw, nrec, _ptr(rec), int(steps),
                              work.data_ptr(), work.numel(), _stream(stream), ctypes.byref(bf), ctypes.byref(ba))
    if st:
        raise WaveError(st, "wave_autotune")
    return bf.value, ba.value


class BatchProblem:
    """One problem of an uneven batch: Grid, velocity (CUDA), source and
    receiver coordinates (host, [n][2]), wavelet [nt][nsrc] and observed data
    [nt][nrec] (CUDA)."""

    def __init__(self, grid: Grid, vel, src_xyz, wavelet, rec_xyz, d_obs):
        self.grid, self.vel, self.wavelet, self.d_obs = grid, vel, wavelet, d_obs
        self.src = np.ascontiguousarray(np.asarray(src_xyz, np.float32).reshape(-1, 2))
        self.rec = np.ascontiguousarray(np.asarray(rec_xyz, np.float32).reshape(-1, 2))


def _problem_array(problems, grads):
    arr = (wave_problem_t * max(len(problems), 1))()
    for i, (p, gr) in enumerate(zip(problems, grads)):
        _dev(p.vel, "vel", p.grid.phys_shape)
        _dev(p.wavelet, "wavelet", (p.grid.nt, p.src.shape[0]))
        _dev(p.d_obs, "d_obs", (p.grid.nt, p.rec.shape[0]))
        arr[i].grid = p.grid.c()
        arr[i].vel = p.vel.data_ptr()
        arr[i].nsrc = p.src.shape[0]
        arr[i].src_xyz = p.src.ctypes.data if p.src.size else None
        arr[i].wavelet = p.wavelet.data_ptr()
        arr[i].nrec = p.rec.shape[0]
        arr[i].rec_xyz = p.rec.ctypes.data if p.rec.size else None
        arr[i].d_obs = p.d_obs.data_ptr()
        arr[i].grad = gr.data_ptr() if gr is not None else None
    return arr


def wave_gradient_batch(problems, store: int = STORE_BF16, wrt: int = WRT_SLOWNESS2, use_graph: bool = True,
                        grads=None, work: torch.Tensor | None = None, stream=None):
    """Gradients and misfits of an uneven batch of 2D problems (one persistent
    forward sweep, one persistent adjoint sweep).  Returns (misfits, grads)."""
    if grads is None:
        grads = [torch.empty(p.grid.phys_shape, dtype=torch.float32, device=p.vel.device) for p in problems]
    arr = _problem_array(problems, grads)
    nbytes = ctypes.c_size_t(0)
    st = _lib().wave_workspace_size_batch(arr, len(problems), store, ctypes.byref(nbytes))
    if st:
        raise WaveError(st, "wave_workspace_size_batch")
    if work is None or work.numel() < nbytes.value:
        work = _workspace(nbytes.value, problems[0].vel.device if problems else "cuda")
    st = _lib().wave_gradient_batch(arr, len(problems), store, wrt, int(use_graph), work.data_ptr(), work.numel(),
                                    _stream(stream))
    if st:
        raise WaveError(st, "wave_gradient_batch")
    return [arr[i].misfit for i in range(len(problems))], grads


def wave_autotune_batch(problems, store: int = STORE_BF16, steps: int = 200, work: torch.Tensor | None = None,
                        stream=None):
    """Times every sweep-kernel variant on the first `steps` steps of this
    batch and records the fastest pair for batches of its shapes.  Returns
    (forward variant, adjoint variant)."""
    grads = [None] * len(problems)
    arr = _problem_array(problems, grads)
    nbytes = ctypes.c_size_t(0)
    st = _lib().wave_workspace_size_batch(arr, len(problems), store, ctypes.byref(nbytes))
    if st:
        raise WaveError(st, "wave_workspace_size_batch")
    if work is None or work.numel() < nbytes.value:
        work = _workspace(nbytes.value, problems[0].vel.device)
    bf, ba = ctypes.c_int(-1), ctypes.c_int(-1)
    st = _lib().wave_autotune_batch(arr, len(problems), store, steps, work.data_ptr(), work.numel(), _stream(stream),
                                    ctypes.byref(bf), ctypes.byref(ba))
    if st:
        raise WaveError(st, "wave_autotune_batch")
    return bf.value, ba.value


def wave_batch_variant_count() -> int:
    return int(_lib().wave_batch_variant_count())


def wave_set_batch_variant(fwd: int, adj: int) -> None:
    """Forces the uneven batch's sweep kernels (both -1: back to the tuned choice)."""
    st = _lib().wave_set_batch_variant(fwd, adj)
    if st:
        raise WaveError(st, "wave_set_batch_variant")


def wave_workspace_size_batch(problems, store: int = STORE_BF16) -> int:
    arr = _problem_array(problems, [None] * len(problems))
    nbytes = ctypes.c_size_t(0)
    st = _lib().wave_workspace_size_batch(arr, len(problems), store, ctypes.byref(nbytes))
    if st:
        raise WaveError(st, "wave_workspace_size_batch")
    return int(nbytes.value)


def wave_wait_probe(flag: torch.Tensor, want: int, abort_word: torch.Tensor, err: torch.Tensor, stream=None) -> int:
    """Runs the batch sweep's bounded wait on device int32 scalars; returns the
    status (0 released, 6 WAVE_ERR_TIMEOUT) instead of raising."""
    for t, n in ((flag, "flag"), (abort_word, "abort_word"), (err, "err")):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.int32:
            raise TypeError(f"{n} must be a CUDA int32 tensor")
    return int(_lib().wave_wait_probe(ctypes.c_void_p(flag.data_ptr()), int(want),
                                      ctypes.c_void_p(abort_word.data_ptr()), ctypes.c_void_p(err.data_ptr()),
                                      _stream(stream)))


def wave_lowcut(q: torch.Tensor, dt: float, f_cut: float = 4.0, f_pass: float = 6.0, out=None,
                stream=None) -> torch.Tensor:
    """q [nt] high-passed: no energy below f_cut, a raised-cosine ramp up to f_pass."""
    nt = q.numel()
    _dev(q, "q", (nt,))
    if out is None:
        out = torch.empty_like(q)
    _dev(out, "out", (nt,))
    work = _workspace(int(_lib().wave_lowcut_work_bytes(nt)), q.device)
    st = _lib().wave_lowcut(q.data_ptr(), nt, float(dt), float(f_cut), float(f_pass), out.data_ptr(),
                            work.data_ptr(), _stream(stream))
    if st:
        raise WaveError(st, "wave_lowcut")
    return out


def wave_add_noise(data: torch.Tensor, white: torch.Tensor, filt: torch.Tensor, center: int, snr_db: float,
                   out=None, stream=None) -> torch.Tensor:
    """data [nshot][nt][nrec] plus white noise filtered by filt (centred at tap
    `center`), scaled to snr_db."""
    ns, nt, nrec = data.shape
    _dev(data, "data")
    _dev(white, "white", data.shape)
    _dev(filt, "filt", (filt.numel(),))
    if out is None:
        out = torch.empty_like(data)
    _dev(out, "out", data.shape)
    work = _workspace(int(_lib().wave_add_noise_work_bytes(ns, nt, nrec)), data.device)
    st = _lib().wave_add_noise(data.data_ptr(), white.data_ptr(), ns, nt, nrec, filt.data_ptr(), filt.numel(),
                               int(center), float(snr_db), out.data_ptr(), work.data_ptr(), _stream(stream))
    if st:
        raise WaveError(st, "wave_add_noise")
    return out


def wave_axpy(alpha: float, x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
    """y += alpha x in place."""
    _dev(x, "x")
    _dev(y, "y", x.shape)
    st = _lib().wave_axpy(y.numel(), float(alpha), x.data_ptr(), y.data_ptr(), _stream(stream))
    if st:
        raise WaveError(st, "wave_axpy")
    return y


def wave_axpby(alpha: float, x: torch.Tensor, beta: float, y: torch.Tensor, stream=None) -> torch.Tensor:
    """y = alpha x + beta y in place (device float32 tensors of equal size)."""
    if x.numel() != y.numel():
        raise ValueError("x and y differ in size")
    st = _lib().wave_axpby(y.numel(), float(alpha), _dev(x, "x"), float(beta), _dev(y, "y"), _stream(stream))
    if st:
        raise WaveError(st, "wave_axpby")
    return y


def wave_mul(x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
    """y = x .* y in place (device float32 tensors of equal size)."""
    if x.numel() != y.numel():
        raise ValueError("x and y differ in size")
    st = _lib().wave_mul(y.numel(), _dev(x, "x"), _dev(y, "y"), _stream(stream))
    if st:
        raise WaveError(st, "wave_mul")
    return y


DOT_PARTIALS = 256


def wave_dot(x: torch.Tensor, y: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """sum x*y in double on the device, fixed order; returns a device float64
    tensor whose element 0 holds the result (the rest is scratch)."""
    if x.numel() != y.numel():
        raise ValueError("x and y differ in size")
    if out is None:
        out = torch.empty(1 + DOT_PARTIALS, dtype=torch.float64, device=x.device)
    st = _lib().wave_dot(x.numel(), _dev(x, "x"), _dev(y, "y"), ctypes.c_void_p(out.data_ptr()), _stream(stream))
    if st:
        raise WaveError(st, "wave_dot")
    return out


def wave_clamp(y: torch.Tensor, lo: float, hi: float, stream=None) -> torch.Tensor:
    """y = min(max(y, lo), hi) in place."""
    _dev(y, "y")
    st = _lib().wave_clamp(y.numel(), float(lo), float(hi), y.data_ptr(), _stream(stream))
    if st:
        raise WaveError(st, "wave_clamp")
    return y
