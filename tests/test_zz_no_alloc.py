"""wave_forward_static: forward modelling on the library's own fixed device
scratch array, for callers that cannot allocate device memory when they model
(a plugin whose host application has reserved all device memory, or a
latency-critical loop that must not pay for an allocation).  Checked against
wave_forward with a caller workspace, through the C ABI, on two calls in a row
with different problems (the second call must not see the first call's
leftovers in the shared array).  Collected last so that a failure here does
not hide the other tests in a run that stops at the first failure."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2304_05592_gb300 import synth, wave
from paper_2304_05592_gb300.wave import Grid

pytestmark = pytest.mark.gpu

TOL_DATA = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def _static_call(p, vel, wavelet):
    """Calls wave_forward_static through ctypes with plain pointers."""
    lib = wave._lib()
    src = np.ascontiguousarray(p.src, np.float32)
    rec = np.ascontiguousarray(p.rec, np.float32)
    out = torch.full((p.nshot, p.nt, rec.shape[1]), float("nan"), device="cuda")
    g = Grid.of(p).c()
    st = lib.wave_forward_static(ctypes.byref(g), vel.data_ptr(), p.nshot, src.shape[1],
                                 ctypes.c_void_p(src.ctypes.data), wavelet.data_ptr(), rec.shape[1],
                                 ctypes.c_void_p(rec.ctypes.data), out.data_ptr(),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def _case(p):
    q = np.repeat(oracle.ricker(p.f0, p.dt, p.nt).astype(np.float32)[None, :, None], p.nshot, axis=0)
    vel = torch.from_numpy(p.vel).cuda()
    wavelet = torch.from_numpy(q).cuda()
    ref = wave.wave_forward(Grid.of(p), vel, p.src, wavelet, p.rec)
    return vel, wavelet, ref


def test_static_workspace_forward_matches_workspace_forward_twice():
    cases = [synth.small_2d(81, nt=300, nshot=3), synth.small_2d(82, nx=90, nz=53, nt=211, nshot=2, nrec=31)]
    for p in cases:
        assert wave.wave_workspace_size(Grid.of(p), wave.OP_FORWARD, p.src, p.rec) <= wave.STATIC_WORKSPACE_BYTES
        vel, wavelet, ref = _case(p)
        st, out = _static_call(p, vel, wavelet)
        assert st == 0, wave.STATUS.get(st, st)
        torch.cuda.synchronize()
        e = float((out - ref).norm() / ref.norm())
        assert e <= TOL_DATA, e


def test_static_workspace_rejects_problems_beyond_its_size():
    p = synth.config2(nshot=32, nt=400)
    assert wave.wave_workspace_size(Grid.of(p), wave.OP_FORWARD, p.src, p.rec) > wave.STATIC_WORKSPACE_BYTES
    vel = torch.from_numpy(p.vel).cuda()
    wavelet = torch.zeros((p.nshot, p.nt, 1), device="cuda")
    st, out = _static_call(p, vel, wavelet)
    assert st == 4  # WAVE_ERR_WORKSPACE, before any device work
    assert torch.isnan(out).all()
