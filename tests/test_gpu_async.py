"""The modelling and gradient entry points are stream-ordered and
asynchronous: calls return before their work has run, two gradients queued on
one stream without a host synchronisation give the bits of synchronous calls,
the misfit lands in a pinned host buffer, and device-side errors (stability
limit, non-finite velocity) are reported by wave_status_wait."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2304_05592_gb300 import synth, wave
from paper_2304_05592_gb300.wave import Grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def case(seed, nt=400, nshot=3):
    p = synth.small_2d(seed, nx=150, nz=61, nt=nt, nshot=nshot, nrec=41)
    q = np.repeat(oracle.ricker(p.f0, p.dt, p.nt).astype(np.float32)[None, :, None], p.nshot, axis=0)
    og = oracle.Grid(2, p.nx, p.nz, p.h, p.dt, p.nt, p.nb, vref=p.vref)
    dobs = oracle.forward(og, p.vel, p.src, q, p.rec).astype(np.float32)
    return p, q, (p.vel * 1.03).astype(np.float32), dobs


def dptr(addr):
    return ctypes.cast(ctypes.c_void_p(addr), ctypes.POINTER(ctypes.c_double))


def raw_gradient(p, vel, q, dobs, grad, misfit_ptr, work, stream):
    """wave_gradient through the C ABI (no synchronisation anywhere)."""
    g = Grid.of(p).c()
    src = np.ascontiguousarray(p.src, np.float32)
    rec = np.ascontiguousarray(p.rec, np.float32)
    return wave._lib().wave_gradient(ctypes.byref(g), vel.data_ptr(), p.nshot, src.shape[1], src.ctypes.data,
                                     q.data_ptr(), rec.shape[1], rec.ctypes.data, dobs.data_ptr(), grad.data_ptr(),
                                     None, misfit_ptr, wave.STORE_CHECKPOINT, 16, wave.WRT_SLOWNESS2,
                                     work.data_ptr(), work.numel(), ctypes.c_void_p(stream.cuda_stream))


def test_two_gradients_queued_without_host_sync_equal_synchronous_calls():
    pa, qa, va, da = case(81)
    pb, qb, vb, db = case(82)
    ref_a = wave.wave_gradient(Grid.of(pa), dev(va), pa.src, dev(qa), pa.rec, dev(da), nsnap=16)
    ref_b = wave.wave_gradient(Grid.of(pb), dev(vb), pb.src, dev(qb), pb.rec, dev(db), nsnap=16)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        args_a = (dev(va), dev(qa), dev(da))
        args_b = (dev(vb), dev(qb), dev(db))
        wa = torch.empty(wave.wave_workspace_size(Grid.of(pa), wave.OP_GRADIENT, pa.src, pa.rec, 0, 16),
                         dtype=torch.uint8, device="cuda")
        wb = torch.empty(wave.wave_workspace_size(Grid.of(pb), wave.OP_GRADIENT, pb.src, pb.rec, 0, 16),
                         dtype=torch.uint8, device="cuda")
        ga = torch.empty(Grid.of(pa).phys_shape, device="cuda")
        gb = torch.empty(Grid.of(pb).phys_shape, device="cuda")
        phis = torch.zeros(2, dtype=torch.float64).pin_memory()
    s.synchronize()
    # a long kernel ahead of the two calls keeps the stream busy while they are queued
    spin = torch.empty(1 << 26, device="cuda")
    with torch.cuda.stream(s):
        for _ in range(200):
            spin.mul_(1.0001)
    st_a = raw_gradient(pa, args_a[0], args_a[1], args_a[2], ga, dptr(phis.data_ptr()), wa, s)
    st_b = raw_gradient(pb, args_b[0], args_b[1], args_b[2], gb, dptr(phis.data_ptr() + 8), wb, s)
    pending = not s.query()
    assert st_a == 0 and st_b == 0
    assert pending, "the calls waited for the stream"
    st, phi_b = wave.wave_status_wait(wb, s)
    assert st == 0
    st, phi_a = wave.wave_status_wait(wa, s)
    assert st == 0
    assert phi_a == ref_a[0] and phi_b == ref_b[0]
    assert phis[0].item() == ref_a[0] and phis[1].item() == ref_b[0]  # pinned host misfits
    assert torch.equal(ga, ref_a[1]) and torch.equal(gb, ref_b[1])


def test_binding_without_sync_and_status_later():
    p, q, v0, dobs = case(83, nt=300)
    g = Grid.of(p)
    work = torch.empty(wave.wave_workspace_size(g, wave.OP_GRADIENT, p.src, p.rec, 0, 8), dtype=torch.uint8,
                       device="cuda")
    phi0, g0, _ = wave.wave_gradient(g, dev(v0), p.src, dev(q), p.rec, dev(dobs), nsnap=8)
    phi, g1, _ = wave.wave_gradient(g, dev(v0), p.src, dev(q), p.rec, dev(dobs), nsnap=8, work=work, sync=False)
    assert phi is None
    st, phi1 = wave.wave_status_wait(work)
    assert st == 0 and phi1 == phi0 and torch.equal(g1, g0)


def test_device_side_errors_come_back_through_status_wait():
    p, q, v0, dobs = case(84, nt=120, nshot=1)
    g = Grid.of(p)
    work = torch.empty(wave.wave_workspace_size(g, wave.OP_FORWARD, p.src, p.rec), dtype=torch.uint8, device="cuda")
    fast = dev(p.vel * 3.0)  # above the stability limit
    wave.wave_forward(g, fast, p.src, dev(q), p.rec, work=work, sync=False)  # queued: no error yet
    assert wave.wave_status_wait(work)[0] == 2  # WAVE_ERR_CFL
    bad = p.vel.copy()
    bad[5, 7] = np.nan
    wave.wave_forward(g, dev(bad), p.src, dev(q), p.rec, work=work, sync=False)
    assert wave.wave_status_wait(work)[0] == 7  # WAVE_ERR_NONFINITE
    # the next call on the same workspace starts clean
    d = wave.wave_forward(g, dev(p.vel), p.src, dev(q), p.rec, work=work, sync=False)
    assert wave.wave_status_wait(work)[0] == 0
    assert torch.isfinite(d).all()
