"""GPU Born modelling, J' of an arbitrary residual, the velocity chain rule,
and the autograd wrapper (the AD rule of the paper: the pullback of F*q
returns J' dy and F' dy), against the FP64 oracle and finite differences."""
import numpy as np
import pytest
import torch

import oracle
from paper_2304_05592_gb300 import synth, wave
from paper_2304_05592_gb300.autograd import forward_model
from paper_2304_05592_gb300.wave import Grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def rel(a, b):
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ogrid(p):
    return oracle.Grid(p.ndim, p.nx, p.nz, p.h, p.dt, p.nt, p.nb, ny=p.ny, vref=p.vref)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def ricker_batch(p):
    q = oracle.ricker(p.f0, p.dt, p.nt).astype(np.float32)
    return np.repeat(q[None, :, None], p.nshot, axis=0)


@pytest.mark.parametrize("mk", [lambda: synth.small_2d(101, nt=250), lambda: synth.small_3d(102, nt=90)])
def test_born_matches_oracle(mk):
    p = mk()
    q = ricker_batch(p)
    rng = np.random.default_rng(4)
    m = 1.0 / p.vel.astype(np.float64) ** 2
    dm = (m * 0.05 * rng.standard_normal(m.shape)).astype(np.float32)
    d = wave.wave_born(Grid.of(p), dev(p.vel), p.src, dev(q), p.rec, dev(dm)).cpu().numpy()
    r = oracle.born(ogrid(p), p.vel, p.src, q, p.rec, dm)
    assert rel(d, r) < 2e-4, rel(d, r)


@pytest.mark.parametrize("store", [wave.STORE_CHECKPOINT, wave.STORE_BF16])
def test_jacobian_adjoint_matches_oracle_and_dot_test(store):
    p = synth.small_2d(103, nt=240)
    q = ricker_batch(p)
    g = Grid.of(p)
    rng = np.random.default_rng(6)
    r = rng.standard_normal((p.nshot, p.nt, p.rec.shape[1])).astype(np.float32)
    jt = wave.wave_jacobian_adjoint(g, dev(p.vel), p.src, dev(q), p.rec, dev(r), store=store, nsnap=5)
    d0 = oracle.forward(ogrid(p), p.vel, p.src, q, p.rec)
    _, jt_ref = oracle.gradient(ogrid(p), p.vel, p.src, q, p.rec, d0 - r)
    assert rel(jt.cpu().numpy(), jt_ref) < (1e-3 if store == wave.STORE_CHECKPOINT else 1e-2)
    if store == wave.STORE_CHECKPOINT:
        m = 1.0 / p.vel.astype(np.float64) ** 2
        dm = (m * 0.05 * rng.standard_normal(m.shape)).astype(np.float32)
        jd = wave.wave_born(g, dev(p.vel), p.src, dev(q), p.rec, dev(dm)).double()
        a = float((jd * dev(r).double()).sum())
        b = float((dev(dm).double() * jt.double()).sum())
        assert abs(a - b) <= 1e-4 * max(abs(a), abs(b)), abs(a - b) / abs(a)


def test_gradient_with_respect_to_velocity():
    p = synth.small_2d(104, nt=200)
    q = ricker_batch(p)
    g = Grid.of(p)
    dobs = synth.observed_noise((p.nshot, p.nt, p.rec.shape[1]), 1e-3, 7)
    v = dev(p.vel)
    _, gm, _ = wave.wave_gradient(g, v, p.src, dev(q), p.rec, dev(dobs), nsnap=8)
    _, gv, _ = wave.wave_gradient(g, v, p.src, dev(q), p.rec, dev(dobs), nsnap=8, wrt=wave.WRT_VELOCITY)
    expect = gm.double() * (-2.0 / v.double() ** 3)
    assert float((gv.double() - expect).norm() / expect.norm()) < 1e-6


def test_autograd_matches_library_gradient_and_finite_differences():
    p = synth.small_2d(105, nt=260)
    q = ricker_batch(p)
    g = Grid.of(p)
    dobs = dev(oracle.forward(ogrid(p), p.vel, p.src, q, p.rec))
    v0 = dev(p.vel * 1.03).requires_grad_(True)
    wav = dev(q).requires_grad_(True)

    def loss_fn(v, w):
        d = forward_model(v, w, g, p.src, p.rec, store=wave.STORE_CHECKPOINT, nsnap=7)
        return 0.5 * ((d.double() - dobs.double()) ** 2).sum()

    loss = loss_fn(v0, wav)
    loss.backward()
    _, gv_lib, _ = wave.wave_gradient(g, v0.detach(), p.src, wav.detach(), p.rec, dobs, nsnap=7,
                                      wrt=wave.WRT_VELOCITY)
    assert float((v0.grad - gv_lib).norm() / gv_lib.norm()) < 1e-5
    # finite differences of the FP32 forward model in a smooth direction
    rng = np.random.default_rng(8)
    dv = dev(rng.standard_normal(p.vel.shape) * 2.0)
    dq = dev(rng.standard_normal(q.shape) * 0.01)
    with torch.no_grad():
        for pert, grad in ((("v", dv), v0.grad), (("q", dq), wav.grad)):
            eps = 1.0
            if pert[0] == "v":
                lp, lm = loss_fn(v0 + eps * dv, wav), loss_fn(v0 - eps * dv, wav)
            else:
                lp, lm = loss_fn(v0, wav + eps * dq), loss_fn(v0, wav - eps * dq)
            fd = float(lp - lm) / (2 * eps)
            an = float((grad.double() * pert[1].double()).sum())
            assert abs(fd - an) <= 2e-3 * abs(an), (pert[0], fd, an)
