"""Pins of the oracle's linear algebra: adjoint dot tests for F (in q) and J
(in m), the Taylor test of the misfit gradient, Born modelling against
finite differences, and input validation."""
import numpy as np
import pytest

import oracle
from paper_2304_05592_gb300 import synth


def _grid(p):
    return oracle.Grid(p.ndim, p.nx, p.nz, p.h, float(p.dt), p.nt, p.nb, ny=p.ny, vref=p.vref)


@pytest.mark.parametrize("mk", [lambda: synth.small_2d(3, nt=220), lambda: synth.small_3d(4, nt=70)])
def test_dot_test_F(mk):
    p = mk()
    g = _grid(p)
    rng = np.random.default_rng(7)
    ns, nsrc, nrec = p.nshot, p.src.shape[1], p.rec.shape[1]
    # two sources per shot to exercise summation of injection
    src = np.concatenate([p.src, p.src[:, :, :] * 0.9 + 1.0], axis=1)
    nsrc = src.shape[1]
    q = rng.standard_normal((ns, p.nt, nsrc))
    r = rng.standard_normal((ns, p.nt, nrec))
    Fq = oracle.forward(g, p.vel, src, q, p.rec)
    Ftr = oracle.adjoint(g, p.vel, src, p.rec, r)
    a = np.vdot(Fq, r)
    b = np.vdot(q, Ftr)
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))


def _fwd_gen(p, seed=3):
    g = _grid(p)
    q = np.repeat(oracle.ricker(p.f0, p.dt, p.nt)[None, :, None], p.nshot, axis=0)
    return g, q


def test_dot_test_J():
    p = synth.small_2d(5, nt=200)
    g, q = _fwd_gen(p)
    rng = np.random.default_rng(9)
    dm = rng.standard_normal(p.vel.shape) * 1e-8
    r = rng.standard_normal((p.nshot, p.nt, p.rec.shape[1]))
    Jdm = oracle.born(g, p.vel, p.src, q, p.rec, dm)
    d0 = oracle.forward(g, p.vel, p.src, q, p.rec)
    _, JTr = oracle.gradient(g, p.vel, p.src, q, p.rec, d0 - r)
    a = np.vdot(Jdm, r)
    b = np.vdot(dm, JTr)
    assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))


def test_dot_test_J_3d():
    p = synth.small_3d(6, nt=60)
    g, q = _fwd_gen(p)
    rng = np.random.default_rng(10)
    dm = rng.standard_normal(p.vel.shape) * 1e-8
    r = rng.standard_normal((p.nshot, p.nt, p.rec.shape[1]))
    Jdm = oracle.born(g, p.vel, p.src, q, p.rec, dm)
    d0 = oracle.forward(g, p.vel, p.src, q, p.rec)
    _, JTr = oracle.gradient(g, p.vel, p.src, q, p.rec, d0 - r)
    a = np.vdot(Jdm, r)
    b = np.vdot(dm, JTr)
    assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))


def _phi(g, vel, p, q, dobs):
    d = oracle.forward(g, vel, p.src, q, p.rec)
    return 0.5 * np.sum((d - dobs) ** 2)


def test_taylor_gradient_first_and_second_order():
    p = synth.small_2d(8, nt=260)
    g, q = _fwd_gen(p)
    v_true = p.vel.astype(np.float64)
    m0 = 1.0 / (v_true * 1.04) ** 2  # smooth-ish starting model: 4 % slower
    dobs = oracle.forward(g, v_true, p.src, q, p.rec)
    phi0, grad = oracle.gradient(g, 1.0 / np.sqrt(m0), p.src, q, p.rec, dobs)
    rng = np.random.default_rng(11)
    dm = m0 * 0.02 * rng.standard_normal(m0.shape)
    e1, e2 = [], []
    eps = [2.0 ** -k for k in range(0, 5)]
    gd = np.vdot(grad, dm)
    for e in eps:
        phi = _phi(g, 1.0 / np.sqrt(m0 + e * dm), p, q, dobs)
        e1.append(abs(phi - phi0))
        e2.append(abs(phi - phi0 - e * gd))
    r1 = np.array(e1[:-1]) / np.array(e1[1:])
    r2 = np.array(e2[:-1]) / np.array(e2[1:])
    assert np.all(np.abs(r1[1:] - 2.0) < 0.25), r1
    assert np.all(np.abs(r2[1:] - 4.0) < 0.5), r2


def test_born_matches_central_differences():
    p = synth.small_2d(12, nt=200, nshot=1)
    g, q = _fwd_gen(p)
    m0 = 1.0 / p.vel.astype(np.float64) ** 2
    rng = np.random.default_rng(13)
    dm = m0 * 0.05 * rng.standard_normal(m0.shape)
    J = oracle.born(g, p.vel.astype(np.float64), p.src, q, p.rec, dm)
    errs = []
    for e in (1e-2, 5e-3):
        dp = oracle.forward(g, 1.0 / np.sqrt(m0 + e * dm), p.src, q, p.rec)
        dn = oracle.forward(g, 1.0 / np.sqrt(m0 - e * dm), p.src, q, p.rec)
        fd = (dp - dn) / (2 * e)
        errs.append(np.linalg.norm(fd - J) / np.linalg.norm(J))
    assert errs[1] < 1e-4
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_gradient_sums_over_shots():
    p = synth.small_2d(14, nt=120, nshot=3)
    g, q = _fwd_gen(p)
    dobs = synth.observed_noise((p.nshot, p.nt, p.rec.shape[1]), 1e-3, 15)
    phis, gs = oracle.gradient(g, p.vel, p.src, q, p.rec, dobs, per_shot=True)
    phi, gsum = oracle.gradient(g, p.vel, p.src, q, p.rec, dobs)
    assert abs(phi - phis.sum()) <= 1e-12 * phi
    assert np.allclose(gsum, gs.sum(0), rtol=0, atol=1e-12 * np.abs(gsum).max())


def test_rejects_points_outside_physical_grid():
    p = synth.small_2d(1, nt=20, nshot=1)
    g, q = _fwd_gen(p)
    rec = p.rec.copy().astype(np.float64)
    rec[0, 0, 0] = (p.nx - 1) * p.h + 1e-3
    with pytest.raises(oracle.OracleError) as e:
        oracle.forward(g, p.vel, p.src, q, rec)
    assert e.value.code == oracle.ERR_GEOMETRY
    rec[0, 0, 0] = (p.nx - 1) * p.h  # the last grid point is inside
    oracle.forward(g, p.vel, p.src, q, rec)
    rec[0, 0, 0] = -1e-3
    with pytest.raises(oracle.OracleError):
        oracle.forward(g, p.vel, p.src, q, rec)


def test_rejects_bad_velocity():
    p = synth.small_2d(1, nt=20, nshot=1)
    g, q = _fwd_gen(p)
    vel = p.vel.astype(np.float64).copy()
    vel[3, 3] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.forward(g, vel, p.src, q, p.rec)
    assert e.value.code == oracle.ERR_ARG
