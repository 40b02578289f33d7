"""Least-squares RTM on the GPU (CGLS with wave_born and
wave_jacobian_adjoint) against the FP64 oracle's CGLS on the same data,
iterate by iterate, and its convergence on a small survey with a known
perturbation; the vector kernels it uses (dot, axpby) against plain sums."""
import numpy as np
import pytest
import torch

import oracle
from oracle import lsrtm as olsrtm
from paper_2304_05592_gb300 import lsrtm, synth, wave
from paper_2304_05592_gb300.wave import Grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_dot_and_axpby_match_plain_sums():
    rng = np.random.default_rng(8)
    for n in (0, 1, 1000, 300001):
        x, y = rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32)
        d = float(wave.wave_dot(dev(x), dev(y))[0].item())
        ref = float(np.dot(x.astype(np.float64), y.astype(np.float64)))
        assert abs(d - ref) <= 1e-12 * max(1.0, np.sum(np.abs(x.astype(np.float64) * y)))
        yd = dev(y)
        wave.wave_axpby(0.5, dev(x), -2.0, yd)
        np.testing.assert_allclose(yd.cpu().numpy(), 0.5 * x.astype(np.float64) - 2.0 * y, rtol=1e-6, atol=1e-6)
    a = dev(rng.standard_normal(5000))
    assert torch.equal(wave.wave_dot(a, a)[:1], wave.wave_dot(a, a)[:1])  # fixed summation order


@pytest.fixture(scope="module")
def survey():
    # 4 shots, 60 receivers around a 60 x 40 grid, two Gaussian blobs of squared slowness
    p = synth.small_2d(5, nx=60, nz=40, nt=400, nshot=4, nrec=60)
    g = oracle.Grid(2, p.nx, p.nz, p.h, p.dt, p.nt, p.nb, vref=p.vref)
    q = np.repeat(oracle.ricker(p.f0, p.dt, p.nt).astype(np.float32)[None, :, None], p.nshot, axis=0)
    zz, xx = np.meshgrid(np.arange(p.nz), np.arange(p.nx), indexing="ij")
    m0 = 1.0 / p.vel.astype(np.float64) ** 2
    dm = 0.05 * m0 * (np.exp(-((zz - 20) ** 2 + (xx - 25) ** 2) / 18.0)
                      - 0.7 * np.exp(-((zz - 28) ** 2 + (xx - 40) ** 2) / 12.0))
    dd = oracle.born(g, p.vel, p.src, q, p.rec, dm).astype(np.float32)
    x_ref, xs_ref, rn_ref = olsrtm.lsrtm(g, p.vel, p.src, q.astype(np.float64), p.rec, dd.astype(np.float64), 10)
    return p, q, dm, dd, xs_ref, rn_ref


def test_lsrtm_matches_oracle_cg_iterate_by_iterate(survey):
    p, q, dm, dd, xs_ref, rn_ref = survey
    x, hist = lsrtm.lsrtm_cgls(Grid.of(p), dev(p.vel), p.src, dev(q), p.rec, dev(dd), 10, nsnap=32,
                               keep_iterates=True)
    errs = [float(np.linalg.norm(xk.cpu().numpy() - xr) / np.linalg.norm(xr))
            for xk, xr in zip(hist.iterates, xs_ref)]
    print(f"LSRTM iterates vs oracle CGLS: rel L2 {['%.1e' % e for e in errs]}")
    assert len(errs) == 10
    # CG amplifies the FP32 rounding of J and J' in its late iterations: the iterates track the
    # FP64 oracle's to about 1e-5 for seven iterations, then drift (about 3e-4 at the ninth,
    # 2e-3 at the tenth); the data residuals agree throughout, to 1e-3 of the data's norm
    assert max(errs[:8]) < 1e-3, errs
    assert max(errs) < 1e-2, errs
    np.testing.assert_allclose(hist.rnorm, rn_ref, rtol=0, atol=1e-3 * rn_ref[0])


def test_lsrtm_reduces_the_data_residual_tenfold(survey):
    p, q, dm, dd, xs_ref, rn_ref = survey
    x, hist = lsrtm.lsrtm_cgls(Grid.of(p), dev(p.vel), p.src, dev(q), p.rec, dev(dd), 10)
    assert hist.rnorm[-1] <= 0.1 * hist.rnorm[0], hist.rnorm
    assert all(b < a for a, b in zip(hist.rnorm, hist.rnorm[1:]))
    # the model error shrinks too (the problem has a null space, so not to zero)
    err = np.linalg.norm(x.cpu().numpy() - dm) / np.linalg.norm(dm)
    assert err < 0.5, err
