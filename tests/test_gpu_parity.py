"""GPU parity: libwave's CUDA kernels, called through the C ABI, against the
FP64 oracle on the same seeded inputs.  Tolerances (relative L2 over the
whole array): 1e-4 for shot records and source-side adjoints, 1e-3 for
gradients (FP32 arithmetic against FP64)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2304_05592_gb300 import synth, wave
from paper_2304_05592_gb300.wave import Grid

pytestmark = pytest.mark.gpu

TOL_DATA = 1e-4
TOL_GRAD = 1e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def ogrid(p):
    return oracle.Grid(p.ndim, p.nx, p.nz, p.h, p.dt, p.nt, p.nb, ny=p.ny, vref=p.vref)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def ricker_batch(p):
    q = oracle.ricker(p.f0, p.dt, p.nt).astype(np.float32)
    return np.repeat(q[None, :, None], p.nshot, axis=0)


def test_ricker_matches_oracle():
    for f, dt, nt in [(15.0, 8e-4, 1000), (20.0, 5e-4, 4000), (7.5, 1e-3, 17)]:
        g = wave.wave_ricker(f, dt, nt).cpu().numpy()
        r = oracle.ricker(np.float32(f), np.float32(dt), nt)
        assert np.abs(g - r).max() < 2e-7


@pytest.mark.parametrize("mk", [lambda: synth.small_2d(21, nt=300),
                                lambda: synth.small_2d(22, nx=150, nz=37, nt=250, nb=20, nshot=4, nrec=61),
                                lambda: synth.small_3d(23, nt=120)])
def test_forward_matches_oracle(mk):
    p = mk()
    q = ricker_batch(p)
    d = wave.wave_forward(Grid.of(p), dev(p.vel), p.src, dev(q), p.rec).cpu().numpy()
    r = oracle.forward(ogrid(p), p.vel, p.src, q, p.rec)
    assert np.all(d[:, 0] == 0)
    for s in range(p.nshot):
        assert rel(d[s], r[s]) < TOL_DATA, (s, rel(d[s], r[s]))


@pytest.mark.parametrize("mk", [lambda: synth.small_2d(31, nt=260), lambda: synth.small_3d(32, nt=100)])
def test_adjoint_matches_oracle(mk):
    p = mk()
    rng = np.random.default_rng(5)
    r = rng.standard_normal((p.nshot, p.nt, p.rec.shape[1])).astype(np.float32)
    g = wave.wave_adjoint(Grid.of(p), dev(p.vel), p.src, p.rec, dev(r)).cpu().numpy()
    o = oracle.adjoint(ogrid(p), p.vel, p.src, p.rec, r)
    assert np.all(g[:, -1] == 0)
    assert rel(g, o) < TOL_DATA, rel(g, o)


def _grad_case(p, seed=7):
    q = ricker_batch(p)
    v_true = p.vel
    v0 = (p.vel * 1.03).astype(np.float32)
    dobs = oracle.forward(ogrid(p), v_true, p.src, q, p.rec).astype(np.float32)
    return q, v0, dobs


@pytest.mark.parametrize("store,nsnap", [(wave.STORE_CHECKPOINT, 3), (wave.STORE_CHECKPOINT, 200),
                                         (wave.STORE_FP32, 1), (wave.STORE_BF16, 1)])
def test_gradient_matches_oracle_2d(store, nsnap):
    p = synth.small_2d(41, nt=280)
    q, v0, dobs = _grad_case(p)
    phi, g, dsyn = wave.wave_gradient(Grid.of(p), dev(v0), p.src, dev(q), p.rec, dev(dobs), store=store,
                                      nsnap=nsnap, want_dsyn=True)
    phi_r, g_r = oracle.gradient(ogrid(p), v0, p.src, q, p.rec, dobs)
    d_r = oracle.forward(ogrid(p), v0, p.src, q, p.rec)
    assert rel(dsyn.cpu().numpy(), d_r) < TOL_DATA
    assert abs(phi - phi_r) <= 1e-4 * phi_r
    e = rel(g.cpu().numpy(), g_r)
    tol = TOL_GRAD if store != wave.STORE_BF16 else 1e-2
    assert e < tol, e


def test_checkpointed_gradient_equals_full_storage_bitwise():
    p = synth.small_2d(42, nt=301, nshot=2)
    q, v0, dobs = _grad_case(p)
    args = (Grid.of(p), dev(v0), p.src, dev(q), p.rec, dev(dobs))
    _, g32, _ = wave.wave_gradient(*args, store=wave.STORE_FP32)
    for nsnap in (1, 4, 37, 500):
        _, gc, _ = wave.wave_gradient(*args, store=wave.STORE_CHECKPOINT, nsnap=nsnap)
        assert torch.equal(gc, g32), nsnap


def test_gradient_matches_oracle_3d():
    p = synth.small_3d(43, nt=90)
    q, v0, dobs = _grad_case(p)
    phi, g, _ = wave.wave_gradient(Grid.of(p), dev(v0), p.src, dev(q), p.rec, dev(dobs), nsnap=6)
    phi_r, g_r = oracle.gradient(ogrid(p), v0, p.src, q, p.rec, dobs)
    assert abs(phi - phi_r) <= 1e-4 * phi_r
    assert rel(g.cpu().numpy(), g_r) < TOL_GRAD


@pytest.mark.parametrize("mk", [lambda: synth.small_2d(51, nt=300), lambda: synth.small_3d(52, nt=100)])
def test_dot_test_fp32(mk):
    p = mk()
    rng = np.random.default_rng(3)
    q = rng.standard_normal((p.nshot, p.nt, 1)).astype(np.float32)
    r = rng.standard_normal((p.nshot, p.nt, p.rec.shape[1])).astype(np.float32)
    g = Grid.of(p)
    Fq = wave.wave_forward(g, dev(p.vel), p.src, dev(q), p.rec).double()
    Ftr = wave.wave_adjoint(g, dev(p.vel), p.src, p.rec, dev(r)).double()
    a = float((Fq * dev(r).double()).sum())
    b = float((dev(q).double() * Ftr).sum())
    assert abs(a - b) <= 1e-5 * max(abs(a), abs(b)), abs(a - b) / abs(a)


def test_batched_shots_equal_one_at_a_time_bitwise():
    p = synth.small_2d(61, nt=200, nshot=5)
    q = ricker_batch(p)
    g = Grid.of(p)
    d_all = wave.wave_forward(g, dev(p.vel), p.src, dev(q), p.rec)
    for s in range(p.nshot):
        d_one = wave.wave_forward(g, dev(p.vel), p.src[s:s + 1], dev(q[s:s + 1]), p.rec[s:s + 1])
        assert torch.equal(d_one[0], d_all[s])


def test_repeatable_bitwise():
    p = synth.small_2d(62, nt=200)
    q, v0, dobs = _grad_case(p)
    args = (Grid.of(p), dev(v0), p.src, dev(q), p.rec, dev(dobs))
    a = wave.wave_gradient(*args, nsnap=5)[1]
    b = wave.wave_gradient(*args, nsnap=5)[1]
    assert torch.equal(a, b)


def test_config1_forward_full_size():
    p = synth.config1()
    q = ricker_batch(p)
    d = wave.wave_forward(Grid.of(p), dev(p.vel), p.src, dev(q), p.rec).cpu().numpy()
    r = oracle.forward(ogrid(p), p.vel, p.src, q, p.rec)
    assert rel(d, r) < TOL_DATA, rel(d, r)


# ---------------------------------------------------------------------------
# Edge cases and errors.


def test_empty_batches_and_single_sample():
    p = synth.small_2d(71, nt=50, nshot=2)
    g = Grid.of(p)
    q = ricker_batch(p)
    d = wave.wave_forward(g, dev(p.vel), p.src[:0], dev(q[:0]), p.rec[:0])
    assert d.shape == (0, p.nt, p.rec.shape[1])
    d = wave.wave_forward(g, dev(p.vel), p.src, dev(q), p.rec[:, :0])
    assert d.shape == (p.nshot, p.nt, 0)
    dobs = np.zeros((p.nshot, p.nt, 0), np.float32)
    phi, gr, _ = wave.wave_gradient(g, dev(p.vel), p.src, dev(q), p.rec[:, :0], dev(dobs))
    assert phi == 0.0 and float(gr.abs().max()) == 0.0
    g1 = Grid(**{**g.__dict__, "nt": 1})
    dobs = synth.observed_noise((p.nshot, 1, p.rec.shape[1]), 1.0, 3)
    phi, gr, _ = wave.wave_gradient(g1, dev(p.vel), p.src, dev(q[:, :1]), p.rec, dev(dobs))
    assert abs(phi - 0.5 * np.sum(dobs.astype(np.float64) ** 2)) < 1e-9 * phi
    assert float(gr.abs().max()) == 0.0


def test_errors_are_reported():
    p = synth.small_2d(72, nt=40, nshot=1)
    g = Grid.of(p)
    q = dev(ricker_batch(p))
    bad = p.vel.copy()
    bad[3, 4] = np.nan
    with pytest.raises(wave.WaveError) as e:
        wave.wave_forward(g, dev(bad), p.src, q, p.rec)
    assert e.value.status == 7
    bad[3, 4] = -1.0
    with pytest.raises(wave.WaveError) as e:
        wave.wave_forward(g, dev(bad), p.src, q, p.rec)
    assert e.value.status == 7
    fast = (p.vel * 3.0).astype(np.float32)
    with pytest.raises(wave.WaveError) as e:
        wave.wave_forward(g, dev(fast), p.src, q, p.rec)
    assert e.value.status == 2
    rec = p.rec.copy()
    rec[0, 0, 1] = (p.nz - 1) * p.h * 1.01
    with pytest.raises(wave.WaveError) as e:
        wave.wave_forward(g, dev(p.vel), p.src, q, rec)
    assert e.value.status == 3
    # the library still works after the errors
    d = wave.wave_forward(g, dev(p.vel), p.src, q, p.rec)
    assert torch.isfinite(d).all()


@pytest.fixture
def restore_variants():
    yield
    wave.wave_set_variant(0, -1)
    wave.wave_set_variant(1, -1)
    wave.wave_set_variant(2, -1)


def test_every_2d_kernel_variant_matches(restore_variants):
    """Each 2D step variant gives the oracle's records and gradient; records
    are bitwise those of variant 0 (the per-point arithmetic does not depend on
    the tiling) and gradients agree to rounding (the shot sum may be grouped)."""
    p = synth.small_2d(91, nx=150, nz=61, nt=240, nshot=3, nrec=41)
    q, v0, dobs = _grad_case(p)
    g = Grid.of(p)
    d_ref = oracle.forward(ogrid(p), v0, p.src, q, p.rec)
    _, g_ref = oracle.gradient(ogrid(p), v0, p.src, q, p.rec, dobs)
    base = None
    for vf in range(wave.wave_variant_count(0)):
        for va in range(wave.wave_variant_count(1)):
            if vf and va and vf != va:
                continue
            wave.wave_set_variant(0, vf)
            wave.wave_set_variant(1, va)
            d = wave.wave_forward(g, dev(v0), p.src, dev(q), p.rec)
            _, gr, _ = wave.wave_gradient(g, dev(v0), p.src, dev(q), p.rec, dev(dobs), nsnap=7)
            assert rel(d.cpu().numpy(), d_ref) < TOL_DATA, (vf, va)
            assert rel(gr.cpu().numpy(), g_ref) < TOL_GRAD, (vf, va)
            if base is None:
                base = (d, gr)
            else:
                # records are bitwise the same; shot-group kernels sum the
                # gradient per group first, so only the summation order differs
                assert torch.equal(d, base[0]), (vf, va)
                assert float((gr - base[1]).norm() / base[1].norm()) < 1e-5, (vf, va)


def test_every_3d_kernel_variant_matches(restore_variants):
    """Each 3D step variant (z-march, TMA plane rings of 8 or 16 rows and 32 or
    64 planes) gives the oracle's records and gradient on a grid with ragged
    tiles in x, y and z, and the records are bitwise the same for all."""
    p = synth.small_3d(94, nx=150, ny=40, nz=70, nt=60, nshot=2, nrec=31)
    q = ricker_batch(p)
    g = Grid.of(p)
    v0 = (p.vel * 1.02).astype(np.float32)
    dobs = oracle.forward(ogrid(p), p.vel, p.src, q, p.rec).astype(np.float32)
    d_ref = oracle.forward(ogrid(p), v0, p.src, q, p.rec)
    _, g_ref = oracle.gradient(ogrid(p), v0, p.src, q, p.rec, dobs)
    base = None
    for v in range(wave.wave_variant_count(2)):
        wave.wave_set_variant(2, v)
        d = wave.wave_forward(g, dev(v0), p.src, dev(q), p.rec)
        _, gr, _ = wave.wave_gradient(g, dev(v0), p.src, dev(q), p.rec, dev(dobs), nsnap=5)
        assert rel(d.cpu().numpy(), d_ref) < TOL_DATA, v
        assert rel(gr.cpu().numpy(), g_ref) < TOL_GRAD, v
        if base is None:
            base = (d, gr)
        else:
            assert torch.equal(d, base[0]), v
            assert float((gr - base[1]).norm() / base[1].norm()) < 1e-6, v


def test_autotune_picks_valid_variants_and_results_hold(restore_variants):
    p = synth.small_2d(92, nx=120, nz=50, nt=200, nshot=4, nrec=30)
    q, v0, dobs = _grad_case(p)
    g = Grid.of(p)
    bf, ba = wave.wave_autotune(g, dev(v0), p.src, dev(q), p.rec, steps=5)
    assert 0 <= bf < wave.wave_variant_count(0) and 0 <= ba < wave.wave_variant_count(1)
    _, gr, _ = wave.wave_gradient(g, dev(v0), p.src, dev(q), p.rec, dev(dobs), nsnap=9)
    _, g_ref = oracle.gradient(ogrid(p), v0, p.src, q, p.rec, dobs)
    assert rel(gr.cpu().numpy(), g_ref) < TOL_GRAD
    p3 = synth.small_3d(93, nt=40)
    assert wave.wave_autotune(Grid.of(p3), dev(p3.vel), p3.src, dev(ricker_batch(p3)), p3.rec, steps=3) == (-1, -1)
