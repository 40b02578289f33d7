"""The FWI-experiment conditions and outer loops on the GPU: the low-cut
wavelet and the band-limited noise match the FP64 oracle; the vector updates
are exact; stochastic FWI with four random shots per iteration lowers the
misfit over all shots on low-cut, noisy data; the time-lapse batch (all vintage x shot
pairs in one uneven batch) matches the FP64 oracle vintage by vintage and equals one
gradient call per vintage."""
import numpy as np
import pytest
import torch

from oracle import conditioning as oc
from paper_2304_05592_gb300 import fwi, precond, synth, wave

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def rel(a, b):
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("nt,dt", [(2000, 0.8e-3), (1001, 0.5e-3)])
def test_lowcut_matches_oracle(nt, dt):
    import oracle

    qh = oracle.ricker(15.0, dt, nt).astype(np.float32)
    y = wave.wave_lowcut(dev(qh), dt, 4.0, 6.0).cpu().numpy()
    ref = oc.lowcut(qh.astype(np.float64), dt, 4.0, 6.0)
    assert rel(y, ref) < 1e-6
    f = np.arange(nt // 2 + 1) / (nt * dt)
    Y = np.abs(np.fft.rfft(y.astype(np.float64)))
    assert Y[f < 4.0].max() < 1e-5 * Y.max()  # float output rounding only


def test_noise_matches_oracle_and_snr():
    rng = np.random.default_rng(5)
    data = rng.standard_normal((3, 400, 37)).astype(np.float32)
    white = rng.standard_normal(data.shape).astype(np.float32)
    import oracle

    filt = oc.lowcut(oracle.ricker(15.0, 0.8e-3, 200), 0.8e-3, 4.0, 6.0).astype(np.float32)
    center = int(np.argmax(np.abs(filt)))
    out = wave.wave_add_noise(dev(data), dev(white), dev(filt), center, 10.0).cpu().numpy()
    ref = oc.add_noise(data, white, filt, center, 10.0)
    assert rel(out, ref) < 1e-5
    noise = out.astype(np.float64) - data
    assert abs(20 * np.log10(np.linalg.norm(data) / np.linalg.norm(noise)) - 10.0) < 1e-3


def test_axpy_and_clamp_are_exact():
    rng = np.random.default_rng(6)
    x, y = rng.standard_normal(1001).astype(np.float32), rng.standard_normal(1001).astype(np.float32)
    yd = dev(y)
    wave.wave_axpy(0.5, dev(x), yd)
    np.testing.assert_array_equal(yd.cpu().numpy(), (np.float32(0.5) * x + y).astype(np.float32))
    wave.wave_clamp(yd, -0.25, 0.75)
    assert float(yd.min()) >= -0.25 and float(yd.max()) <= 0.75


def _survey(nshot=8, nt=700):
    p = synth.plume_acquisition(nx=128, nz=64, h=10.0, nshot=nshot, nt=nt, nb=20)
    base, dv = synth.plume_model(7, nx=128, nz=64)
    return p, base, dv


def test_stochastic_fwi_with_lowcut_noisy_data_reduces_full_misfit():
    from scipy.ndimage import gaussian_filter

    p, base, dv = _survey()
    acq = precond.Acquisition.of(p)
    q = wave.wave_lowcut(acq.wavelet[0, :, 0].contiguous(), p.dt, 4.0, 6.0)
    acq.wavelet = q[None, :, None].repeat(p.nshot, 1, 1).contiguous()
    v_true = (base + dv).astype(np.float64)
    clean = wave.wave_forward(acq.grid, dev(v_true), p.src, acq.wavelet, p.rec)
    white = dev(np.random.default_rng(9).standard_normal(clean.shape))
    d_obs = wave.wave_add_noise(clean, white, q, int(torch.argmax(q.abs()).item()), 30.0)
    v0 = gaussian_filter(v_true, 8.0, mode="nearest")  # smooth starting model
    v, h = fwi.fwi_subsampled(acq, d_obs, dev(v0), iters=8, nsub=4, seed=1, full_every=4)
    assert all(len(s) == 4 for s in h.shots)
    assert h.solves >= 8 * 3  # forward + adjoint of the subset, and line-search forwards
    first, last = h.full_misfit[0][1], h.full_misfit[-1][1]
    assert last < 0.9 * first, h.full_misfit
    # most subset steps found descent
    assert sum(1 for a in h.step if a > 0) >= 6, h.step


@pytest.mark.parametrize("store,tol", [(wave.STORE_FP32, 1e-3), (wave.STORE_BF16, 1e-2)])
def test_timelapse_batch_matches_oracle_per_vintage(store, tol):
    # the block-diagonal time-lapse operator: every (vintage, shot) pair in one uneven batch, each
    # vintage's misfit and gradient checked against the FP64 oracle on its own model and data
    import oracle

    p, base, dv = _survey(nshot=3, nt=700)  # long enough for the plume's reflections to arrive
    vints = [base, base + 0.5 * dv, base + dv]
    models = [dev(v) for v in vints]
    og = oracle.Grid(2, p.nx, p.nz, p.h, p.dt, p.nt, p.nb, vref=p.vref)
    q32 = np.repeat(oracle.ricker(p.f0, p.dt, p.nt).astype(np.float32)[None, :, None], p.nshot, axis=0)
    q = q32.astype(np.float64)  # the same wavelet values on both sides, from the oracle
    # each vintage's observed data come from a model 2 % faster with a stronger plume: a
    # residual of a good fraction of the records (a residual of 1 % of them would be
    # dominated by the FP32 rounding of the 700-step synthetic records, about 4e-5 of them)
    d_obs_h = [oracle.forward(og, (1.02 * v + 0.5 * dv).astype(np.float64), p.src, q, p.rec) for v in vints]
    d_obs = [dev(d) for d in d_obs_h]
    mb, gb = fwi.timelapse_gradients(wave.Grid.of(p), models, p.src, p.rec, dev(q32), d_obs, store=store,
                                     wrt=wave.WRT_SLOWNESS2, batched=True)
    errs = []
    for i, v in enumerate(vints):
        phi_ref, g_ref = oracle.gradient(og, v.astype(np.float64), p.src, q, p.rec, d_obs_h[i])
        # the misfit is quadratic in records that match to 1e-4 (as in the uneven-batch tests)
        assert abs(mb[i] - phi_ref) <= 3e-4 * phi_ref, (i, mb[i], phi_ref)
        errs.append(rel(gb[i].cpu().numpy(), g_ref))
    print(f"time-lapse batch vs oracle, store {store}: gradient rel L2 per vintage {errs}")
    assert max(errs) < tol, errs


def test_timelapse_batch_equals_one_call_per_vintage():
    p, base, dv = _survey(nshot=3, nt=400)
    acq = precond.Acquisition.of(p)
    models = [dev(base), dev(base + 0.5 * dv), dev(base + dv)]
    d_obs = [wave.wave_forward(acq.grid, m, p.src, acq.wavelet, p.rec) for m in
             (dev(base + 0.1 * dv), dev(base + 0.6 * dv), dev(base + 1.1 * dv))]
    mb, gb = fwi.timelapse_gradients(acq.grid, models, p.src, p.rec, acq.wavelet, d_obs, batched=True)
    ml, gl = fwi.timelapse_gradients(acq.grid, models, p.src, p.rec, acq.wavelet, d_obs, batched=False)
    for a, b, x, y in zip(mb, ml, gb, gl):
        assert abs(a - b) <= 1e-5 * b
        assert float((x - y).norm() / y.norm()) < 1e-4
