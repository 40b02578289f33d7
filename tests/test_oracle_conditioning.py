"""Pins of the data-conditioning oracle (low-cut wavelet, band-limited noise)
against closed forms: DFT-grid sinusoids pass with gain 0, H(f) or 1; an
impulse of white noise reproduces the filter; the SNR is met exactly."""
import numpy as np

from oracle import conditioning as oc


def test_lowcut_gain_on_grid_sinusoids():
    nt, dt = 1000, 1e-3  # df = 1 Hz
    t = np.arange(nt) * dt
    for f, gain in ((2.0, 0.0), (4.0, 0.0), (5.0, 0.5), (6.0, 1.0), (30.0, 1.0)):
        x = np.cos(2 * np.pi * f * t + 0.3)
        y = oc.lowcut(x, dt, 4.0, 6.0)
        np.testing.assert_allclose(y, gain * x, atol=1e-12)
    np.testing.assert_allclose(oc.highpass_gain([4.5], 4.0, 6.0), [0.5 * (1 - np.cos(np.pi / 4))])


def test_lowcut_removes_low_band_of_a_ricker():
    from oracle import ricker
    nt, dt = 2000, 0.8e-3
    q = ricker(15.0, dt, nt)
    y = oc.lowcut(q, dt, 4.0, 6.0)
    f = np.arange(nt // 2 + 1) / (nt * dt)
    Y = np.abs(np.fft.rfft(y))
    assert Y[f < 4.0].max() < 1e-12 * Y.max()
    # far above the ramp the spectrum is untouched
    Q = np.abs(np.fft.rfft(q))
    np.testing.assert_allclose(Y[f > 10], Q[f > 10], rtol=1e-9, atol=1e-12 * Q.max())


def test_noise_impulse_response_and_snr():
    rng = np.random.default_rng(3)
    data = rng.standard_normal((2, 50, 3))
    filt = np.array([0.25, 1.0, -0.5, 0.125])
    white = np.zeros_like(data)
    white[1, 20, 2] = 1.0
    out = oc.add_noise(data, white, filt, 1, 12.0)
    noise = out - data
    # the only non-zero trace holds the filter, shifted by -center
    assert np.count_nonzero(np.abs(noise) > 1e-15) == filt.size
    tr = noise[1, :, 2]
    np.testing.assert_allclose(tr[19:23] / tr[20], filt / filt[1], atol=1e-12)
    assert abs(20 * np.log10(np.linalg.norm(data) / np.linalg.norm(noise)) - 12.0) < 1e-9
