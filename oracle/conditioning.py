"""FP64 oracle of the data conditioning of the paper's FWI experiment (test
infrastructure only; only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import it): a wavelet with no energy
below a cut frequency and additive coloured Gaussian noise with the bandwidth
of the noise-free data (arxiv 2304.05592, section "Deep priors and
normalizing flows").

* ``lowcut``: the real DFT of q (numpy.fft, a library routine) times the gain
  H(f) = 0 for f < f_cut, 0.5 (1 - cos(pi (f - f_cut) / (f_pass - f_cut))) up to
  f_pass, 1 above; then the inverse real DFT.
* ``add_noise``: each trace of the white draws convolved with the filter
  (centred at tap `center`), scaled so that 20 log10(||data|| / ||noise||) equals
  the requested SNR, and added to the data.

Pinned by ``tests/test_oracle_conditioning.py``: sinusoids on the DFT grid
below, inside and above the ramp come out scaled by exactly 0, H(f) and 1; an
impulse of white noise returns the shifted, scaled filter; the SNR is exact.
"""
from __future__ import annotations

import numpy as np


def highpass_gain(f, f_cut: float, f_pass: float):
    f = np.asarray(f, float)
    ramp = 0.5 * (1.0 - np.cos(np.pi * (f - f_cut) / (f_pass - f_cut)))
    return np.where(f < f_cut, 0.0, np.where(f < f_pass, ramp, 1.0))


def lowcut(q, dt: float, f_cut: float, f_pass: float) -> np.ndarray:
    q = np.asarray(q, float)
    nt = q.size
    Q = np.fft.rfft(q)
    f = np.arange(Q.size) / (nt * dt)
    return np.fft.irfft(Q * highpass_gain(f, f_cut, f_pass), n=nt)


def add_noise(data, white, filt, center: int, snr_db: float) -> np.ndarray:
    """data, white: [nshot][nt][nrec]; filt: [nf]."""
    data = np.asarray(data, float)
    white = np.asarray(white, float)
    filt = np.asarray(filt, float)
    ns, nt, nr = data.shape
    noise = np.zeros_like(data)
    for s in range(ns):
        for r in range(nr):
            full = np.convolve(white[s, :, r], filt)  # full[t'] = sum_k f[k] w[t' - k]
            noise[s, :, r] = full[center:center + nt]
    scale = 10.0 ** (-snr_db / 20.0) * np.linalg.norm(data) / np.linalg.norm(noise)
    return data + scale * noise
