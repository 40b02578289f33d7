"""Pins of the FP64 FNO oracle against facts that do not come from the oracle
itself: brute-force DFT sums, exact reconstruction of band-limited fields,
the sign convention on single Fourier modes, dot tests of the hand-written
adjoints, closed-form GELU values, finite differences of the whole network and
the Adam update written out for one scalar."""
import math

import numpy as np
import pytest

from oracle import fno

RNG = np.random.default_rng(1234)


def brute_dft(v, mz, mx):
    Nz, Nx = v.shape
    rows = list(range(mz)) + list(range(Nz - mz, Nz))
    X = np.zeros((2 * mz, mx), complex)
    for a, kz in enumerate(rows):
        for kx in range(mx):
            s = 0j
            for z in range(Nz):
                for x in range(Nx):
                    s += v[z, x] * complex(math.cos(2 * math.pi * (kz * z / Nz + kx * x / Nx)),
                                           -math.sin(2 * math.pi * (kz * z / Nz + kx * x / Nx)))
            X[a, kx] = s
    return X


def brute_idft(Y, Nz, Nx):
    mz, mx = Y.shape[0] // 2, Y.shape[1]
    rows = list(range(mz)) + list(range(Nz - mz, Nz))
    y = np.zeros((Nz, Nx))
    for z in range(Nz):
        for x in range(Nx):
            s = 0.0
            for a, kz in enumerate(rows):
                for kx in range(mx):
                    ang = 2 * math.pi * (kz * z / Nz + kx * x / Nx)
                    w = 1.0 if kx == 0 else 2.0
                    s += w * (Y[a, kx].real * math.cos(ang) - Y[a, kx].imag * math.sin(ang))
            y[z, x] = s / (Nz * Nx)
    return y


def test_truncated_dft_matches_brute_force():
    v = RNG.standard_normal((8, 10))
    X = fno.dft_trunc(v, 2, 3)
    np.testing.assert_allclose(X, brute_dft(v, 2, 3), rtol=0, atol=1e-12)


def test_truncated_inverse_matches_brute_force():
    Y = RNG.standard_normal((4, 3)) + 1j * RNG.standard_normal((4, 3))
    np.testing.assert_allclose(fno.idft_trunc(Y, 8, 10), brute_idft(Y, 8, 10), rtol=0, atol=1e-12)


def test_band_limited_field_is_reconstructed():
    # a real field whose spectrum lies inside the kept modes (and their
    # conjugates) survives S T exactly: this pins the 1/(Nz Nx) and w_kx
    Nz, Nx, mz, mx = 16, 20, 3, 4
    z, x = np.meshgrid(np.arange(Nz), np.arange(Nx), indexing="ij")
    v = np.zeros((Nz, Nx))
    for kz in range(-mz + 1, mz):
        for kx in range(mx):
            a, b = RNG.standard_normal(2)
            ang = 2 * np.pi * (kz * z / Nz + kx * x / Nx)
            v += a * np.cos(ang) + b * np.sin(ang)
    np.testing.assert_allclose(fno.idft_trunc(fno.dft_trunc(v, mz, mx), Nz, Nx), v, atol=1e-11)


def test_single_mode_sign_convention():
    # v = cos(psi) with R = 1 returns cos(psi); with R = i it returns -sin(psi)
    Nz, Nx, mz, mx = 12, 16, 3, 4
    z, x = np.meshgrid(np.arange(Nz), np.arange(Nx), indexing="ij")
    psi = 2 * np.pi * (2 * z / Nz + 3 * x / Nx)
    X = fno.dft_trunc(np.cos(psi), mz, mx)
    np.testing.assert_allclose(fno.idft_trunc(X, Nz, Nx), np.cos(psi), atol=1e-12)
    np.testing.assert_allclose(fno.idft_trunc(1j * X, Nz, Nx), -np.sin(psi), atol=1e-12)
    # a mode outside the kept band is removed
    far = np.cos(2 * np.pi * (5 * z / Nz))
    np.testing.assert_allclose(fno.idft_trunc(fno.dft_trunc(far, mz, mx), Nz, Nx), 0.0, atol=1e-12)


@pytest.mark.parametrize("shape", [(8, 10, 2, 3), (16, 12, 4, 5)])
def test_adjoints_pass_dot_tests(shape):
    Nz, Nx, mz, mx = shape
    v = RNG.standard_normal((2, Nz, Nx))
    dX = RNG.standard_normal((2, 2 * mz, mx)) + 1j * RNG.standard_normal((2, 2 * mz, mx))
    lhs = np.sum(np.real(np.conj(fno.dft_trunc(v, mz, mx)) * dX))
    rhs = np.sum(v * fno.dft_trunc_adjoint(dX, Nz, Nx))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    Y = RNG.standard_normal((2, 2 * mz, mx)) + 1j * RNG.standard_normal((2, 2 * mz, mx))
    dy = RNG.standard_normal((2, Nz, Nx))
    lhs = np.sum(fno.idft_trunc(Y, Nz, Nx) * dy)
    rhs = np.sum(np.real(np.conj(Y) * fno.idft_trunc_adjoint(dy, mz, mx)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_gelu_closed_forms():
    # GELU(x) = x Phi(x): Phi(1) = 0.841344746068543 (standard normal table)
    assert abs(fno.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(fno.gelu(-1.0) + 0.15865525393145707) < 1e-15
    assert fno.gelu(0.0) == 0.0
    assert abs(fno.gelu_grad(0.0) - 0.5) < 1e-15
    x = np.linspace(-4, 4, 33)
    h = 1e-6
    np.testing.assert_allclose(fno.gelu_grad(x), (fno.gelu(x + h) - fno.gelu(x - h)) / (2 * h), atol=1e-9)


def test_network_gradient_matches_finite_differences():
    cfg = fno.Config(cin=3, width=4, hidden=5, layers=3, mz=2, mx=3)
    p = fno.init_params(cfg, seed=7)
    x = RNG.standard_normal((2, 3, 8, 12))
    target = RNG.standard_normal((2, 1, 8, 12))

    def loss(q):
        out, _ = fno.forward(q, x, cfg)
        return fno.mse(out, target)[0]

    out, cache = fno.forward(p, x, cfg)
    _, dout = fno.mse(out, target)
    g = fno.backward(p, cache, dout, cfg)
    h = 1e-6
    for name in p:
        arr = p[name]
        for _ in range(3):
            idx = tuple(int(RNG.integers(0, s)) for s in arr.shape)
            for part, unit in (("re", 1.0), ("im", 1j)):
                if part == "im" and not np.iscomplexobj(arr):
                    continue
                q = {k: v.copy() for k, v in p.items()}
                q[name][idx] += h * unit
                lp = loss(q)
                q[name][idx] -= 2 * h * unit
                lm = loss(q)
                fd = (lp - lm) / (2 * h)
                an = g[name][idx].real if part == "re" else g[name][idx].imag
                assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)), (name, idx, part, fd, an)


def test_adam_first_step_is_sign_times_lr():
    # with m0 = v0 = 0 the bias-corrected first step is lr * g / (|g| + eps)
    p, m, v = fno.adam(np.array([1.0, -2.0]), np.array([0.5, -3.0]), np.zeros(2), np.zeros(2), 1, 0.1)
    np.testing.assert_allclose(p, [1.0 - 0.1 * 0.5 / (0.5 + 1e-8), -2.0 + 0.1 * 3.0 / (3.0 + 1e-8)], atol=1e-15)


def test_adam_constant_gradient_moves_lr_per_step_for_every_t():
    # with a constant gradient the bias-corrected moments are exactly g and g^2 at every t
    # (m_t = (1 - b1^t) g, v_t = (1 - b2^t) g^2), so each of the first steps moves
    # lr * g / (|g| + eps); a bias-correction exponent frozen at 1 fails from t = 2 on
    for b1, b2 in [(0.9, 0.999), (0.8, 0.95)]:
        g = np.array([0.5, -3.0, 1e-8])
        p, m, v = np.array([1.0, -2.0, 0.0]), np.zeros(3), np.zeros(3)
        for t in range(1, 6):
            p, m, v = fno.adam(p, g, m, v, t, 0.1, b1, b2)
            np.testing.assert_allclose(m, (1 - b1 ** t) * g, rtol=1e-13, atol=0)
            np.testing.assert_allclose(v, (1 - b2 ** t) * g * g, rtol=1e-13, atol=0)
            step = 0.1 * g / (np.abs(g) + 1e-8)  # eps outside the square root: the tiny entry moves lr / 2
            np.testing.assert_allclose(p, np.array([1.0, -2.0, 0.0]) - t * step, rtol=1e-12, atol=1e-15)


def test_adam_alternating_gradient_matches_closed_form_moments():
    # g_t = (-1)^(t+1): m_t = (1-b1) (-1)^(t+1) (1 - (-b1)^t) / (1 + b1) and v_t = 1 - b2^t, so
    # vhat_t = 1 and the step is lr * m_t / (1 - b1^t) / (1 + eps); swapping b1 and b2 in the
    # moment updates (or in the bias corrections) changes every one of these
    lr = 0.05
    for b1, b2 in [(0.9, 0.999), (0.8, 0.95)]:
        p, m, v = np.array([0.3]), np.zeros(1), np.zeros(1)
        expect_p = 0.3
        for t in range(1, 8):
            g = np.array([(-1.0) ** (t + 1)])
            p, m, v = fno.adam(p, g, m, v, t, lr, b1, b2)
            mt = (1 - b1) * (-1.0) ** (t + 1) * (1 - (-b1) ** t) / (1 + b1)
            vt = 1 - b2 ** t
            np.testing.assert_allclose(m, [mt], rtol=1e-13)
            np.testing.assert_allclose(v, [vt], rtol=1e-13)
            expect_p -= lr * (mt / (1 - b1 ** t)) / (1.0 + 1e-8)
            np.testing.assert_allclose(p, [expect_p], rtol=1e-13)


def test_twiddle_tables_factor_the_truncated_transforms():
    # T v = sum_z conj(ez) (v fwd), S Y = Re(ez Y inv^T), and the two adjoints through bwd and adj,
    # against the brute-force-pinned dft_trunc / idft_trunc and their adjoints
    rng = np.random.default_rng(11)
    Nz, Nx, mz, mx = 10, 14, 3, 4
    fwd, inv, bwd, adj, ez = fno.twiddle_tables(Nz, Nx, mz, mx)
    v = rng.standard_normal((Nz, Nx))
    np.testing.assert_allclose(np.conj(ez).T @ (v @ fwd), fno.dft_trunc(v, mz, mx), atol=1e-11)
    Y = rng.standard_normal((2 * mz, mx)) + 1j * rng.standard_normal((2 * mz, mx))
    np.testing.assert_allclose(((ez @ Y) @ inv.T).real, fno.idft_trunc(Y, Nz, Nx), atol=1e-13)
    dy = rng.standard_normal((Nz, Nx))
    np.testing.assert_allclose(np.conj(ez).T @ (dy @ bwd), fno.idft_trunc_adjoint(dy, mz, mx), atol=1e-13)
    np.testing.assert_allclose(((ez @ Y) @ adj.T).real, fno.dft_trunc_adjoint(Y, Nz, Nx), atol=1e-11)
