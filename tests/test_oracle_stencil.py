"""Pins of the oracle's spatial operator against mathematics fixed independently
of its source: Taylor-derived weights, polynomial exactness, 8th-order
convergence, symmetry, and the stability limit of the leapfrog scheme."""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def taylor_weights():
    """Weights c_0..c_4 of the symmetric 9-point second derivative, solved from
    the moment conditions sum_j c_|j| j^p = 2 [p == 2], p = 0, 2, 4, 6, 8,
    in exact rational arithmetic (Gauss-Jordan on Fractions)."""
    rows = []
    for p in (0, 2, 4, 6, 8):
        row = [Fraction(1 if p == 0 else 0)]  # j = 0 contributes 0^p
        for k in range(1, 5):
            row.append(Fraction(2 * k ** p))
        rows.append(row + [Fraction(2 if p == 2 else 0)])
    n = 5
    for i in range(n):
        piv = next(r for r in range(i, n) if rows[r][i] != 0)
        rows[i], rows[piv] = rows[piv], rows[i]
        rows[i] = [x / rows[i][i] for x in rows[i]]
        for r in range(n):
            if r != i and rows[r][i] != 0:
                f = rows[r][i]
                rows[r] = [a - f * b for a, b in zip(rows[r], rows[i])]
    return [rows[i][n] for i in range(n)]


def test_taylor_weights_are_textbook():
    c = taylor_weights()
    assert c == [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315), Fraction(-1, 560)]


def _grid2(nx=31, nz=27, h=0.1, nb=0):
    return oracle.Grid(2, nx, nz, h, 1e-4, 2, nb)


@pytest.mark.parametrize("deg", [2, 5, 9])
def test_laplacian_exact_on_polynomials(deg):
    g = _grid2()
    Nz, Nx = g.pad_shape
    x = (np.arange(Nx) - Nx / 2) * g.h
    z = (np.arange(Nz) - Nz / 2) * g.h
    rng = np.random.default_rng(deg)
    a = rng.standard_normal(deg + 1)
    b = rng.standard_normal(deg + 1)
    P = np.polynomial.Polynomial(a)
    Q = np.polynomial.Polynomial(b)
    u = P(x)[None, :] + Q(z)[:, None] + 0.0 * x[None, :] * z[:, None]
    exact = P.deriv(2)(x)[None, :] + Q.deriv(2)(z)[:, None]
    Lu = oracle.laplacian(g, u)
    inner = (slice(4, Nz - 4), slice(4, Nx - 4))
    err = np.abs(Lu[inner] - exact[inner]).max() / np.abs(exact[inner]).max()
    assert err < 1e-9


def test_laplacian_error_on_degree_10_is_the_tenth_moment():
    """For x^10 the only surviving Taylor term is h^8 sum_j c_|j| j^10 (a
    constant): the stencil is not exact there, and the error is that constant."""
    c = taylor_weights()
    m10 = float(2 * sum(c[k] * k ** 10 for k in range(1, 5)))
    assert m10 != 0.0
    g = _grid2()
    Nz, Nx = g.pad_shape
    x = (np.arange(Nx) - Nx / 2) * g.h
    u = np.repeat((x ** 10)[None, :], Nz, axis=0)
    exact = 90 * x ** 8
    Lu = oracle.laplacian(g, u)
    err = Lu[Nz // 2, 4:-4] - exact[4:-4]
    assert np.allclose(err, m10 * g.h ** 8, rtol=1e-5, atol=0)


def test_laplacian_eighth_order_convergence():
    errs = []
    for h in (0.1, 0.05):
        n = int(round(4.0 / h)) + 1
        g = oracle.Grid(2, n, 9, h, 1e-4, 2, 0)
        Nz, Nx = g.pad_shape
        x = np.arange(Nx) * h
        k = 2.0
        u = np.repeat(np.sin(k * x)[None, :], Nz, axis=0)
        Lu = oracle.laplacian(g, u)
        e = np.abs(Lu[4, 4:-4] + k * k * np.sin(k * x[4:-4])).max()
        errs.append(e)
    ratio = errs[0] / errs[1]
    assert 200 < ratio < 300, ratio  # 2^8 = 256


def test_laplacian_3d_matches_axis_sum():
    g = oracle.Grid(3, 11, 9, 0.2, 1e-4, 2, 2, ny=10)
    rng = np.random.default_rng(5)
    Nz, Ny, Nx = g.pad_shape
    x = np.arange(Nx) * g.h
    y = np.arange(Ny) * g.h
    z = np.arange(Nz) * g.h
    u = (np.sin(1.3 * x)[None, None, :] * np.cos(0.7 * y)[None, :, None] * np.exp(0.1 * z)[:, None, None])
    Lu = oracle.laplacian(g, u)
    exact = (-1.69 - 0.49 + 0.01) * u
    inner = (slice(4, -4),) * 3
    assert np.abs(Lu[inner] - exact[inner]).max() / np.abs(exact[inner]).max() < 1e-6
    a = rng.standard_normal(g.pad_shape)
    b = rng.standard_normal(g.pad_shape)
    lhs = np.vdot(a, oracle.laplacian(g, b))
    rhs = np.vdot(oracle.laplacian(g, a), b)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_laplacian_symmetric_with_zero_ghosts():
    g = _grid2(13, 11, 1.0, 3)
    rng = np.random.default_rng(1)
    a = rng.standard_normal(g.pad_shape)
    b = rng.standard_normal(g.pad_shape)
    lhs = np.vdot(a, oracle.laplacian(g, b))
    rhs = np.vdot(oracle.laplacian(g, a), b)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("ndim", [2, 3])
def test_courant_limit_from_symbol(ndim):
    c = [float(x) for x in taylor_weights()]
    k = np.linspace(0, np.pi, 100001)
    symbol = c[0] + 2 * sum(c[j] * np.cos(j * k) for j in range(1, 5))
    kmax = np.abs(symbol).max()
    assert abs(kmax - 2048 / 315) < 1e-9
    limit = 2.0 / np.sqrt(ndim * kmax)
    assert abs(oracle.courant_limit(ndim) - limit) < 1e-12


def test_cfl_rejected_just_above_limit_and_stable_below():
    from paper_2304_05592_gb300 import synth

    nx = nz = 40
    h = 10.0
    vel = np.full((nz, nx), 2000.0)
    lim = oracle.courant_limit(2) * h / 2000.0
    src = np.array([[[200.0, 200.0]]])
    rec = np.array([[[100.0, 100.0]]])
    g = oracle.Grid(2, nx, nz, h, lim * 1.001, 50, 4)
    with pytest.raises(oracle.OracleError) as e:
        oracle.forward(g, vel, src, np.ones((1, 50, 1)), rec)
    assert e.value.code == oracle.ERR_CFL
    g = oracle.Grid(2, nx, nz, h, lim * 0.98, 3000, 4)
    q = np.zeros((1, 3000, 1))
    q[0, :20, 0] = 1.0
    d = oracle.forward(g, vel, src, q, rec)
    assert np.isfinite(d).all() and np.abs(d).max() < 1.0
    assert synth is not None
