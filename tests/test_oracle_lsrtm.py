"""Pins of the least-squares RTM oracle (oracle/lsrtm.py): CGLS on dense
matrices against the textbook least-squares solution and CG properties, and
the oracle's J' against its Born operator (dot test)."""
import numpy as np

import oracle
from oracle import lsrtm
from paper_2304_05592_gb300 import synth


def test_cgls_reaches_the_least_squares_solution_in_n_steps():
    # in exact arithmetic CGLS solves an n-unknown problem in n steps; numpy's lstsq is the reference
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 12)) @ np.diag(np.linspace(1.0, 5.0, 12))
    b = rng.standard_normal(40)
    x, xs, rn = lsrtm.cgls(lambda v: A @ v, lambda r: A.T @ r, b, (12,), 12)
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    np.testing.assert_allclose(x, ref, rtol=1e-8, atol=1e-10)
    assert len(xs) == 12 and len(rn) == 13


def test_cgls_residuals_decrease_and_first_step_is_exact_line_search():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((60, 30))
    b = rng.standard_normal(60)
    x, xs, rn = lsrtm.cgls(lambda v: A @ v, lambda r: A.T @ r, b, (30,), 10)
    assert all(rn[k + 1] < rn[k] for k in range(10))  # ||b - A x_k|| decreases strictly
    # x_1 is the steepest-descent step along A'b with the exact step length
    s = A.T @ b
    alpha = (s @ s) / np.sum((A @ s) ** 2)
    np.testing.assert_allclose(xs[0], alpha * s, rtol=1e-12)
    # normal-equation residuals of successive iterates are orthogonal (a CG property)
    g = [A.T @ (b - A @ xk) for xk in xs]
    for k in range(len(g) - 1):
        assert abs(g[k] @ g[k + 1]) <= 1e-8 * np.linalg.norm(g[k]) * np.linalg.norm(g[k + 1])


def test_cgls_breaks_off_on_a_zero_right_hand_side():
    A = np.eye(3)
    x, xs, rn = lsrtm.cgls(lambda v: A @ v, lambda r: A.T @ r, np.zeros(3), (3,), 5)
    assert not xs and np.all(x == 0) and rn == [0.0]


def test_oracle_jacobian_adjoint_passes_the_dot_test():
    p = synth.small_2d(3, nx=30, nz=24, nt=120, nshot=2, nrec=9)
    g = oracle.Grid(2, p.nx, p.nz, p.h, p.dt, p.nt, p.nb, vref=p.vref)
    q = np.repeat(oracle.ricker(p.f0, p.dt, p.nt)[None, :, None], p.nshot, axis=0)
    rng = np.random.default_rng(4)
    dm = rng.standard_normal(g.phys_shape) * 1e-8
    r = rng.standard_normal((p.nshot, p.nt, p.rec.shape[1]))
    lhs = np.vdot(oracle.born(g, p.vel, p.src, q, p.rec, dm), r)
    rhs = np.vdot(dm, lsrtm.jacobian_adjoint(g, p.vel, p.src, q, p.rec, r))
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), abs(rhs))
