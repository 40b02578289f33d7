"""Physics pins of the oracle: the Ricker wavelet's closed-form features, the
analytic homogeneous Green's functions (2D, 3D) convolved with the wavelet,
source-receiver reciprocity, exact discrete energy conservation without
damping, and absorption by the sponge."""
import numpy as np
import pytest
from scipy.ndimage import correlate1d

import oracle

from test_oracle_stencil import taylor_weights


def test_ricker_closed_form_features():
    f, dt, nt = 20.0, 1e-4, 2000
    q = oracle.ricker(f, dt, nt)
    t = np.arange(nt) * dt
    t0 = 1.0 / f
    n0 = int(round(t0 / dt))
    assert abs(q[n0] - 1.0) < 1e-12 and q.argmax() == n0 and abs(n0 * dt - t0) < 1e-15
    # zeros at t0 +/- 1/(pi f sqrt 2)
    tz = t0 + 1.0 / (np.pi * f * np.sqrt(2.0))
    i = int(np.floor(tz / dt))
    assert q[i] * q[i + 1] <= 0.0
    # minima at t0 +/- sqrt(3/2)/(pi f) with value -2 e^{-3/2}
    tm = t0 + np.sqrt(1.5) / (np.pi * f)
    j = int(round(tm / dt))
    assert abs(q[j - 3:j + 4].min() + 2 * np.exp(-1.5)) < 1e-6
    # amplitude spectrum peaks at f
    spec = np.abs(np.fft.rfft(q, 1 << 16))
    freqs = np.fft.rfftfreq(1 << 16, dt)
    assert abs(freqs[spec.argmax()] - f) < 0.2
    assert np.all(np.isfinite(t))


def _ricker_cont(t, f):
    a = (np.pi * f * (t - 1.0 / f)) ** 2
    return np.where(t >= 0, (1 - 2 * a) * np.exp(-a), 0.0)


def green2d_ricker(r, t, v, f, ns=6000):
    """(1/2 pi) int_0^{acosh(vt/r)} q(t - (r/v) cosh s) ds: the 2D Green's
    function H(vt-r) v / (2 pi sqrt(v^2 t^2 - r^2)) convolved in time with q."""
    out = np.zeros_like(t)
    for i, ti in enumerate(t):
        if v * ti <= r:
            continue
        S = np.arccosh(v * ti / r)
        s = np.linspace(0.0, S, ns)
        out[i] = np.trapezoid(_ricker_cont(ti - (r / v) * np.cosh(s), f), s) / (2 * np.pi)
    return out


def _homog_2d(h, dt, T, v=2000.0, f=15.0, L=1000.0):
    """Source at the centre of an L x L box with a 400 m sponge; receivers on
    the x axis and on the diagonal, all on grid points.  Over T = 0.36 s no
    wave returning from the sponge (path >= 800 m) reaches them."""
    n = int(round(L / h)) + 1
    nt = int(round(T / dt)) + 1
    g = oracle.Grid(2, n, n, h, dt, nt, int(round(400.0 / h)), vref=v)
    vel = np.full((n, n), v)
    c = (n // 2) * h
    src = np.array([[[c, c]]])
    pts = [(100.0, 0.0), (150.0, 0.0), (200.0, 0.0), (100.0, 100.0)]
    rec = np.array([[[c + a, c + b] for a, b in pts]])
    q = oracle.ricker(f, dt, nt)
    d = oracle.forward(g, vel, src, q[None, :, None], rec)[0]
    t = np.arange(nt) * dt
    ref = np.stack([green2d_ricker(np.hypot(a, b), t, v, f) for a, b in pts], axis=1)
    return d, ref


def test_green_2d_homogeneous_converges():
    d5, r5 = _homog_2d(5.0, 2e-4, 0.36)
    d10, r10 = _homog_2d(10.0, 4e-4, 0.36)
    e5 = np.linalg.norm(d5 - r5) / np.linalg.norm(r5)
    e10 = np.linalg.norm(d10 - r10) / np.linalg.norm(r10)
    assert e5 < 1e-2, e5
    assert e10 > 2.0 * e5, (e10, e5)


def _homog_3d(h, dt, T, v=2000.0, f=15.0, L=600.0):
    """Source at the centre of an L^3 box with a 200 m sponge; receivers at
    100 m and 150 m on grid points.  With T = 0.2 s the direct wave has passed
    before anything returning from the sponge (path >= 450 m) arrives."""
    n = int(round(L / h)) + 1
    nt = int(round(T / dt)) + 1
    nb = int(round(200.0 / h))
    g = oracle.Grid(3, n, n, h, dt, nt, nb, ny=n, vref=v)
    vel = np.full((n, n, n), v)
    c = (n // 2) * h
    src = np.array([[[c, c, c]]])
    pts = [(100.0, 0.0, 0.0), (0.0, 0.0, 100.0), (100.0, 100.0, 0.0), (0.0, 0.0, 140.0)]
    rec = np.array([[[c + a, c + b, c + e] for a, b, e in pts]])
    q = oracle.ricker(f, dt, nt)
    d = oracle.forward(g, vel, src, q[None, :, None], rec)[0]
    t = np.arange(nt) * dt
    ref = np.stack([_ricker_cont(t - np.linalg.norm(o) / v, f) / (4 * np.pi * np.linalg.norm(o))
                    for o in pts], axis=1)
    return d, ref


def test_green_3d_homogeneous_converges():
    d10, r10 = _homog_3d(10.0, 5e-4, 0.2)
    d20, r20 = _homog_3d(20.0, 1e-3, 0.2)
    e10 = np.linalg.norm(d10 - r10) / np.linalg.norm(r10)
    e20 = np.linalg.norm(d20 - r20) / np.linalg.norm(r20)
    assert e10 < 1e-2, e10
    assert e20 > 2.0 * e10, (e20, e10)


def _two_layer(nx=61, nz=51, h=10.0):
    z = np.arange(nz) * h
    v = np.where(z >= 250.0, 2600.0, 1600.0)
    return np.repeat(v[:, None], nx, axis=1)


def test_reciprocity_exact_with_sponge_and_offgrid_points():
    vel = _two_layer()
    nz, nx = vel.shape
    h = 10.0
    dt = 0.4 * oracle.courant_limit(2) * h / vel.max()
    g = oracle.Grid(2, nx, nz, h, dt, 500, 12, vref=vel.max())
    a = np.array([[[123.4, 37.9]]])
    b = np.array([[[471.2, 388.6]]])
    q = oracle.ricker(18.0, dt, g.nt)[None, :, None]
    d_ab = oracle.forward(g, vel, a, q, b)[0, :, 0]
    d_ba = oracle.forward(g, vel, b, q, a)[0, :, 0]
    assert np.abs(d_ab).max() > 0
    assert np.abs(d_ab - d_ba).max() <= 1e-12 * np.abs(d_ab).max()


def _own_laplacian(u, h):
    c = [float(x) for x in taylor_weights()]
    w = np.array(c[:0:-1] + c)  # c4..c1, c0, c1..c4
    out = np.zeros_like(u)
    for ax in range(u.ndim):
        out += correlate1d(u, w, axis=ax, mode="constant", cval=0.0)
    return out / (h * h)


@pytest.mark.parametrize("ndim", [2, 3])
def test_energy_conserved_without_damping(ndim):
    h = 10.0
    if ndim == 2:
        vel = _two_layer(41, 35, h)
        g0 = dict(nx=41, nz=35)
    else:
        z = np.arange(17) * h
        vel = np.repeat(np.where(z >= 80.0, 2600.0, 1600.0)[:, None, None], 19, axis=1)
        vel = np.repeat(vel, 21, axis=2)
        g0 = dict(nx=21, nz=17, ny=19)
    dt = 0.5 * oracle.courant_limit(ndim) * h / vel.max()
    nt = 700
    g = oracle.Grid(ndim, h=h, dt=dt, nt=nt, nb=3, vref=0.0, **g0)
    f = 25.0
    q = oracle.ricker(f, dt, nt)[None, :, None]
    src = np.array([[[150.0, 60.0] if ndim == 2 else [100.0, 90.0, 60.0]]])
    rec = src.copy()
    _, U = oracle.forward(g, vel, src, q, rec, fields=True)
    U = U[0]
    m = np.pad(1.0 / vel ** 2, 3, mode="edge")
    start = int(np.ceil(4.0 / f / dt))  # wavelet below 1e-16 beyond 3 t0 after its peak
    E = []
    for n in range(start, nt - 1):
        du = U[n + 1] - U[n]
        E.append(np.sum(m * du * du) - dt * dt * np.sum(U[n + 1] * _own_laplacian(U[n], h)))
    E = np.array(E)
    assert E[0] > 0
    assert (E.max() - E.min()) / E[0] < 1e-10


def test_sponge_absorbs():
    vel = np.full((41, 41), 2000.0)
    h = 10.0
    dt = 0.4 * oracle.courant_limit(2) * h / 2000.0
    nt = 1200
    src = np.array([[[200.0, 200.0]]])
    rec = np.array([[[200.0, 200.0], [100.0, 300.0]]])
    q = oracle.ricker(20.0, dt, nt)[None, :, None]
    late = slice(nt - 300, nt)
    d_abs = oracle.forward(oracle.Grid(2, 41, 41, h, dt, nt, 30, vref=2000.0), vel, src, q, rec)[0]
    d_ref = oracle.forward(oracle.Grid(2, 41, 41, h, dt, nt, 30, vref=0.0), vel, src, q, rec)[0]
    assert np.abs(d_abs[late]).max() < 5e-3 * np.abs(d_ref[late]).max()


def _sponge_eta(shape, nb, h, vref):
    """The sponge reading written out independently: eta = gamma0 (d/nb)^2 / vref^2,
    gamma0 = 3 vref ln(1000) / (2 nb h), d = depth into the sponge in cells (max over axes)."""
    depth = np.zeros(shape, dtype=np.int64)
    for ax, N in enumerate(shape):
        i = np.arange(N)
        d1 = np.maximum(np.maximum(nb - i, i - (N - nb - 1)), 0)
        sl = [None] * len(shape)
        sl[ax] = slice(None)
        depth = np.maximum(depth, d1[tuple(sl)])
    gamma0 = 3.0 * vref * np.log(1000.0) / (2.0 * nb * h)
    return gamma0 * (depth / nb) ** 2 / vref ** 2


def test_energy_balance_with_damping():
    """With damping the discrete energy drops each step by exactly
    ||u^{n+1} - u^{n-1}||^2_E, E = diag(eta dt / 2) (inner product of the step
    with u^{n+1} - u^{n-1}); this pins where and how eta enters the update."""
    h = 10.0
    vel = _two_layer(41, 35, h)
    nb = 8
    dt = 0.5 * oracle.courant_limit(2) * h / vel.max()
    nt = 500
    vref = float(vel.max())
    g = oracle.Grid(2, 41, 35, h, dt, nt, nb, vref=vref)
    f = 25.0
    q = oracle.ricker(f, dt, nt)[None, :, None]
    src = np.array([[[150.0, 60.0]]])
    _, U = oracle.forward(g, vel, src, q, src, fields=True)
    U = U[0]
    m = np.pad(1.0 / vel ** 2, nb, mode="edge")
    eta = _sponge_eta(m.shape, nb, h, vref)
    E = eta * dt / 2
    start = int(np.ceil(4.0 / f / dt))

    def energy(n):
        du = U[n + 1] - U[n]
        return np.sum(m * du * du) - dt * dt * np.sum(U[n + 1] * _own_laplacian(U[n], h))

    drops, preds = [], []
    for n in range(start, nt - 1):
        drops.append(energy(n) - energy(n - 1))
        c = U[n + 1] - U[n - 1]
        preds.append(-np.sum(E * c * c))
    drops, preds = np.array(drops), np.array(preds)
    assert np.all(preds < 0) and np.abs(preds).max() > 1e-6 * energy(start)
    assert np.abs(drops - preds).max() <= 1e-9 * np.abs(preds).max()
