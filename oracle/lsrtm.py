"""FP64 CPU oracle of least-squares reverse-time migration (test
infrastructure only; only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import it).

Least-squares RTM fits a model perturbation dm to data dd through the Born
operator J = judiJacobian(F, q) of the paper (section "Wave-equation-based
inversion"): min 1/2 ||J dm - dd||^2.  The paper names J and J' and leaves
the solver open; the reading here is conjugate gradients on the normal
equations J'J dm = J' dd in the Hestenes-Stiefel form for least squares
(CGLS), starting from dm = 0:

    r = dd, s = J' r, p = s, gamma = <s, s>
    repeat: q = J p;  alpha = gamma / <q, q>;  dm += alpha p;  r -= alpha q;
            s = J' r;  gamma' = <s, s>;  p = s + (gamma' / gamma) p;  gamma = gamma'

``cgls`` takes the operator and its adjoint as callables (pinned on dense
matrices against numpy's least-squares solution); ``lsrtm`` plugs in the
oracle's Born modelling and J' (the gradient of the misfit at the data
F(m) q - r is J' r).
"""
from __future__ import annotations

import numpy as np

from . import born, forward, gradient


def cgls(A, At, dd: np.ndarray, x_shape, niter: int):
    """CGLS iterates of min 1/2 ||A x - dd||^2 from x = 0.  Returns (x, xs,
    rnorms): the last iterate, every iterate x_1..x_niter, and ||dd - A x_k||
    for k = 0..niter."""
    x = np.zeros(x_shape)
    r = np.array(dd, dtype=np.float64, copy=True)
    s = At(r)
    p = s.copy()
    gamma = float(np.vdot(s, s))
    xs, rn = [], [float(np.linalg.norm(r))]
    for _ in range(niter):
        q = A(p)
        qq = float(np.vdot(q, q))
        if qq == 0.0 or gamma == 0.0:
            break
        alpha = gamma / qq
        x = x + alpha * p
        r = r - alpha * q
        s = At(r)
        gamma_new = float(np.vdot(s, s))
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        xs.append(x.copy())
        rn.append(float(np.linalg.norm(r)))
    return x, xs, rn


def jacobian_adjoint(g, vel, src, wavelet, rec, r) -> np.ndarray:
    """J' r summed over shots: the misfit gradient at observed data F(m) q - r."""
    d0 = forward(g, vel, src, wavelet, rec)
    return gradient(g, vel, src, wavelet, rec, d0 - np.asarray(r, dtype=np.float64))[1]


def lsrtm(g, vel, src, wavelet, rec, dd, niter: int):
    """CGLS on the wave problem: dm (physical grid) fitting the data dd
    [nshot][nt][nrec] through the Born operator at the velocity vel."""
    d0 = forward(g, vel, src, wavelet, rec)

    def A(dm):
        return born(g, vel, src, wavelet, rec, dm)

    def At(r):
        return gradient(g, vel, src, wavelet, rec, d0 - r)[1]

    return cgls(A, At, dd, g.phys_shape, niter)
