"""Preconditioned MinRes (oracle side, test infrastructure).

Textbook Lanczos-based MINRES for a symmetric (possibly indefinite) operator K
with a symmetric positive definite preconditioner P ~ K^{-1}, minimising the
residual in the P-norm (Paige & Saunders 1975; the preconditioned form of
Elman, Silvester & Wathen, Alg. 4.1).  The paper solves with GMRES (Sec. 7);
MinRes is the symmetric alternative the block preconditioner eq.
(mhatinvfactor) permits because it is symmetric positive definite.
"""
from __future__ import annotations

import math

import numpy as np


def minres(K, P, b, x0=None, rtol=1e-10, maxit=1000, project=None):
    """Solve K x = b.  K, P are callables.  Stops when the preconditioned residual
    norm ||r||_P falls below rtol * ||r0||_P.  ``project`` (optional) is applied to
    every preconditioned vector (e.g. removing the pressure mean).

    Returns (x, iterations, history of ||r||_P)."""
    proj = project if project is not None else (lambda v: v)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    v_old = np.zeros_like(b)
    v = b - K(x)
    z = proj(P(v))
    gamma = math.sqrt(max(float(z @ v), 0.0))
    gamma_old = 1.0
    eta = gamma
    hist = [gamma]
    if gamma == 0.0:
        return x, 0, hist
    c_old, c = 1.0, 1.0
    s_old, s = 0.0, 0.0
    w_old = np.zeros_like(b)
    w = np.zeros_like(b)
    res0 = gamma
    it = 0
    for it in range(1, maxit + 1):
        z = z / gamma
        Kz = K(z)
        delta = float(Kz @ z)
        v_new = Kz - (delta / gamma) * v - (gamma / gamma_old) * v_old
        z_new = proj(P(v_new))
        gamma_new = math.sqrt(max(float(z_new @ v_new), 0.0))
        a0 = c * delta - c_old * s * gamma
        a1 = math.sqrt(a0 * a0 + gamma_new * gamma_new)
        a2 = s * delta + c_old * c * gamma
        a3 = s_old * gamma
        c_old, s_old = c, s
        c, s = a0 / a1, gamma_new / a1
        w_new = (z - a3 * w_old - a2 * w) / a1
        x = x + c * eta * w_new
        eta = -s * eta
        hist.append(abs(eta))
        w_old, w = w, w_new
        v_old, v = v, v_new
        z = z_new
        gamma_old, gamma = gamma, gamma_new
        if abs(eta) <= rtol * res0 or gamma == 0.0:
            break
    return x, it, hist
