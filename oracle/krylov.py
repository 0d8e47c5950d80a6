"""Preconditioned MinRes and GMRES (oracle side, test infrastructure).

Textbook Lanczos-based MINRES for a symmetric (possibly indefinite) operator K
with a symmetric positive definite preconditioner P ~ K^{-1}, minimising the
residual in the P-norm (Paige & Saunders 1975; the preconditioned form of
Elman, Silvester & Wathen, Alg. 4.1).  The paper solves with GMRES (Sec. 8);
MinRes is the symmetric alternative the block preconditioner eq.
(mhatinvfactor) permits because it is symmetric positive definite.  ``gmres``
is the textbook right-preconditioned, unrestarted GMRES (Saad & Schultz 1986:
Arnoldi with modified Gram-Schmidt, Givens rotations), minimising ||b - K x||_2,
for comparison with the paper's iteration counts.
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


def gmres(K, P, b, x0=None, rtol=1e-6, maxit=500, project=None):
    """Right-preconditioned GMRES for K x = b: x = x0 + P y with y from the Krylov space of K P,
    minimising ||b - K x||_2; stops when it falls below rtol * ||b - K x0||_2.  ``project`` is
    applied to every preconditioned vector.  Returns (x, iterations, history of ||r||_2)."""
    proj = project if project is not None else (lambda v: v)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - K(x)
    beta = float(np.linalg.norm(r))
    hist = [beta]
    if beta == 0.0:
        return x, 0, hist
    V = [r / beta]
    Z = []
    H = np.zeros((maxit + 1, maxit))
    cs, sn = np.zeros(maxit), np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    it = 0
    for j in range(maxit):
        z = proj(P(V[j]))
        Z.append(z)
        w = K(z)
        for i in range(j + 1):                      # modified Gram-Schmidt
            H[i, j] = float(w @ V[i])
            w = w - H[i, j] * V[i]
        hn = float(np.linalg.norm(w))
        H[j + 1, j] = hn
        V.append(w / hn if hn > 0.0 else w)
        for i in range(j):                          # previous rotations
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        den = math.hypot(H[j, j], H[j + 1, j])
        cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        it = j + 1
        hist.append(abs(g[j + 1]))
        if abs(g[j + 1]) <= rtol * beta or hn == 0.0:
            break
    y = np.linalg.solve(np.triu(H[:it, :it]), g[:it])
    for i in range(it):
        x = x + y[i] * Z[i]
    return x, it, hist
