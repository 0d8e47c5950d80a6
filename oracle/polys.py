"""Reference-simplex polynomials and quadrature for the oracle (test infrastructure).

Reference simplex T_n = {x in R^n : x_i >= 0, sum x_i <= 1}, vertices 0, e_1..e_n.

Orthonormal (Dubiner / Koornwinder) basis on T_n, n = 1, 2, 3, built from
Jacobi polynomials P_m^{(alpha,0)} written in homogeneous form

    H_m^{(alpha)}(x, s) = s^m P_m^{(alpha,0)}(2x/s - 1),

which is a polynomial in (x, s).  The unnormalised basis functions are

    n = 1:  H_p^{(0)}(x, 1)
    n = 2:  H_p^{(0)}(x, 1-y) H_q^{(2p+1)}(y, 1)
    n = 3:  H_p^{(0)}(x, 1-y-z) H_q^{(2p+1)}(y, 1-z) H_r^{(2p+2q+2)}(z, 1)

each scaled to unit L2(T_n) norm (no sign change).  Order: total degree
ascending; n = 2: q ascending within a degree; n = 3: r ascending, then q
ascending.  This family, its order and its normalisation are the basis of the
pressure space Q_h and of the facet moments in the dof contract; the paper
leaves bases open (it only cites a hierarchical basis in Sec. 4.2), so this is
a reading recorded with the dof contract.

Quadrature: collapsed (Duffy) Gauss rules with SciPy's Gauss-Legendre and
Gauss-Jacobi nodes (library primitives); q points per direction integrate total
degree 2q-1 exactly.
"""
from __future__ import annotations

import functools
import math

import numpy as np
from scipy.special import roots_jacobi


def n_poly(n: int, k: int) -> int:
    """dim P^k(R^n) (0 for k < 0)."""
    if k < 0:
        return 0
    return math.comb(k + n, n)


def index_list(n: int, k: int):
    """Multi-indices of the orthonormal basis of P^k(T_n) in the basis order."""
    out = []
    for m in range(k + 1):
        if n == 1:
            out.append((m,))
        elif n == 2:
            for q in range(m + 1):
                out.append((m - q, q))
        elif n == 3:
            for r in range(m + 1):
                for q in range(m - r + 1):
                    out.append((m - q - r, q, r))
        else:
            raise ValueError(n)
    return out


def hjacobi(m: int, alpha: int, x, s):
    """H_m^{(alpha)}(x, s) and its partial derivatives (value, d/dx, d/ds).

    Homogenised form of the three-term recurrence of P_m^{(alpha,0)}.
    """
    x = np.asarray(x, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64) * np.ones_like(x)
    h0, h0x, h0s = np.ones_like(x), np.zeros_like(x), np.zeros_like(x)
    if m == 0:
        return h0, h0x, h0s
    h1 = (alpha + 2) * x - s
    h1x = np.full_like(x, alpha + 2.0)
    h1s = -np.ones_like(x)
    a = alpha
    for nn in range(2, m + 1):
        an = 2 * nn * (nn + a) * (2 * nn + a - 2)
        bn = (2 * nn + a - 1) * (2 * nn + a) * (2 * nn + a - 2)
        cn = (2 * nn + a - 1) * a * a
        dn = 2 * (nn + a - 1) * (nn - 1) * (2 * nn + a)
        lin = bn * (2 * x - s) + cn * s
        h2 = (lin * h1 - dn * s * s * h0) / an
        h2x = (2 * bn * h1 + lin * h1x - dn * s * s * h0x) / an
        h2s = ((cn - bn) * h1 + lin * h1s - 2 * dn * s * h0 - dn * s * s * h0s) / an
        h0, h0x, h0s = h1, h1x, h1s
        h1, h1x, h1s = h2, h2x, h2s
    return h1, h1x, h1s


def _raw(n: int, idx, pts):
    """Unnormalised basis function idx at points pts[..., n]: (value, gradient[..., n])."""
    pts = np.asarray(pts, dtype=np.float64)
    if n == 1:
        (p,) = idx
        v, vx, _ = hjacobi(p, 0, pts[..., 0], 1.0)
        return v, vx[..., None]
    if n == 2:
        p, q = idx
        x, y = pts[..., 0], pts[..., 1]
        A, Ax, As = hjacobi(p, 0, x, 1.0 - y)
        B, Bx, _ = hjacobi(q, 2 * p + 1, y, 1.0)
        val = A * B
        gx = Ax * B
        gy = -As * B + A * Bx
        return val, np.stack([gx, gy], axis=-1)
    if n == 3:
        p, q, r = idx
        x, y, z = pts[..., 0], pts[..., 1], pts[..., 2]
        A, Ax, As = hjacobi(p, 0, x, 1.0 - y - z)
        B, Bx, Bs = hjacobi(q, 2 * p + 1, y, 1.0 - z)
        C, Cx, _ = hjacobi(r, 2 * p + 2 * q + 2, z, 1.0)
        val = A * B * C
        gx = Ax * B * C
        gy = -As * B * C + A * Bx * C
        gz = -As * B * C - A * Bs * C + A * B * Cx
        return val, np.stack([gx, gy, gz], axis=-1)
    raise ValueError(n)


def quadrature(n: int, q: int):
    """Collapsed Gauss rule on T_n with q points per direction: (points[nq, n], weights[nq])."""
    if n == 0:
        return np.zeros((1, 0)), np.ones(1)
    a, wa = roots_jacobi(q, 0.0, 0.0)
    if n == 1:
        return ((1 + a) / 2)[:, None], wa / 2
    b, wb = roots_jacobi(q, 1.0, 0.0)
    if n == 2:
        A, B = np.meshgrid(a, b, indexing="ij")
        WA, WB = np.meshgrid(wa, wb, indexing="ij")
        y = (1 + B) / 2
        x = (1 + A) * (1 - B) / 4
        return np.stack([x.ravel(), y.ravel()], axis=1), (WA * WB).ravel() / 8
    c, wc = roots_jacobi(q, 2.0, 0.0)
    if n == 3:
        A, B, C = np.meshgrid(a, b, c, indexing="ij")
        WA, WB, WC = np.meshgrid(wa, wb, wc, indexing="ij")
        z = (1 + C) / 2
        y = (1 + B) * (1 - C) / 4
        x = (1 + A) * (1 - B) * (1 - C) / 8
        return (np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1),
                (WA * WB * WC).ravel() / 64)
    raise ValueError(n)


@functools.lru_cache(maxsize=None)
def _norms(n: int, k: int):
    pts, w = quadrature(n, k + 2)
    out = []
    for idx in index_list(n, k):
        v, _ = _raw(n, idx, pts)
        out.append(1.0 / math.sqrt(float(np.sum(w * v * v))))
    return np.array(out)


def dubiner(n: int, k: int, pts):
    """Orthonormal basis of P^k(T_n) at pts[..., n]: values[..., nb], gradients[..., nb, n]."""
    pts = np.asarray(pts, dtype=np.float64)
    norms = _norms(n, k)
    vals, grads = [], []
    for c, idx in zip(norms, index_list(n, k)):
        v, g = _raw(n, idx, pts)
        vals.append(c * v)
        grads.append(c * g)
    return np.stack(vals, axis=-1), np.stack(grads, axis=-2)


def degrees(n: int, k: int):
    """Total degree of each orthonormal basis function, in basis order."""
    return np.array([sum(i) for i in index_list(n, k)])
