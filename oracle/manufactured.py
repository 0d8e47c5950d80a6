"""Manufactured Stokes solutions (oracle side, test infrastructure).

Right-hand sides are derived symbolically from the strong form eq. (stokes):
f = -div(nu eps(u)) + grad p, with nu as printed (reading R5).

* 2D: u = curl psi = (d_y psi, -d_x psi) (reading R7), psi = x^2(1-x)^2 y^2(1-y)^2,
      p = sin(pi x) cos(pi y)  (mean zero on the unit square).
* 3D: u = curl (psi, psi, psi), psi = x^2(1-x)^2 y^2(1-y)^2 z^2(1-z)^2,
      p = sin(pi x) sin(pi y) sin(pi z) - (2/pi)^3  (mean removed).
"""
from __future__ import annotations

import functools

import numpy as np
import sympy as sy


@functools.lru_cache(maxsize=None)
def _symbolic(dim: int):
    if dim == 2:
        x, y = X = sy.symbols("x y")
        psi = x**2 * (1 - x)**2 * y**2 * (1 - y)**2
        u = [sy.diff(psi, y), -sy.diff(psi, x)]
        p = sy.sin(sy.pi * x) * sy.cos(sy.pi * y)
    else:
        x, y, z = X = sy.symbols("x y z")
        psi = x**2 * (1 - x)**2 * y**2 * (1 - y)**2 * z**2 * (1 - z)**2
        A = [psi, psi, psi]
        u = [sy.diff(A[2], y) - sy.diff(A[1], z),
             sy.diff(A[0], z) - sy.diff(A[2], x),
             sy.diff(A[1], x) - sy.diff(A[0], y)]
        p = sy.sin(sy.pi * x) * sy.sin(sy.pi * y) * sy.sin(sy.pi * z) - (2 / sy.pi) ** 3
    nu = sy.symbols("nu")
    d = len(X)
    eps = [[(sy.diff(u[a], X[b]) + sy.diff(u[b], X[a])) / 2 for b in range(d)] for a in range(d)]
    f = [-sum(sy.diff(nu * eps[a][b], X[b]) for b in range(d)) + sy.diff(p, X[a]) for a in range(d)]
    grad_u = [[sy.diff(u[a], X[b]) for b in range(d)] for a in range(d)]
    return X, nu, u, p, f, grad_u


class Manufactured:
    def __init__(self, dim: int, nu: float):
        X, nus, u, p, f, gu = _symbolic(dim)
        self.dim = dim
        self.nu = nu
        sub = {nus: nu}
        self._u = [sy.lambdify(X, c, "numpy") for c in u]
        self._p = sy.lambdify(X, p, "numpy")
        self._f = [sy.lambdify(X, c.subs(sub), "numpy") for c in f]
        self._gu = [[sy.lambdify(X, c, "numpy") for c in row] for row in gu]

    def _ev(self, fns, x):
        args = [x[..., a] for a in range(self.dim)]
        return np.stack([np.broadcast_to(fn(*args), x.shape[:-1]) for fn in fns], axis=-1)

    def u(self, x):
        return self._ev(self._u, x)

    def p(self, x):
        args = [x[..., a] for a in range(self.dim)]
        return np.broadcast_to(self._p(*args), x.shape[:-1]).astype(np.float64)

    def f(self, x):
        return self._ev(self._f, x)

    def grad_u(self, x):
        return np.stack([self._ev(row, x) for row in self._gu], axis=-2)


@functools.lru_cache(maxsize=None)
def _symbolic_outflow():
    """2D, Gamma_Ntilde = {x = 1}, Dirichlet elsewhere: u = curl psi with
    psi = x^2 (3 - 2x) y^2 (1 - y)^2, so u = 0 on x = 0 and y = 0, 1, u_y = 0 and u_x != 0 on x = 1;
    p = nu d_x u_x + (1 - x) cos(pi y), so that ((sigma + p I) n).n = -nu d_x u_x + p = 0 on x = 1."""
    x, y = X = sy.symbols("x y")
    nu = sy.symbols("nu")
    psi = x**2 * (3 - 2 * x) * y**2 * (1 - y)**2
    u = [sy.diff(psi, y), -sy.diff(psi, x)]
    p = nu * sy.diff(u[0], x) + (1 - x) * sy.cos(sy.pi * y)
    eps = [[(sy.diff(u[a], X[b]) + sy.diff(u[b], X[a])) / 2 for b in range(2)] for a in range(2)]
    f = [-sum(sy.diff(nu * eps[a][b], X[b]) for b in range(2)) + sy.diff(p, X[a]) for a in range(2)]
    return X, nu, u, p, f


class ManufacturedOutflow(Manufactured):
    """Manufactured solution with the outflow condition of eq. (stokes_NT) on x = 1 (2D)."""

    def __init__(self, nu: float):
        X, nus, u, p, f = _symbolic_outflow()
        self.dim = 2
        self.nu = nu
        sub = {nus: nu}
        self._u = [sy.lambdify(X, c, "numpy") for c in u]
        self._p = sy.lambdify(X, p.subs(sub), "numpy")
        self._f = [sy.lambdify(X, c.subs(sub), "numpy") for c in f]
        self._gu = [[sy.lambdify(X, sy.diff(c, v), "numpy") for v in X] for c in u]
