"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

Holds none of the method's arithmetic: only closed-form data (manufactured
solutions and their right-hand sides, derived by hand from the strong form
f = -div(nu eps(u)) + grad p with div u = 0, i.e. f = -(nu/2) Lap u + grad p),
seeded random coefficient vectors, and the workload definitions.

Workloads (the paper's channel and airplane meshes are not available; these
structured Kuhn meshes stand in for them, with the paper's element types, degrees
and dof densities):
  c1: 2D 8x8 cells (128 triangles), k=2, nu=1, manufactured solution.
  c2: 2D 256x256 cells (131,072 triangles), 5 multigrid levels (16^2 coarsest),
      k=3, nu=1e-2, manufactured solution.
  c3: 3D 32^3 cubes x 6 (196,608 tets), 4 levels (4^3 coarsest), k=2, nu=1.
  c4: 3D 16^3 x 6 (24,576 tets), k in {2..6} here (k=1 needs the Sec. 6 variant),
      random f = sum c_j phi_j with c_j ~ N(0,1), seed-fixed, nu=1.
"""
from __future__ import annotations

import math

import numpy as np

WORKLOADS = {
    "c1": dict(dim=2, N=8, k=2, nu=1.0, levels=-1, rhs="manufactured", rtol=1e-10),
    "c2": dict(dim=2, N=256, k=3, nu=1e-2, levels=5, rhs="manufactured", rtol=1e-8),
    "c3": dict(dim=3, N=32, k=2, nu=1.0, levels=4, rhs="manufactured", rtol=1e-8),
}


def _ns(x):
    try:
        import torch
        if isinstance(x, torch.Tensor):
            return torch
    except ImportError:
        pass
    return np


def _ab(t, ns):
    """a(t) = t^2 (1-t)^2 and its first three derivatives."""
    a = t * t * (1 - t) * (1 - t)
    a1 = 2 * t - 6 * t * t + 4 * t ** 3
    a2 = 2 - 12 * t + 12 * t * t
    a3 = -12 + 24 * t
    return a, a1, a2, a3


def manufactured_f(dim: int, nu: float, x):
    """Right-hand side of the manufactured Stokes solution at points x[..., dim]."""
    ns = _ns(x)
    pi = math.pi
    if dim == 2:
        X, Y = x[..., 0], x[..., 1]
        a, a1, a2, a3 = _ab(X, ns)
        b, b1, b2, b3 = _ab(Y, ns)
        f1 = -0.5 * nu * (a2 * b1 + a * b3) + pi * ns.cos(pi * X) * ns.cos(pi * Y)
        f2 = 0.5 * nu * (a3 * b + a1 * b2) - pi * ns.sin(pi * X) * ns.sin(pi * Y)
        return ns.stack([f1, f2], -1)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    a, a1, a2, a3 = _ab(X, ns)
    b, b1, b2, b3 = _ab(Y, ns)
    c, c1, c2, c3 = _ab(Z, ns)
    Dx = a3 * b * c + a1 * b2 * c + a1 * b * c2
    Dy = a2 * b1 * c + a * b3 * c + a * b1 * c2
    Dz = a2 * b * c1 + a * b2 * c1 + a * b * c3
    sx, sy, sz = ns.sin(pi * X), ns.sin(pi * Y), ns.sin(pi * Z)
    cx, cy, cz = ns.cos(pi * X), ns.cos(pi * Y), ns.cos(pi * Z)
    f1 = -0.5 * nu * (Dy - Dz) + pi * cx * sy * sz
    f2 = -0.5 * nu * (Dz - Dx) + pi * sx * cy * sz
    f3 = -0.5 * nu * (Dx - Dy) + pi * sx * sy * cz
    return ns.stack([f1, f2, f3], -1)


def manufactured_u(dim: int, x):
    ns = _ns(x)
    if dim == 2:
        a, a1, _, _ = _ab(x[..., 0], ns)
        b, b1, _, _ = _ab(x[..., 1], ns)
        return ns.stack([a * b1, -a1 * b], -1)
    a, a1, _, _ = _ab(x[..., 0], ns)
    b, b1, _, _ = _ab(x[..., 1], ns)
    c, c1, _, _ = _ab(x[..., 2], ns)
    px, py, pz = a1 * b * c, a * b1 * c, a * b * c1
    return ns.stack([py - pz, pz - px, px - py], -1)


def manufactured_p(dim: int, x):
    ns = _ns(x)
    pi = math.pi
    if dim == 2:
        return ns.sin(pi * x[..., 0]) * ns.cos(pi * x[..., 1])
    return ns.sin(pi * x[..., 0]) * ns.sin(pi * x[..., 1]) * ns.sin(pi * x[..., 2]) - (2 / pi) ** 3


def random_coefficients(n: int, seed: int) -> np.ndarray:
    """i.i.d. N(0,1) coefficients (numpy default_rng)."""
    return np.random.default_rng(seed).standard_normal(n)
