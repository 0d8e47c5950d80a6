"""Oracle pins: reference polynomials and quadrature against closed forms and SciPy."""
import math

import numpy as np
import pytest
from scipy.special import eval_jacobi

from oracle import polys


@pytest.mark.parametrize("alpha", [0, 1, 3, 7])
def test_homogeneous_jacobi_matches_scipy(alpha):
    x = np.linspace(0.05, 0.95, 11)
    for m in range(8):
        v, _, _ = polys.hjacobi(m, alpha, x, 1.0)
        assert np.allclose(v, eval_jacobi(m, alpha, 0, 2 * x - 1), rtol=1e-13, atol=1e-13)
        # homogeneity: H(t x, t s) = t^m H(x, s)
        v2, _, _ = polys.hjacobi(m, alpha, 0.5 * x, 0.5)
        assert np.allclose(v2, 0.5 ** m * v, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_quadrature_exact_on_monomials(n):
    # int_{T_n} x^a = prod(a_i!) / (|a| + n)!
    pts, w = polys.quadrature(n, 5)
    for a in np.ndindex(*(10,) * n):
        if sum(a) > 9:
            continue
        exact = np.prod([math.factorial(i) for i in a]) / math.factorial(sum(a) + n)
        got = np.sum(w * np.prod(pts ** np.array(a), axis=1))
        assert abs(got - exact) < 1e-14 * max(1.0, exact) + 1e-16


@pytest.mark.parametrize("n,k", [(1, 6), (2, 6), (3, 5)])
def test_dubiner_orthonormal_and_hierarchical(n, k):
    pts, w = polys.quadrature(n, k + 2)
    V, _ = polys.dubiner(n, k, pts)
    assert np.abs((V * w[:, None]).T @ V - np.eye(V.shape[1])).max() < 1e-13
    assert V.shape[1] == polys.n_poly(n, k)
    # the first dim P^{k-1} functions span P^{k-1}: orthogonal to all monomials of degree < deg
    degs = polys.degrees(n, k)
    for j in range(V.shape[1]):
        for a in np.ndindex(*(k + 1,) * n):
            if sum(a) < degs[j]:
                mono = np.prod(pts ** np.array(a), axis=1)
                assert abs(np.sum(w * mono * V[:, j])) < 1e-13


@pytest.mark.parametrize("n", [2, 3])
def test_dubiner_gradients_fd(n):
    rng = np.random.default_rng(1)
    p = rng.random((6, n)) * (0.8 / n)
    V, G = polys.dubiner(n, 5, p)
    h = 1e-6
    for a in range(n):
        e = np.zeros(n)
        e[a] = h
        fd = (polys.dubiner(n, 5, p + e)[0] - polys.dubiner(n, 5, p - e)[0]) / (2 * h)
        assert np.abs(fd - G[..., a]).max() < 1e-6 * max(1, np.abs(G).max())
