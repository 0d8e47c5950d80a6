"""Pins of the oracle's geometric multigrid (the conforming solver C of Sec. 6.1, reading R11).

The device V-cycle is checked step for step against ``oracle.precond.GMG``; these tests fix the
oracle itself by what the mathematics of nested conforming P1 spaces gives, independently of how
the prolongation and the V-cycle are written:

* the prolongation is the inclusion of the coarse P1 space: a coarse field (random values at the
  interior vertices, zero on the boundary), evaluated at every fine vertex by locating it in a
  coarse element and taking barycentric coordinates there, equals P applied to its coarse values;
* Galerkin identity: for nested spaces and the same form abar = nu (eps, eps) (eq. defAhat,
  reading R1), P^T Abar_h P = Abar_{2h} exactly (to rounding), over one and over several levels;
* the V-cycle is a symmetric operator B with eigenvalues of B Abar in (0, 1], which is what
  Corollary aux_pc_mult asks of C (Abar <= C, i.e. lambda_max(C^{-1} Abar) <= 1).

Each pin is shown to fail when a plausible mistake is planted in the oracle (CPU only): a midpoint
weight of 1 instead of 1/2, an off-by-one coarse vertex, a dropped post-smoothing sweep, and the
plain diagonal in place of the l1 diagonal.
"""
import numpy as np
import pytest

from oracle import mesh, precond


def _coarse_field_at(coarse: mesh.Mesh, vals: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Piecewise-linear field of the coarse mesh (vertex values vals [nv, d]) at the point x:
    the first coarse element whose barycentric coordinates of x are all >= 0."""
    d = coarse.dim
    for T in range(coarse.elems.shape[0]):
        V = coarse.coords[coarse.elems[T]]
        J = (V[1:] - V[0]).T
        lam_r = np.linalg.solve(J, x - V[0])
        lam = np.concatenate([[1.0 - lam_r.sum()], lam_r])
        if lam.min() >= -1e-12:
            return lam @ vals[coarse.elems[T]]
    raise AssertionError("point outside the coarse mesh")


def _interp_by_location(coarse: mesh.Mesh, fine: mesh.Mesh, c: np.ndarray) -> np.ndarray:
    """Fine interior dofs of the coarse P1 field with interior dofs c (vertex-major rank*d + comp)."""
    d = coarse.dim
    rc, nc = precond.p1_map(coarse)
    rf, nf = precond.p1_map(fine)
    vals = np.zeros((coarse.coords.shape[0], d))
    inner = rc >= 0
    vals[inner] = c.reshape(nc, d)[rc[inner]]
    out = np.zeros((nf, d))
    for vid in np.nonzero(rf >= 0)[0]:
        out[rf[vid]] = _coarse_field_at(coarse, vals, fine.coords[vid])
    return out.ravel()


LEVEL_CASES = [(2, 2, 4), (2, 4, 2), (3, 2, 3), (3, 2, 2)]   # (dim, coarsest N, levels)


def _hierarchy(d, N0, levels):
    return [mesh.structured(d, N0 << l) for l in range(levels)]


@pytest.mark.parametrize("d,N0,levels", LEVEL_CASES)
def test_prolongation_is_the_inclusion(d, N0, levels):
    ms = _hierarchy(d, N0, levels)
    rng = np.random.default_rng(5)
    for l in range(1, levels):
        P = precond.prolongation(ms[l - 1], ms[l])
        _, nc = precond.p1_map(ms[l - 1])
        for _ in range(2):
            c = rng.standard_normal(nc * d)
            ref = _interp_by_location(ms[l - 1], ms[l], c)
            assert np.abs(P @ c - ref).max() <= 1e-14 * max(np.abs(ref).max(), 1.0)


@pytest.mark.parametrize("d,N0,levels", LEVEL_CASES)
def test_galerkin_identity(d, N0, levels, nu=0.37):
    """P^T Abar_h P = Abar_{2h} for each pair of levels, and for the product over all levels."""
    ms = _hierarchy(d, N0, levels)
    A = [precond.abar(m, nu).toarray() for m in ms]
    Ps = [precond.prolongation(ms[l - 1], ms[l]).toarray() for l in range(1, levels)]
    for l in range(1, levels):
        G = Ps[l - 1].T @ A[l] @ Ps[l - 1]
        assert np.abs(G - A[l - 1]).max() <= 1e-13 * np.abs(A[l - 1]).max()
    Pall = np.eye(A[0].shape[0])
    for P in Ps:
        Pall = P @ Pall
    G = Pall.T @ A[-1] @ Pall
    assert np.abs(G - A[0]).max() <= 1e-13 * np.abs(A[0]).max()


def _vcycle_matrix(g: precond.GMG) -> np.ndarray:
    n = g.A[-1].shape[0]
    B = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        B[:, j] = g.vcycle(e)
    return B


VCYCLE_CASES = [(2, 8, 3), (2, 16, 4), (3, 4, 2), (3, 8, 3)]   # (dim, N, levels)


@pytest.mark.parametrize("d,N,levels", VCYCLE_CASES)
def test_vcycle_symmetric_and_bounded_by_abar(d, N, levels, nu=2.5):
    """C^{-1} = B symmetric positive definite with lambda(B Abar) in (0, 1] (Abar <= C)."""
    g = precond.GMG(d, N, levels, nu)
    B = _vcycle_matrix(g)
    A = g.A[-1].toarray()
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    # eigenvalues of B A = those of the symmetric A^{1/2} B A^{1/2}
    ev = np.linalg.eigvals(B @ A)
    assert np.abs(ev.imag).max() <= 1e-10
    ev = ev.real
    assert ev.min() > 1e-6 and ev.max() <= 1 + 1e-10, (ev.min(), ev.max())


# ------------------------------------------------------------------ planted mistakes (oracle, CPU)
def _wrong_weight(P):
    P = P.copy()
    P.data[np.isclose(P.data, 0.5)] = 1.0     # edge midpoint weight 1 instead of 1/2
    return P


def _shifted_vertex(P, d):
    P = P.tocoo()
    col = (P.col + d) % P.shape[1]           # every coarse vertex read one rank too far
    import scipy.sparse as sp
    return sp.csr_matrix((P.data, (P.row, col)), shape=P.shape)


@pytest.mark.parametrize("mistake", ["weight", "index"])
def test_prolongation_pins_catch(monkeypatch, mistake):
    orig = precond.prolongation
    d, N0 = 2, 4
    bad = (lambda c, f: _wrong_weight(orig(c, f))) if mistake == "weight" else \
        (lambda c, f: _shifted_vertex(orig(c, f), d))
    monkeypatch.setattr(precond, "prolongation", bad)
    ms = _hierarchy(d, N0, 2)
    P = precond.prolongation(ms[0], ms[1])
    _, nc = precond.p1_map(ms[0])
    c = np.random.default_rng(1).standard_normal(nc * d)
    ref = _interp_by_location(ms[0], ms[1], c)
    assert np.abs(P @ c - ref).max() > 1e-3 * np.abs(ref).max()
    A0, A1 = precond.abar(ms[0], 1.0).toarray(), precond.abar(ms[1], 1.0).toarray()
    assert np.abs(P.T @ A1 @ P - A0).max() > 1e-3 * np.abs(A0).max()


class _NoPostSmoothing(precond.GMG):
    """Planted mistake: the last post-smoothing sweep dropped."""

    def vcycle(self, b, l=None):
        l = len(self.A) - 1 if l is None else l
        if l == 0:
            return self.coarse @ b
        A, D = self.A[l], self.Dl1[l]
        x = np.zeros_like(b)
        for _ in range(self.smooth):
            x = x + (b - A @ x) / D
        x = x + self.P[l] @ self.vcycle(self.P[l].T @ (b - A @ x), l - 1)
        for _ in range(self.smooth - 1):
            x = x + (b - A @ x) / D
        return x


def test_dropped_post_sweep_is_caught():
    g = _NoPostSmoothing(2, 8, 3, 1.0)
    B = _vcycle_matrix(g)
    assert np.abs(B - B.T).max() > 1e-3 * np.abs(B).max()


def test_plain_jacobi_diagonal_is_caught():
    """With D = diag(A) instead of the l1 row sums the undamped sweeps overshoot: lambda(B Abar) > 1."""
    g = precond.GMG(2, 8, 3, 1.0)
    g.Dl1 = [A.diagonal().copy() for A in g.A]
    ev = np.linalg.eigvals(_vcycle_matrix(g) @ g.A[-1].toarray()).real
    assert ev.max() > 1 + 1e-3 or ev.min() <= 0
