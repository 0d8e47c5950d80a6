"""The gamma experiment of Corollary schur_SPD on single elements (oracle only)."""
import numpy as np
import pytest

from oracle import hdg


@pytest.mark.parametrize("k", [2, 3])
def test_pencil_kernel_and_bounds(k):
    """Both forms vanish exactly on the 6 rigid-body motions; on the rest the pencil lies in
    [1/gamma, d + 2] (the provable form of eq. schur_SPD's upper bound, reading R22)."""
    g, lmax, gap = hdg.gamma(k)
    assert gap > 1e8
    assert 1.0 < g < 100.0 and 0.0 < lmax <= 5.0


def test_rigid_motions_in_both_kernels():
    AT, N, sz = hdg.element_forms(2)
    Ad, Nd = hdg.schur_on_coupling(AT, sz), hdg.schur_on_coupling(N, sz)
    w, V = np.linalg.eigh(0.5 * (Nd + Nd.T))
    ker = V[:, :6]
    assert w[5] < 1e-10 * w[-1] < w[6]
    assert np.abs(Ad @ ker).max() < 1e-10 * np.abs(Ad).max()


def test_gamma_is_invariant_under_similarity_and_nu():
    """Both forms scale like h^{d-2} under x -> c Q x + b and like nu, so gamma does not change."""
    X0 = hdg.unit_tetrahedron()
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    X1 = 0.37 * X0 @ Q.T + np.array([0.2, -1.0, 0.5])
    g0, l0, _ = hdg.gamma(2)
    g1, l1, _ = hdg.gamma(2, nu=0.3, X=X1)
    assert abs(g1 - g0) < 1e-7 * g0 and abs(l1 - l0) < 1e-7 * l0


def test_gamma_depends_on_shape():
    """A flattened element has a larger constant than the unit tetrahedron (shape regularity enters)."""
    X = hdg.unit_tetrahedron().copy()
    X[0, 3, 2] = 0.2
    assert hdg.gamma(2, X=X)[0] > hdg.gamma(2)[0]


def test_bubble_basis_does_not_change_gamma():
    """The infimum over the bubbles (eq. epshschur) and the double Schur complement are independent of
    the bubble basis: the contract's L2-orthonormal bubbles and the unorthonormalised monomial list
    give the same pencil."""
    a = hdg.gamma(3, bubble_basis="monomial")
    b = hdg.gamma(3)
    assert abs(a[0] - b[0]) < 1e-8 * a[0] and abs(a[1] - b[1]) < 1e-8 * a[1]
    assert b[2] > a[2]                       # the orthonormal basis resolves the kernel better
