"""Oracle pins for the outflow boundary Gamma_Ntilde (eq. stokes_NT, Lemma outflow): on x_1 = 1,
u_t = 0 (uhat = 0, no uhat dofs) and ((sigma + p I) n).n = 0 (natural), u_n free (BDM dofs kept)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fem, krylov, manufactured, mesh, precond, system


def _disc(d, N, k, nu=1.0):
    m = mesh.with_outflow(mesh.structured(d, N))
    return system.discretize(m, k, nu)


def test_outflow_dofs_and_nonsingular_system():
    """BDM moments on interior and outflow facets, uhat on interior facets only; with Gamma_Ntilde of
    positive measure the pressure has no constant mode, so K is nonsingular."""
    d, N, k = 2, 3, 2
    D = _disc(d, N, k)
    m = D.mesh
    n_out = int(m.outflow.sum())
    assert n_out == N
    assert D.n_dd == (m.n_int + n_out) * D.sz["nF"] and D.n_hat == m.n_int * D.sz["n_hatF"]
    K = system.condensed_system(D, system.condense(D)).toarray()
    sv = np.linalg.svd(K, compute_uv=False)
    assert sv[-1] > 1e-8 * sv[0]
    Dd = system.discretize(mesh.structured(d, N), k, 1.0)            # all Dirichlet: singular
    sv = np.linalg.svd(system.condensed_system(Dd, system.condense(Dd)).toarray(), compute_uv=False)
    assert sv[-1] < 1e-12 * sv[0]


@pytest.mark.parametrize("k", [2, 3])
def test_outflow_manufactured_convergence(k):
    """Optimal orders with the outflow condition, the pressure determined without a mean constraint:
    L2(u) ~ h^{k+1}, L2(p) ~ h^k (parity unpinned by the paper, which prints no rates); a wrong sign
    or a dropped boundary term in the natural condition would stall the pressure."""
    res = []
    for N in (4, 8):
        D = _disc(2, N, k)
        m = D.mesh
        ms = manufactured.ManufacturedOutflow(1.0)
        x = system.solve_condensed(D, system.load(D, ms.f))
        X = m.coords[m.elems]
        Dd = fem.element_data(X, m.signs, k, q=k + 4)
        xu = np.where(D.u_map >= 0, x[np.maximum(D.u_map, 0)], 0.0)
        uh = np.einsum("eqia,ei->eqa", Dd.U, xu)
        ph = np.einsum("eqi,ei->eq", Dd.P, x[D.p_map])
        res.append((np.sqrt(np.sum(Dd.wq * np.sum((uh - ms.u(Dd.xq)) ** 2, -1))),
                    np.sqrt(np.sum(Dd.wq * (ph - ms.p(Dd.xq)) ** 2))))
        assert np.abs(np.einsum("eqi,ei->eq", Dd.divU, xu)).max() < 1e-9
    assert np.log2(res[0][0] / res[1][0]) > k + 1 - 0.3
    assert np.log2(res[0][1] / res[1][1]) > k - 0.2


def _embedding_pencil(d, N, k, C):
    D = _disc(d, N, k)
    A = system.condensed_system(D, system.condense(D))
    E = precond.embedding(D)
    Ab = precond.abar(D.mesh, 1.0, k, C).toarray()
    return sla.eigh((E.T @ A @ E).toarray(), Ab, eigvals_only=True)


def test_lemma_outflow_penalty():
    """Lemma outflow: with the tangential penalty nu C k^2/h on Gamma_Ntilde and pi_0 (no uhat there),
    |pi_0 E ubar|_A ~ |ubar|_Abar uniformly in h (C = OUTFLOW_C, reading R23); without the penalty
    the upper constant grows like 1/h."""
    for d, N, k in [(2, 4, 2), (2, 8, 2), (2, 4, 3), (3, 2, 2)]:
        ev = _embedding_pencil(d, N, k, precond.OUTFLOW_C)
        assert 0.3 < ev.min() and ev.max() < 1.05
    e4 = _embedding_pencil(2, 4, 2, 0.0).max()
    e8 = _embedding_pencil(2, 8, 2, 0.0).max()
    assert e4 > 5.0 and e8 > 2.0 * e4


def test_minres_with_outflow_asp():
    """MinRes with Khat^{-1} (ASP: facet blocks with uhat only on interior facets, E with pi_0, GMG on
    the penalised Abar with free vertices on Gamma_Ntilde) reaches the direct solution; the
    iteration count stays bounded under refinement."""
    its = []
    for N, lev in [(4, 2), (8, 3)]:
        D = _disc(2, N, 2)
        AT = system.condense(D)
        A = system.condensed_system(D, AT)
        g = precond.GMG(2, N, lev, 1.0, outflow_k=2)
        bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, g))
        F = system.load(D, manufactured.ManufacturedOutflow(1.0).f)
        x, it, _ = krylov.minres(lambda v: A @ v, bp.apply, F, rtol=1e-10, maxit=500)
        xd = system.solve_condensed(D, F, AT)
        assert np.abs(x - xd).max() < 1e-7 * np.abs(xd).max()
        its.append(it)
    assert its[1] < 1.5 * its[0]
