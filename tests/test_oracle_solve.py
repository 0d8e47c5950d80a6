"""Oracle pins: the discrete solution (div-free, pressure robust, convergent, condensed = uncondensed)."""
import numpy as np
import pytest

from oracle import fem, krylov, manufactured, mesh, polys, precond, system


def _errors(D, x, ms):
    m = D.mesh
    X = m.coords[m.elems]
    Dd = fem.element_data(X, m.signs, D.k, q=D.k + 4)
    xu = np.where(D.u_map >= 0, x[np.maximum(D.u_map, 0)], 0.0)
    uh = np.einsum("eqia,ei->eqa", Dd.U, xu)
    ph = np.einsum("eqi,ei->eq", Dd.P, x[D.p_map])
    eu = np.sqrt(np.sum(Dd.wq * np.sum((uh - ms.u(Dd.xq)) ** 2, -1)))
    ep = np.sqrt(np.sum(Dd.wq * (ph - ms.p(Dd.xq)) ** 2))
    div = np.abs(np.einsum("eqi,ei->eq", Dd.divU, xu)).max()
    return eu, ep, div


@pytest.mark.parametrize("k", [2, 3])
def test_manufactured_convergence_2d(k):
    """Best-approximation orders of the spaces (parity unpinned by the paper, which prints no rates):
    L2 velocity ~ h^{k+1}, L2 pressure ~ h^k; div u_h = 0 pointwise (div V_h = Q_h)."""
    res = []
    for N in (2, 4, 8):
        m = mesh.structured(2, N)
        D = system.discretize(m, k, 1.0)
        ms = manufactured.Manufactured(2, 1.0)
        F = system.load(D, ms.f)
        x, _, _ = system.solve_full(D, F)
        x = system.mean_zero_pressure(D, x)
        eu, ep, div = _errors(D, x, ms)
        assert div < 1e-10 * max(1.0, np.abs(x).max())
        res.append((eu, ep))
    ru = np.log2(res[1][0] / res[2][0])
    rp = np.log2(res[1][1] / res[2][1])
    assert ru > k + 1 - 0.3 and rp > k - 0.2


def test_condensed_equals_uncondensed():
    for d, k, N in [(2, 2, 1), (2, 2, 2), (2, 3, 2), (2, 2, 8), (3, 2, 1)]:
        m = mesh.structured(d, N)
        D = system.discretize(m, k, 1.0)
        ms = manufactured.Manufactured(d, 1.0)
        F = system.load(D, ms.f)
        x, _, _ = system.solve_full(D, F)
        xc = system.solve_condensed(D, F)
        x, xc = system.mean_zero_pressure(D, x), system.mean_zero_pressure(D, xc)
        assert np.abs(x - xc).max() < 1e-11 * np.abs(x).max()


def test_pressure_robustness():
    """f = grad(phi) gives u_h = 0 and p_h = Pi_Q phi - mean (exact closed form)."""
    m = mesh.structured(2, 4)
    k = 3
    D = system.discretize(m, k, 0.3)
    phi = lambda x: np.sin(2 * x[..., 0]) * x[..., 1] ** 2 + x[..., 0] * x[..., 1]
    gphi = lambda x: np.stack([2 * np.cos(2 * x[..., 0]) * x[..., 1] ** 2 + x[..., 1],
                               2 * np.sin(2 * x[..., 0]) * x[..., 1] + x[..., 0]], -1)
    F = system.load(D, gphi)
    x = system.mean_zero_pressure(D, system.solve_condensed(D, F))
    n = D.off_p
    assert np.abs(x[:n]).max() < 1e-10 * np.abs(x[n:]).max()
    X = m.coords[m.elems]
    Dd = fem.element_data(X, m.signs, k, q=k + 6)
    # the weak form has -(div v, p): f = grad phi balances p = phi up to the projection
    proj = np.einsum("eq,eq,eqi->ei", Dd.wq, phi(Dd.xq), Dd.P) / np.abs(Dd.detJ)[:, None]
    y = np.zeros(D.ndof)
    y[D.p_map] = proj
    y = system.mean_zero_pressure(D, y)
    assert np.abs(x[n:] - y[n:]).max() < 1e-10 * np.abs(y[n:]).max()
    # adding grad(phi) to a manufactured f leaves u_h unchanged
    ms = manufactured.Manufactured(2, 0.3)
    F0 = system.load(D, ms.f)
    x0 = system.solve_condensed(D, F0)
    x1 = system.solve_condensed(D, F0 + F)
    assert np.abs(x1[:n] - x0[:n]).max() < 1e-10 * np.abs(x0[:n]).max()


def test_minres_matches_direct_and_iterations_bounded():
    """Preconditioned MinRes reaches the direct solution; #IT stays bounded under refinement (qualitative)."""
    its = []
    for N, lev in [(4, 2), (8, 3), (16, 4)]:
        m = mesh.structured(2, N)
        D = system.discretize(m, 2, 1.0)
        AT = system.condense(D)
        A = system.condensed_system(D, AT)
        bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, precond.GMG(2, N, lev, 1.0)))
        ms = manufactured.Manufactured(2, 1.0)
        F = system.load(D, ms.f)
        proj = lambda v: system.mean_zero_pressure(D, v)
        x, it, _ = krylov.minres(lambda v: A @ v, bp.apply, F, rtol=1e-10, maxit=400, project=proj)
        xd = system.mean_zero_pressure(D, system.solve_condensed(D, F, AT))
        x = system.mean_zero_pressure(D, x)
        assert np.abs(x - xd).max() < 1e-7 * np.abs(xd).max()
        its.append(it)
    assert max(its) < 1.6 * min(its)
