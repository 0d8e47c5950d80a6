"""Oracle Krylov solvers: textbook properties of GMRES and MinRes against it on the MCS system."""
import numpy as np

from oracle import krylov, manufactured, mesh, precond, system


def test_gmres_finite_termination_and_monotone_residual():
    """Unrestarted GMRES on an n x n nonsymmetric matrix reaches the solution within n steps, and its
    residual norm never increases (it minimises over nested Krylov spaces)."""
    rng = np.random.default_rng(0)
    n = 30
    A = rng.standard_normal((n, n)) + 8.0 * np.eye(n)
    b = rng.standard_normal(n)
    x, it, hist = krylov.gmres(lambda v: A @ v, lambda v: v, b, rtol=1e-14, maxit=n)
    assert it <= n
    assert np.linalg.norm(A @ x - b) < 1e-12 * np.linalg.norm(b)
    assert np.all(np.diff(hist) <= 1e-12 * hist[0])
    # with the exact inverse as (right) preconditioner it converges in one step
    Ai = np.linalg.inv(A)
    x, it, _ = krylov.gmres(lambda v: A @ v, lambda v: Ai @ v, b, rtol=1e-12, maxit=5)
    assert it == 1 and np.linalg.norm(A @ x - b) < 1e-12 * np.linalg.norm(b)


def test_gmres_and_minres_with_the_block_preconditioner():
    """The paper's solver (GMRES, rel. residual 1e-6, Sec. 8) and MinRes reach the direct solution with
    similar iteration counts on the same preconditioner."""
    d, N, k, lev = 2, 8, 2, 3
    D = system.discretize(mesh.structured(d, N), k, 1.0)
    AT = system.condense(D)
    K = system.condensed_system(D, AT)
    bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, precond.GMG(d, N, lev, 1.0)))
    F = system.load(D, manufactured.Manufactured(d, 1.0).f)
    proj = lambda v: system.mean_zero_pressure(D, v)
    xd = system.mean_zero_pressure(D, system.solve_condensed(D, F, AT))
    xg, itg, _ = krylov.gmres(lambda v: K @ v, bp.apply, F, rtol=1e-10, maxit=200, project=proj)
    xm, itm, _ = krylov.minres(lambda v: K @ v, bp.apply, F, rtol=1e-10, maxit=200, project=proj)
    for x in (xg, xm):
        assert np.abs(proj(x) - xd).max() < 1e-7 * np.abs(xd).max()
    assert 0.7 * itm <= itg <= 1.3 * itm
