"""Oracle pins for the ASP on the full velocity block (Theorem aux_pc) against the condensed route."""
import numpy as np
import pytest

from oracle import krylov, manufactured, mesh, precond, system


def _setup(d, N, k, lev, nu=1.0):
    D = system.discretize(mesh.structured(d, N), k, nu)
    AT = system.condense(D)
    return D, AT, precond.GMG(d, N, lev, nu)


@pytest.mark.parametrize("d,N,k,lev", [(2, 4, 2, 2), (3, 2, 2, 1), (2, 2, 3, 1)])
def test_multiplicative_full_equals_condensed(d, N, k, lev):
    """Colour-ordered block Gauss-Seidel on the full block with one block per facet plus its two
    elements' bubbles is the condensed multiplicative ASP wrapped by eq. (factorSsigma): a block solve
    eliminates the bubbles exactly (its facet part is the D_F of A^d), and after a complete sweep
    every element's bubbles were last solved with its last-coloured facet, so the coarse residual
    E^T (b - A x) equals E^d^T (r_d - A^d x_d) and the output bubbles are the harmonic extension."""
    D, AT, g = _setup(d, N, k, lev, nu=0.6)
    r = np.random.default_rng(1).standard_normal(D.ndof)
    za = precond.ASP(D, AT, g).apply(r)
    zb = precond.FullASP(D, AT, g).apply(r)
    assert np.abs(za - zb).max() < 1e-11 * np.abs(za).max()


def test_additive_full_is_a_different_spd_preconditioner():
    """Theorem aux_pc: M^{-1} + E C^{-1} E^T (overlapping facet blocks) is SPD and spectrally
    equivalent to A; it is not the condensed additive ASP."""
    D, AT, g = _setup(2, 4, 2, 1)
    full = precond.FullASP(D, AT, g, multiplicative=False)
    vel = np.arange(D.off_p)
    A = system.condensed_system(D, AT)[:D.off_p][:, :D.off_p].toarray()
    P = np.zeros((len(vel), len(vel)))
    for j in vel:
        e = np.zeros(D.ndof)
        e[j] = 1.0
        P[:, j] = full.apply(e)[vel]
    assert np.abs(P - P.T).max() < 1e-12 * np.abs(P).max()
    ev = np.sort(np.linalg.eigvals(P @ A).real)
    assert ev[0] > 0.01 and ev[-1] < 10.0
    r = np.random.default_rng(2).standard_normal(D.ndof)
    cond = precond.ASP(D, AT, g, multiplicative=False).apply(r)[vel]
    assert np.abs(P @ r[vel] - cond).max() > 1e-6 * np.abs(cond).max()


def test_minres_with_full_asp():
    D, AT, g = _setup(3, 2, 2, 1)
    A = system.condensed_system(D, AT)
    F = system.load(D, manufactured.Manufactured(3, 1.0).f)
    proj = lambda v: system.mean_zero_pressure(D, v)
    xd = system.mean_zero_pressure(D, system.solve_condensed(D, F, AT))
    its = {}
    for mult in (True, False):
        bp = precond.BlockPreconditioner(D, precond.FullASP(D, AT, g, multiplicative=mult))
        x, it, _ = krylov.minres(lambda v: A @ v, bp.apply, F, rtol=1e-10, maxit=600, project=proj)
        assert np.abs(proj(x) - xd).max() < 1e-7 * np.abs(xd).max()
        its[mult] = it
    assert its[True] < its[False]
