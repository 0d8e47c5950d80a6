"""Oracle pins: identities the paper proves (Lemma SPD, Corollary embed, eq. factorSsigma, ...)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fem, manufactured, mesh, precond, system

CASES = [(2, 2, 4), (2, 3, 2), (3, 2, 2)]


def _disc(d, k, N, nu=0.7):
    m = mesh.structured(d, N)
    D = system.discretize(m, k, nu)
    return D, system.condense(D)


@pytest.mark.parametrize("d,k,N", CASES)
def test_embedding_energy_identity(d, k, N):
    """Corollary embed with eq. (schur_SPD_cont): E^T A E = Abar = nu (eps, eps) (reading R1)."""
    D, AT = _disc(d, k, N)
    A = system.condensed_system(D, AT)
    E = precond.embedding(D)
    Ab = precond.abar(D.mesh, D.nu).toarray()
    assert np.abs((E.T @ A @ E).toarray() - Ab).max() < 1e-12 * np.abs(Ab).max()


@pytest.mark.parametrize("d,k,N", CASES)
def test_energy_identity_and_spd(d, k, N):
    """eq. (schurnormmat): |(u,uhat)|_A^2 = nu^{-1}|sigma|^2 + nu/d |div u|^2; Lemma SPD: A > 0."""
    D, AT = _disc(d, k, N)
    A = system.condensed_system(D, AT)
    n = D.off_p
    rng = np.random.default_rng(3)
    for _ in range(3):
        x = np.zeros(D.ndof)
        x[:n] = rng.standard_normal(n)
        sig, _ = system.recover_stress(D, x)
        sig_sq = np.einsum("ei,eij,ej->", sig, D.mats["M"], sig)      # nu^{-1} |sigma|^2
        xu = np.where(D.u_map >= 0, x[np.maximum(D.u_map, 0)], 0.0)
        div_sq = np.einsum("ei,eij,ej->", xu, D.mats["Adiv"], xu)     # nu/d |div u|^2
        lhs = x @ (A @ x)
        assert abs(lhs - sig_sq - div_sq) < 1e-11 * lhs
    ev = np.linalg.eigvalsh(A[:n, :n].toarray())
    assert ev.min() > 1e-10 * ev.max()


@pytest.mark.parametrize("d,k,N", CASES)
def test_conforming_stress_recovery(d, k, N):
    """Lemma SPD proof: for conforming E ubar, sigma_h = -nu dev eps(ubar), omega_h = kappa(curl ubar)."""
    D, AT = _disc(d, k, N)
    m = D.mesh
    E = precond.embedding(D)
    rng = np.random.default_rng(5)
    ub = rng.standard_normal(E.shape[1])
    x = E @ ub
    sig, om = system.recover_stress(D, x)
    X = m.coords[m.elems]
    data = fem.element_data(X, m.signs, k)
    S = np.einsum("eqsab,es->eqab", data.S, sig)
    W = np.einsum("eqsab,es->eqab", data.W, om)
    # gradient of the P1 field per element
    rank, _ = precond.p1_map(m)
    vals = np.zeros((len(m.elems), d + 1, d))
    for v in range(d + 1):
        r = rank[m.elems[:, v]]
        ok = r >= 0
        vals[ok, v, :] = ub.reshape(-1, d)[r[ok]]
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
    Du = np.einsum("eca,eab->ecb", np.transpose(vals[:, 1:, :] - vals[:, :1, :], (0, 2, 1)), np.linalg.inv(J))
    eps = 0.5 * (Du + np.transpose(Du, (0, 2, 1)))
    dev = eps - np.einsum("eaa->e", eps)[:, None, None] / d * np.eye(d)
    skw = 0.5 * (Du - np.transpose(Du, (0, 2, 1)))
    assert np.abs(S + D.nu * dev[:, None]).max() < 1e-10 * np.abs(D.nu * dev).max()
    assert np.abs(W - skw[:, None]).max() < 1e-10 * np.abs(skw).max()
    if d == 2:   # kappa(curl u), curl u = -d2 u1 + d1 u2
        curl = -Du[:, 0, 1] + Du[:, 1, 0]
        kap = 0.5 * np.stack([np.stack([0 * curl, -curl], -1), np.stack([curl, 0 * curl], -1)], -2)
        assert np.abs(skw - kap).max() < 1e-12 * np.abs(kap).max()


@pytest.mark.parametrize("d,k,N", CASES)
def test_bubble_factorization(d, k, N):
    """eq. (factorSsigma): A_T = L diag(A^d, A_oo) L^T exactly, element by element."""
    D, AT = _disc(d, k, N)
    Ad, G, Aoo = system.bubble_condense(D, AT)
    o, c = system.local_split(D)
    perm = np.concatenate([c, o])
    Ap = AT[:, perm][:, :, perm]
    nc, no = len(c), len(o)
    for e in range(len(AT)):
        L = np.eye(nc + no)
        L[:nc, nc:] = G[e].T       # A_do A_oo^{-1} = G^T
        Dm = sla.block_diag(Ad[e], Aoo[e])
        assert np.abs(L @ Dm @ L.T - Ap[e]).max() < 1e-11 * np.abs(Ap[e]).max()


@pytest.mark.parametrize("d,k,N", CASES)
def test_condensed_embedding_bound(d, k, N):
    """Corollary embed_schur: E^d^T A^d E^d <= Abar (harmonic extension minimises energy)."""
    D, AT = _disc(d, k, N)
    asp = precond.ASP(D, AT, precond.GMG(d, N, 1, D.nu))
    Ed = asp.Ed.toarray()
    lhs = Ed.T @ asp.Ad_glob.toarray() @ Ed
    Ab = precond.abar(D.mesh, D.nu).toarray()
    ev = sla.eigh(lhs, Ab, eigvals_only=True)
    assert ev.max() <= 1 + 1e-10


def test_multiplicative_asp_bounds():
    """Corollary aux_pc_mult: with C = Abar and block Gauss-Seidel, A^d <= Ahat^d_m (eigs of Ahat_m^{-1} A^d in (0, 1])."""
    D, AT = _disc(2, 2, 4)
    asp = precond.ASP(D, AT, precond.GMG(2, 4, 1, D.nu))
    cd = np.concatenate([np.arange(D.n_dd), D.off_h + np.arange(D.n_hat)])
    n = D.ndof
    P = np.zeros((len(cd), len(cd)))
    for j, g in enumerate(cd):
        e = np.zeros(n)
        e[g] = 1.0
        P[:, j] = asp.apply_ad(e)[cd]
    Ad = asp.Ad_glob.toarray()[np.ix_(cd, cd)]
    assert np.abs(P - P.T).max() < 1e-10 * np.abs(P).max()
    ev = np.linalg.eigvals(P @ Ad).real
    assert ev.min() > 0 and ev.max() <= 1 + 1e-10


def test_block_preconditioner_two_applications():
    """eq. (mhatinvfactor): the 2-application form equals the dense triple product; it is SPD."""
    D, AT = _disc(2, 2, 2)
    bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, precond.GMG(2, 2, 1, D.nu)))
    P = bp.dense()
    rng = np.random.default_rng(0)
    for _ in range(3):
        z = rng.standard_normal(D.ndof)
        assert np.abs(P @ z - bp.apply(z)).max() < 1e-12 * np.abs(P @ z).max()
    assert np.abs(P - P.T).max() < 1e-12 * np.abs(P).max()
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0


def test_nu_scaling_exact():
    """A(nu) = nu A(1) element by element; u_h(nu) = u_h(1)/nu, p_h(nu) = p_h(1) (reading P8)."""
    m = mesh.structured(2, 4)
    D1 = system.discretize(m, 2, 1.0)
    D2 = system.discretize(m, 2, 0.01)
    A1, A2 = system.condense(D1), system.condense(D2)
    assert np.abs(A2 - 0.01 * A1).max() < 1e-13 * np.abs(0.01 * A1).max()
    ms = manufactured.Manufactured(2, 1.0)
    F = system.load(D1, ms.f)
    x1 = system.mean_zero_pressure(D1, system.solve_condensed(D1, F, A1))
    x2 = system.mean_zero_pressure(D2, system.solve_condensed(D2, F, A2))
    n = D1.off_p
    assert np.abs(x2[:n] - x1[:n] / 0.01).max() < 1e-9 * np.abs(x1[:n] / 0.01).max()
    assert np.abs(x2[n:] - x1[n:]).max() < 1e-9 * np.abs(x1[n:]).max()
