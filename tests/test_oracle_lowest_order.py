"""Oracle pins for the lowest-order variant (k = 1, Sec. 7; three dimensions).

The variant keeps the MCS forms but takes the rotation in H(div): W_h = P^0(T, R^3) + x P^0(T)
with one normal-flux dof per facet, writes kappa(omega) wherever omega occurs, adds the consistent
term (div omega, div eta) (coefficient nu, reading R21) and embeds the conforming space by
E ubar = (ubar, Pi^0 (ubar)_t, curl ubar).  The pins below follow from that text and from the
mathematics: the per-facet dof counts the section names, the energy identity of the embedding
(for P^1 fields sigma_h = -nu dev eps(ubar) exactly), the Korn-type SPD property, the
condensation, pressure robustness and convergence.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fem, krylov, manufactured, mesh, precond, system

NU = 0.7


def _disc(N, nu=NU):
    m = mesh.structured(3, N)
    D = system.discretize(m, 1, nu)
    return D, system.condense(D)


def test_local_dimensions():
    """Sec. 7: BDM^1 has three and Vhat_h two coupling dofs per facet, W_h one more; Sigma_h(T) is
    P^1 trace-free with P^0 nt-trace (32 - 16 = 16 functions); Q_h = P^0; no velocity bubbles."""
    sz = fem.local_sizes(3, 1)
    assert (sz["nF"], sz["n_tF"], sz["n_hatF"] - sz["n_tF"]) == (3, 2, 1)
    assert (sz["n_sigma"], sz["n_bub"], sz["n_p"], sz["n_omega"]) == (16, 0, 1, 0)
    assert sz["n_A"] == 4 * (3 + 3)
    with pytest.raises(ValueError):
        fem.local_sizes(2, 1)


def test_rotation_space_fluxes_and_divergence():
    """The rotation function of local facet f has flux s_{T,f} through F_f and none through the other
    facets (checked through the facet normal of the recovered vector field), and constant divergence
    s_{T,f}/|T| (Gauss); the stabilisation block is then nu s_f s_g / |T|."""
    m = mesh.structured(3, 2)
    X = m.coords[m.elems]
    Dd = fem.element_data(X, m.signs, 1)
    mats = fem.element_matrices(X, m.signs, 1, NU)
    vol = np.abs(Dd.detJ) / 6.0
    # recover the vector field from kappa (entries (2,1), (0,2), (1,0) carry v/2)
    W = Dd.W
    v = 2.0 * np.stack([W[..., 2, 1], W[..., 0, 2], W[..., 1, 0]], axis=-1)      # [E, nq, 4, 3]
    # the field is affine: v(x) = v(x0) + slope (x - x0); its flux through F_g = |F_g| v(centroid).n
    for e in range(0, X.shape[0], 7):
        xq, vq = Dd.xq[e], v[e]
        A = np.hstack([np.ones((len(xq), 1)), xq])
        coef, *_ = np.linalg.lstsq(A, vq.reshape(len(xq), -1), rcond=None)
        for f in range(4):
            for g in range(4):
                lv = [w for w in range(4) if w != g]
                c = X[e, lv].mean(axis=0)
                vc = (np.concatenate([[1.0], c]) @ coef).reshape(4, 3)[f]
                area = 0.5 * np.linalg.norm(np.cross(X[e, lv[1]] - X[e, lv[0]], X[e, lv[2]] - X[e, lv[0]]))
                flux = area * vc @ Dd.fn[e, g]
                assert abs(flux - (m.signs[e, f] if f == g else 0.0)) < 1e-12
        assert np.allclose(Dd.divW[e], m.signs[e][None, :] / vol[e], rtol=1e-13)
    rows = [2, 5, 8, 11]
    S = mats["Shat"][:, rows][:, :, rows]
    ref = NU * np.einsum("ef,eg->efg", m.signs, m.signs) / vol[:, None, None]
    assert np.abs(S - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("N", [2, 3])
def test_embedding_energy_identity(N):
    """E = (ubar, Pi^0 ubar_t, curl ubar): for P^1 fields the local problem gives sigma = -nu dev eps,
    so E^T A E = Abar = nu (eps, eps) exactly; a wrong sign or scale of the rotation coupling,
    of kappa or of the curl rows breaks it."""
    D, AT = _disc(N)
    A = system.condensed_system(D, AT)
    E = precond.embedding(D)
    Ab = precond.abar(D.mesh, D.nu).toarray()
    assert np.abs((E.T @ A @ E).toarray() - Ab).max() < 1e-12 * np.abs(Ab).max()


def test_conforming_stress_recovery():
    """For x = E ubar the element stresses are -nu dev eps(ubar) (constant per element)."""
    D, AT = _disc(3)
    m = D.mesh
    E = precond.embedding(D)
    ub = np.random.default_rng(5).standard_normal(E.shape[1])
    sig, om = system.recover_stress(D, E @ ub)
    assert om.shape[1] == 0
    X = m.coords[m.elems]
    data = fem.element_data(X, m.signs, 1)
    S = np.einsum("eqsab,es->eqab", data.S, sig)
    # gradient of the P^1 field per element from its vertex values
    rank, _ = precond.p1_map(m)
    vals = np.zeros((m.coords.shape[0], 3))
    iv = rank >= 0
    vals[iv] = ub.reshape(-1, 3)[rank[iv]]
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
    dU = vals[m.elems[:, 1:]] - vals[m.elems[:, :1]]                  # [E, 3 edges, 3 comps]
    Du = np.einsum("eia,eib->eab", dU, np.linalg.inv(J))              # Du[a, b] = d u_a / d x_b
    eps = 0.5 * (Du + np.transpose(Du, (0, 2, 1)))
    dev = eps - np.einsum("eaa->e", eps)[:, None, None] * np.eye(3) / 3.0
    assert np.abs(S - (-D.nu * dev)[:, None]).max() < 1e-11 * np.abs(D.nu * dev).max()


def test_energy_identity_and_spd():
    """|(u, uhat, omega)|_A^2 = nu^{-1}|sigma|^2 + nu/d |div u|^2 + nu |div omega|^2; A > 0 (Korn)."""
    D, AT = _disc(2)
    A = system.condensed_system(D, AT)
    n = D.off_p
    rng = np.random.default_rng(3)
    hm = D.h_map
    for _ in range(3):
        x = np.zeros(D.ndof)
        x[:n] = rng.standard_normal(n)
        sig, _ = system.recover_stress(D, x)
        sig_sq = np.einsum("ei,eij,ej->", sig, D.mats["M"], sig)
        xu = np.where(D.u_map >= 0, x[np.maximum(D.u_map, 0)], 0.0)
        div_sq = np.einsum("ei,eij,ej->", xu, D.mats["Adiv"], xu)
        xw = np.where(hm[:, 2::3] >= 0, x[np.maximum(hm[:, 2::3], 0)], 0.0)   # [E, 4] fluxes
        vol = np.abs(np.linalg.det(np.transpose(
            D.mesh.coords[D.mesh.elems][:, 1:] - D.mesh.coords[D.mesh.elems][:, :1], (0, 2, 1)))) / 6.0
        divw = np.einsum("ef,ef->e", D.mesh.signs, xw) / vol                # div omega_h per element
        stab = D.nu * np.sum(divw ** 2 * vol)
        lhs = x @ (A @ x)
        assert abs(lhs - sig_sq - div_sq - stab) < 1e-11 * lhs
    ev = np.linalg.eigvalsh(A[:n, :n].toarray())
    assert ev.min() > 1e-8 * ev.max()


def test_condensed_equals_uncondensed():
    for N in (1, 2):
        D, AT = _disc(N, 1.0)
        ms = manufactured.Manufactured(3, 1.0)
        F = system.load(D, ms.f)
        x, _, _ = system.solve_full(D, F)
        xc = system.solve_condensed(D, F, AT)
        x, xc = system.mean_zero_pressure(D, x), system.mean_zero_pressure(D, xc)
        assert np.abs(x - xc).max() < 1e-11 * np.abs(x).max()


def test_pressure_robustness():
    """f = grad(phi) gives u_h = 0, uhat_h = 0, omega_h = 0 (div V_h = Q_h, exact)."""
    D, AT = _disc(2, 0.3)
    gphi = lambda x: np.stack([x[..., 1] * x[..., 2], x[..., 0] * x[..., 2] + 2 * x[..., 1],
                               x[..., 0] * x[..., 1]], -1)
    x = system.mean_zero_pressure(D, system.solve_condensed(D, system.load(D, gphi), AT))
    n = D.off_p
    assert np.abs(x[:n]).max() < 1e-10 * np.abs(x[n:]).max()


def test_manufactured_convergence():
    """u_h converges (L2, first order at least: BDM^1 approximates to second order, the scheme is
    stable by the section's Korn inequality); div u_h = 0 pointwise.  Parity unpinned by the paper,
    which prints no rates."""
    errs = []
    for N in (2, 4):
        D, AT = _disc(N, 1.0)
        ms = manufactured.Manufactured(3, 1.0)
        x = system.mean_zero_pressure(D, system.solve_condensed(D, system.load(D, ms.f), AT))
        m = D.mesh
        X = m.coords[m.elems]
        Dd = fem.element_data(X, m.signs, 1, q=5)
        xu = np.where(D.u_map >= 0, x[np.maximum(D.u_map, 0)], 0.0)
        uh = np.einsum("eqia,ei->eqa", Dd.U, xu)
        errs.append(np.sqrt(np.sum(Dd.wq * np.sum((uh - ms.u(Dd.xq)) ** 2, -1))))
        assert np.abs(np.einsum("eqi,ei->eq", Dd.divU, xu)).max() < 1e-10 * max(1.0, np.abs(x).max())
    assert math.log2(errs[0] / errs[1]) > 1.0


def test_minres_with_asp_matches_direct():
    """MinRes with the block preconditioner (facet blocks of 6 incl. the rotation flux, E with the
    curl rows, GMG for Abar) reaches the direct solution; E^d^T A^d E^d <= Abar.  With the
    stabilisation weight nu (reading R21) the ASP condition number grows under refinement
    (exact C: about 77, 222, 393 for N = 2, 3, 4), so no iteration bound is pinned."""
    for N, lev in [(2, 1), (3, 1)]:
        D, AT = _disc(N, 1.0)
        A = system.condensed_system(D, AT)
        asp = precond.ASP(D, AT, precond.GMG(3, N, lev, 1.0))
        Ed = asp.Ed.toarray()
        Ab = precond.abar(D.mesh, 1.0).toarray()
        assert sla.eigh(Ed.T @ asp.Ad_glob.toarray() @ Ed, Ab, eigvals_only=True).max() <= 1 + 1e-10
        bp = precond.BlockPreconditioner(D, asp)
        F = system.load(D, manufactured.Manufactured(3, 1.0).f)
        proj = lambda v: system.mean_zero_pressure(D, v)
        x, it, _ = krylov.minres(lambda v: A @ v, bp.apply, F, rtol=1e-10, maxit=1000, project=proj)
        xd = system.mean_zero_pressure(D, system.solve_condensed(D, F, AT))
        assert it < 1000 and np.abs(proj(x) - xd).max() < 1e-7 * np.abs(xd).max()


def _identity_defect(N=2):
    D, AT = _disc(N)
    A = system.condensed_system(D, AT)
    E = precond.embedding(D)
    Ab = precond.abar(D.mesh, D.nu).toarray()
    return np.abs((E.T @ A @ E).toarray() - Ab).max() / np.abs(Ab).max()


@pytest.mark.parametrize("scale", [-1.0, 2.0, 0.5])
def test_rotation_coupling_mistakes_are_caught(monkeypatch, scale):
    """A flipped sign of the kappa(omega) coupling, or a dropped / doubled 1/2 of kappa, breaks the
    energy identity of the embedding."""
    orig = fem.element_matrices

    def bad(X, signs, k, nu, *rest):
        out = orig(X, signs, k, nu, *rest)
        out["Bh"][:, 2::3, :] *= scale
        return out
    monkeypatch.setattr(fem, "element_matrices", bad)
    assert _identity_defect() > 1e-6


def test_curl_row_sign_is_caught(monkeypatch):
    orig = precond.embedding

    def bad(D):
        E = orig(D).tolil()
        rows = D.off_h + np.arange(D.mesh.n_int) * 3 + 2
        E[rows] = -E[rows]
        return E.tocsr()
    monkeypatch.setattr(precond, "embedding", bad)
    assert _identity_defect() > 1e-6


def test_dropped_stabilisation_is_caught(monkeypatch):
    """Without nu (div omega, div eta) the energy split of test_energy_identity_and_spd fails."""
    orig = fem.element_matrices

    def bad(X, signs, k, nu, *rest):
        out = orig(X, signs, k, nu, *rest)
        out["Shat"] = np.zeros_like(out["Shat"])
        return out
    monkeypatch.setattr(fem, "element_matrices", bad)
    with pytest.raises(AssertionError):
        test_energy_identity_and_spd()


def _asp_condition(N, lo_stab):
    D = system.discretize(mesh.structured(3, N), 1, 1.0, lo_stab=lo_stab)
    AT = system.condense(D)
    asp = precond.ASP(D, AT, precond.GMG(3, N, 1, 1.0))
    cd = np.concatenate([np.arange(D.n_dd), D.off_h + np.arange(D.n_hat)])
    P = np.zeros((len(cd), len(cd)))
    for j, g in enumerate(cd):
        e = np.zeros(D.ndof)
        e[g] = 1.0
        P[:, j] = asp.apply_ad(e)[cd]
    ev = np.sort(np.linalg.eigvals(P @ asp.Ad_glob.toarray()[np.ix_(cd, cd)]).real)
    return ev[-1] / ev[0]


def test_stabilisation_weight_and_conditioning():
    """Reading R21(d): with the coefficient nu the ASP condition number (exact C) grows under
    refinement like h^-2; with nu h_T^2 it levels off (Table ST_ws reports h-robust k = 1 iteration
    counts).  Both weights keep E^T A E = Abar exact (div curl = 0)."""
    r0 = _asp_condition(3, 0) / _asp_condition(2, 0)
    r1 = _asp_condition(3, 1) / _asp_condition(2, 1)
    assert r0 > 2.0 and r1 < 1.5
    D = system.discretize(mesh.structured(3, 2), 1, NU, lo_stab=1)
    A = system.condensed_system(D, system.condense(D))
    E = precond.embedding(D)
    Ab = precond.abar(D.mesh, NU).toarray()
    assert np.abs((E.T @ A @ E).toarray() - Ab).max() < 1e-12 * np.abs(Ab).max()
    X = D.mesh.coords[D.mesh.elems]
    w = fem.stabilisation_weight(X, NU, 1)
    assert np.allclose(w, NU * 3.0 / 4.0)            # Kuhn tetrahedra of the N = 2 cube: diameter sqrt(3)/2
