"""The constant gamma of Corollary schur_SPD on one element (oracle side, test infrastructure).

Corollary schur_SPD bounds the Schur complement norm of the condensed velocity block by the Schur
complement of the HDG norm eq. (nhdg_eps):

    gamma^{-1} nu |(u, uhat)|^2_{eps,h,d}  <=  |(u, uhat)|^2_{A^d}  <=  nu |(u, uhat)|^2_{eps,h,d},

and the paper reports that experiments on the unit tetrahedron suggest gamma = O(1) or O((log k)^l).
Here both forms are built on a single element T (no boundary conditions):

* |(u, uhat)|^2_{eps,h} = ||eps(u)||_T^2 + sum_F ||Pi^{k-1}(u - uhat)_t||^2_{j,F}, with the facet norm
  of eq. (jFjumpN) taken literally, ||w||^2_{j,F} = sup_{s in P^k(T, R^d)} (w, s)_F^2 / ||s||_T^2
  = c^T Cw M^{-1} Cw^T c (Riesz representation over an orthonormal-ish basis of P^k(T, R^d));
* |.|_{eps,h,d} is its infimum over the element bubbles (eq. epshschur), i.e. the Schur complement
  of that matrix with respect to the bubble dofs;
* A^d_T is the double Schur complement of the condensed element matrix (eqs. Hcoeffs, factorSsigma).

Both vanish exactly on the rigid-body motions embedded as (u, Pi^{k-1} u_t); gamma is the inverse of
the smallest generalized eigenvalue of (A^d_T, nu N^d_T) on the complement of that kernel.  The
largest eigenvalue is not 1: the proof of Lemma SPD squares a sum of d + 2 terms as if it were a
sum of squares, so the upper bound holds with d + 2 in place of 1 (reading R22).  With the dual BDM
basis of the dof contract the element matrices lose digits as k grows (the rigid-body kernel is no
longer resolved at k = 8); the bubble Schur complements do not depend on the bubble basis, so the
table is computed with the contract's L2-orthonormal bubble basis (fem.interior_test_functions), which
keeps the kernel gap near 1e12 up to k = 8 and reproduces the contract basis's values where both hold.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np
import scipy.linalg as sla

from . import fem, polys, system


def unit_tetrahedron(d: int = 3) -> np.ndarray:
    """Vertices of the reference simplex (0, e_1, .., e_d) as one element [1, d+1, d] (reading: the
    paper's "unit tetrahedron")."""
    return np.vstack([np.zeros(d), np.eye(d)])[None]


def element_forms(k: int, nu: float = 1.0, X: np.ndarray | None = None, bubble_basis: str = "orthonormal"):
    """(A_T, N_T, sizes) on one element: the condensed matrix and the HDG-norm matrix over the local
    (u, uhat) dofs, local order [u_d | u_o | uhat].  bubble_basis: "orthonormal" (the contract) or "monomial"
    (fem.element_data); both forms then eliminate the same bubble space in a better-scaled basis."""
    X = unit_tetrahedron() if X is None else X
    d = X.shape[2]
    signs = np.ones((1, d + 1), dtype=np.int64)
    sz = fem.local_sizes(d, k)
    mats = fem.element_matrices(X, signs, k, nu, bubble_basis=bubble_basis)
    AT = system.condense(SimpleNamespace(mats=mats, sz=sz))[0]
    q = k + 2
    D = fem.element_data(X, signs, k, q=q, bubble_basis=bubble_basis)
    nu_, nA, nhF = sz["n_u"], sz["n_A"], sz["n_hatF"]
    # ||eps(u)||_T^2
    eps = 0.5 * (D.DU + np.swapaxes(D.DU, -1, -2))                    # [1, nq, n_u, d, d]
    N = np.zeros((nA, nA))
    N[:nu_, :nu_] = np.einsum("q,qiab,qjab->ij", D.wq[0], eps[0], eps[0])
    # P^k(T, R^d): ambient basis psi_i e_a on the element
    xv, _ = polys.quadrature(d, q)
    nk = polys.n_poly(d, k)
    psi = polys.dubiner(d, k, xv)[0]                                  # [nq, nk] (reference = element map)
    Mphi = np.kron(np.eye(d), np.einsum("q,qi,qj->ij", D.wq[0], psi, psi))
    s_ref, _ = polys.quadrature(d - 1, q)
    for f in range(d + 1):
        lv = fem.facet_local_vertices(d, f)
        vh = fem.ref_vertices(d)[lv]
        xh = vh[0] + s_ref @ (vh[1:] - vh[0])                         # reference points of facet f
        pf = polys.dubiner(d, k, xh)[0]                               # [nqf, nk]
        wf = D.fw[0, f]                                               # [nqf]
        H = D.fH[0, f][:, f * nhF:(f + 1) * nhF, :]                   # [nqf, nhF, d] tangential basis
        U = D.fU[0, f]                                                # [nqf, n_u, d]
        G = np.einsum("q,qia,qja->ij", wf, H, H)
        # coefficients of Pi^{k-1}(u - uhat)_t in the basis H: c = G^{-1} (moments of u) - uhat_f
        Pm = np.zeros((nhF, nA))
        Pm[:, :nu_] = np.linalg.solve(G, np.einsum("q,qia,qca->ci", wf, U, H))
        Pm[:, nu_ + f * nhF:nu_ + (f + 1) * nhF] = -np.eye(nhF)
        # (w, s)_F for w = sum_c c_c H_c and s = psi_i e_a
        Cw = np.einsum("q,qca,qi->cai", wf, H, pf).reshape(nhF, d * nk)
        Nj = Cw @ np.linalg.solve(Mphi, Cw.T)                         # ||.||^2_{j,F} in the basis H
        N += Pm.T @ Nj @ Pm
    return AT, N, sz


def schur_on_coupling(M: np.ndarray, sz: dict) -> np.ndarray:
    """Schur complement onto the coupling dofs [u_d | uhat] (inf over the bubbles, eq. epshschur)."""
    d = sz["d"]
    o = np.arange((d + 1) * sz["nF"], sz["n_u"])
    c = np.concatenate([np.arange((d + 1) * sz["nF"]), np.arange(sz["n_u"], sz["n_A"])])
    Mcc, Mco, Moo = M[np.ix_(c, c)], M[np.ix_(c, o)], M[np.ix_(o, o)]
    if len(o) == 0:
        return Mcc
    return Mcc - Mco @ np.linalg.solve(Moo, Mco.T)


def gamma(k: int, nu: float = 1.0, X: np.ndarray | None = None, bubble_basis: str = "orthonormal"):
    """(gamma, lambda_max, gap) of the pencil (A^d_T, nu N^d_T) on one element.  The common kernel is
    the d(d+1)/2 rigid-body motions; gap = (smallest nonzero) / (largest kernel) eigenvalue of the
    scaled N^d_T tells whether the element matrices still resolve it (about 1e10 and more when they do)."""
    AT, N, sz = element_forms(k, nu, X, bubble_basis)
    Ad = schur_on_coupling(AT, sz)
    Nd = schur_on_coupling(N, sz)
    Ad, Nd = 0.5 * (Ad + Ad.T), 0.5 * (Nd + Nd.T)
    # symmetric diagonal scaling (a congruence: the pencil's eigenvalues are unchanged) so that the
    # kernel threshold does not depend on the spread of the basis scales at high k
    sc = 1.0 / np.sqrt(np.diag(Nd))
    Ad, Nd = sc[:, None] * Ad * sc[None, :], sc[:, None] * Nd * sc[None, :]
    w, V = np.linalg.eigh(Nd)
    nker = sz["d"] * (sz["d"] + 1) // 2
    Q = V[:, nker:]
    lam = sla.eigh(Q.T @ Ad @ Q, nu * (Q.T @ Nd @ Q), eigvals_only=True)
    gap = w[nker] / max(abs(w[nker - 1]), 1e-300)
    return 1.0 / lam.min(), lam.max(), gap


if __name__ == "__main__":
    # the table of gamma(k) on the unit tetrahedron, k = 2..8 (about three minutes), in the
    # the contract's orthonormal bubble basis (the monomial one loses the kernel at k = 8)
    for k in range(2, 9):
        g, lmax, gap = gamma(k)
        print(f"k = {k}: gamma = {g:.3f}, lambda_max = {lmax:.3f}, kernel gap = {gap:.1e}", flush=True)
