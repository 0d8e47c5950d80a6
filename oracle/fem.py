"""Spaces and element matrices of the MCS method (oracle side, test infrastructure).

Spaces (Sec. 3, eqs. fes_V .. fes_Vbar), for k >= 2 on a simplex T:

* V_h = BDM^k: P^k(T, R^d), normal-continuous.  Basis = dual basis of the
  functionals (dof contract)
    - facet f, mode j:   int_F u.n_out q_j ds, q_j the orthonormal basis of
      P^k on the facet parameter simplex (sorted facet vertices);
    - interior m:        int_T u . (J^{-T} g_m(xhat)) dx, i.e. the moment of the
      Piola pull-back against g_m on the reference simplex, where g_m runs over
      (i) psi_a(xhat) e_c for the orthonormal psi_a of degree <= k-2
          (a-major, c-minor) and
      (ii) d=2: (-y, x) x^a y^b, a+b = k-2, a descending;
           d=3: x cross (x^alpha e_c), |alpha| = k-2, alpha in descending
           lexicographic order, c minor, skipping c = 3 when alpha_3 >= 1
      (the first-kind Nedelec space N_{k-1}), this list made L2(T_hat)-orthonormal in
      list order (Gram-Schmidt) so that the dual basis stays well scaled at high k.
  Global facet functions carry the orientation sign s_{T,f} so that their
  moment is taken against the global facet normal n_F.
* Vhat_h: on each facet q_j(s) e_m with q_j of degree <= k-1 and e_m the facet
  edge vectors (m-major).
* Q_h = P^{k-1}(T): orthonormal reference basis composed with the inverse
  element map.
* Sigma_h(T) = {tau in P^k(T, trace-free): tau_nt in P^{k-1}(F) on every facet}
  (element-local, hybridized), built here as the null space of the nt
  constraints in physical coordinates; W_h(T) = P^{k-1}(T, skew).  The condensed
  matrices do not depend on these two bases.

Element matrices follow the printed definitions after eq. (bigfemSPmat), with
physical quadrature on each element and facet.
"""
from __future__ import annotations

import functools
import itertools
import math
from dataclasses import dataclass

import numpy as np

from . import polys


def n_bdm_facet(d, k):
    return polys.n_poly(d - 1, k)


def local_sizes(d: int, k: int) -> dict:
    """Local dimensions.  k = 1 is the lowest-order variant of Sec. 7 (d = 3 only): W_h is
    the H(div) space P^0(T, R^3) + x P^0(T) with one normal-flux dof per facet, kept after
    condensation; its dof sits behind the two tangential Vhat_h dofs of each facet, so
    n_hatF = 3, n_tF = 2 (tangential) and n_omega = 0 (no element-local rotations)."""
    if k == 1:
        if d != 3:
            raise ValueError("the lowest-order variant (k = 1) is three-dimensional")
        sz = local_sizes_general(d, 1)
        sz.update(lowest=True, n_tF=2, n_hatF=3, n_hat=(d + 1) * 3, n_omega=0,
                  n_A=sz["n_full"] + (d + 1) * 3)
        return sz
    return local_sizes_general(d, k)


def local_sizes_general(d: int, k: int) -> dict:
    nk = polys.n_poly(d, k)
    n_full = d * nk
    nF = n_bdm_facet(d, k)
    n_bub = n_full - (d + 1) * nF
    n_hatF = (d - 1) * polys.n_poly(d - 1, k - 1)
    n_p = polys.n_poly(d, k - 1)
    n_omega = (d * (d - 1) // 2) * polys.n_poly(d, k - 1)
    n_raw_sigma = (d * d - 1) * nk
    n_con = (d + 1) * (d - 1) * (polys.n_poly(d - 1, k) - polys.n_poly(d - 1, k - 1))
    return dict(d=d, k=k, nk=nk, n_full=n_full, nF=nF, n_bub=n_bub, n_dd=(d + 1) * nF,
                n_hatF=n_hatF, n_tF=n_hatF, lowest=False, n_hat=(d + 1) * n_hatF, n_p=n_p,
                n_omega=n_omega,
                n_sigma=n_raw_sigma - n_con, n_raw_sigma=n_raw_sigma, n_con=n_con,
                n_u=n_full, n_A=n_full + (d + 1) * n_hatF)


def ref_vertices(d):
    return np.vstack([np.zeros(d), np.eye(d)])


def facet_local_vertices(d, f):
    return [v for v in range(d + 1) if v != f]


def interior_test_functions(d: int, k: int, xh: np.ndarray, basis: str = "orthonormal") -> np.ndarray:
    """g_m(xhat) at reference points xh[nq, d] -> [nq, n_bub, d].

    The dof contract's interior moment functions are the list (i)+(ii) below made L2(T_hat)-orthonormal
    in list order (Gram-Schmidt, i.e. the rows of L^{-1} for the Cholesky factor L of the list's Gram
    matrix on T_hat).  Without it the monomial part (ii) makes the dual BDM basis badly scaled at high k
    (2D k = 6: element matrices with entries near 1e11 around facet Schur complements near 1e2).
    basis="monomial": the list itself (the same BDM space, another bubble basis)."""
    raw = _interior_list(d, k, xh)
    if basis == "monomial" or raw.shape[1] == 0:
        return raw
    return np.einsum("qna,mn->qma", raw, _interior_orthonormaliser(d, k))


@functools.lru_cache(maxsize=None)
def _interior_orthonormaliser(d: int, k: int) -> np.ndarray:
    """L^{-1} with L L^T the Gram matrix of the interior list on T_hat (exact collapsed Gauss rule)."""
    x, w = polys.quadrature(d, k + 1)
    g = _interior_list(d, k, x)
    G = np.einsum("q,qma,qna->mn", w, g, g)
    return np.linalg.inv(np.linalg.cholesky(G))


def _interior_list(d: int, k: int, xh: np.ndarray) -> np.ndarray:
    """The list (i) psi_a e_c, deg psi_a <= k-2 (a-major, c-minor), then (ii) the Nedelec-type
    functions (-y, x) x^a y^b (2D, a descending) or x cross (x^alpha e_c) (3D, alpha descending
    lexicographic, c minor, c = 3 skipped when alpha_3 >= 1), |alpha| = k-2, at xh[nq, d]."""
    out = []
    if k >= 2:
        psi, _ = polys.dubiner(d, k - 2, xh)
        for a in range(psi.shape[1]):
            for c in range(d):
                g = np.zeros(xh.shape)
                g[:, c] = psi[:, a]
                out.append(g)
        m = k - 2
        if d == 2:
            x, y = xh[:, 0], xh[:, 1]
            for a in range(m, -1, -1):
                b = m - a
                mono = x ** a * y ** b
                out.append(np.stack([-y * mono, x * mono], axis=1))
        else:
            alphas = [al for al in itertools.product(range(m, -1, -1), repeat=3) if sum(al) == m]
            alphas.sort(reverse=True)
            for al in alphas:
                mono = xh[:, 0] ** al[0] * xh[:, 1] ** al[1] * xh[:, 2] ** al[2]
                for c in range(3):
                    if c == 2 and al[2] >= 1:
                        continue
                    q = np.zeros(xh.shape)
                    q[:, c] = mono
                    out.append(np.cross(xh, q))
    if not out:                                                 # k = 1: BDM^1 has no bubbles
        return np.zeros((xh.shape[0], 0, d))
    return np.stack(out, axis=1)


def trace_free_units(d):
    out = []
    for a in range(d):
        for b in range(d):
            if a != b:
                E = np.zeros((d, d))
                E[a, b] = 1.0
                out.append(E)
    for a in range(d - 1):
        E = np.zeros((d, d))
        E[a, a] = 1.0
        E[d - 1, d - 1] = -1.0
        out.append(E)
    return np.stack(out)


def skew_units(d):
    out = []
    for a in range(d):
        for b in range(a + 1, d):
            E = np.zeros((d, d))
            E[b, a] = 1.0
            E[a, b] = -1.0
            out.append(E)
    return np.stack(out)


@dataclass
class ElementData:
    """Physical basis values on a batch of elements."""
    detJ: np.ndarray      # [E]
    wq: np.ndarray        # [E, nq] physical volume weights
    xq: np.ndarray        # [E, nq, d] physical volume points
    U: np.ndarray         # [E, nq, n_u, d]
    DU: np.ndarray        # [E, nq, n_u, d, d]   DU[..., a, b] = d u_a / d x_b
    divU: np.ndarray      # [E, nq, n_u]
    P: np.ndarray         # [E, nq, n_p]
    S: np.ndarray         # [E, nq, n_s, d, d]
    divS: np.ndarray      # [E, nq, n_s, d]
    W: np.ndarray         # [E, nq, n_w, d, d]
    # facet data, per local facet f
    fw: np.ndarray        # [E, d+1, nqf] physical facet weights
    fx: np.ndarray        # [E, d+1, nqf, d]
    fn: np.ndarray        # [E, d+1, d] outward unit normal
    fU: np.ndarray        # [E, d+1, nqf, n_u, d]
    fS: np.ndarray        # [E, d+1, nqf, n_s, d, d]
    fH: np.ndarray        # [E, d+1, nqf, n_hat, d]  hat basis (zero off its facet)
    divW: np.ndarray | None = None   # k = 1: [E, nq, d+1] div of the H(div) rotation functions


@functools.lru_cache(maxsize=None)
def _ref_rules(d, q):
    xv, wv = polys.quadrature(d, q)
    s, ws = polys.quadrature(d - 1, q)
    return xv, wv, s, ws


def element_data(X: np.ndarray, signs: np.ndarray, k: int, q: int | None = None,
                 velocity_only: bool = False, bubble_basis: str = "orthonormal") -> ElementData:
    """Physical bases of all spaces on the elements with vertex coordinates X[E, d+1, d].

    bubble_basis: "orthonormal" (the dof contract) or "monomial" (the unorthonormalised interior list;
    the same BDM space and facet functions, another bubble basis: quantities that eliminate the bubbles,
    such as A^d_T, change only by rounding).

    velocity_only: only U, DU, divU and P are evaluated (the other fields are None)."""
    E_, dp1, d = X.shape
    sz = local_sizes(d, k)
    q = q if q is not None else k + 2
    xv, wv, s, ws = _ref_rules(d, q)
    nq, nqf = len(wv), len(ws)
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))      # [E, d, d] columns x_i - x_0
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    JinvT = np.transpose(Jinv, (0, 2, 1))
    xq = X[:, :1, :] + np.einsum("eab,qb->eqa", J, xv)
    wq = np.abs(detJ)[:, None] * wv[None, :]
    nk = sz["nk"]
    psi, gpsi_ref = polys.dubiner(d, k, xv)                     # [nq, nk], [nq, nk, d]
    gpsi = np.einsum("eab,qnb->eqna", JinvT, gpsi_ref)          # physical gradients

    # facet geometry, reference points of each local facet
    Vref = ref_vertices(d)
    fxh, fw, fx, fn, Fmeas = [], [], [], [], []
    for f in range(dp1):
        lv = facet_local_vertices(d, f)
        vh = Vref[lv]
        xh = vh[0] + s @ (vh[1:] - vh[0])                        # [nqf, d]
        fxh.append(xh)
        Xf = X[:, lv, :]                                        # [E, d, d]
        Ef = Xf[:, 1:, :] - Xf[:, :1, :]
        G = np.einsum("ema,ena->emn", Ef, Ef)
        meas = np.sqrt(np.linalg.det(G)) / np.prod(np.arange(1, d))  # |F| = sqrt(det G)/(d-1)!
        Fmeas.append(meas)
        ref_meas = 1.0 / np.prod(np.arange(1, d))               # |T_{d-1}|
        fw.append(meas[:, None] / ref_meas * ws[None, :])
        fx.append(Xf[:, :1, :] + np.einsum("qm,ema->eqa", s, Ef))
        # outward normal: perpendicular to facet, pointing away from the opposite vertex
        if d == 2:
            e = Ef[:, 0, :]
            nrm = np.stack([-e[:, 1], e[:, 0]], axis=1)
        else:
            nrm = np.cross(Ef[:, 0, :], Ef[:, 1, :])
        nrm = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
        away = Xf[:, 0, :] - X[:, f, :]
        nrm = nrm * np.sign(np.einsum("ea,ea->e", nrm, away))[:, None]
        fn.append(nrm)
    fw = np.stack(fw, axis=1)
    fx = np.stack(fx, axis=1)
    fn = np.stack(fn, axis=1)

    # ---------------- BDM^k: dual basis -------------------------------------
    n_full = sz["n_full"]
    # ambient basis Phi_(a, i) = psi_i e_a, index c = a*nk + i
    def amb_vals(psiv):                                         # psiv [..., nk] -> [..., n_full, d]
        out = np.zeros(psiv.shape[:-1] + (n_full, d))
        for a in range(d):
            out[..., a * nk:(a + 1) * nk, a] = psiv
        return out

    def amb_grads(gp):                                          # gp [..., nk, d] -> [..., n_full, d, d]
        out = np.zeros(gp.shape[:-2] + (n_full, d, d))
        for a in range(d):
            out[..., a * nk:(a + 1) * nk, a, :] = gp
        return out

    C = np.zeros((E_, n_full, n_full))
    qF = polys.dubiner(d - 1, k, s)[0]                          # [nqf, nF]
    nF = sz["nF"]
    fpsi = []
    for f in range(dp1):
        pv, _ = polys.dubiner(d, k, fxh[f])                     # [nqf, nk]
        fpsi.append(pv)
        Phi = amb_vals(pv)                                      # [nqf, n_full, d]
        flux = np.einsum("qca,ea->eqc", Phi, fn[:, f, :])       # [E, nqf, n_full]
        C[:, f * nF:(f + 1) * nF, :] = np.einsum("eq,qj,eqc->ejc", fw[:, f, :], qF, flux)
    g = interior_test_functions(d, k, xv, bubble_basis)         # [nq, n_bub, d]
    gphys = np.einsum("eab,qmb->eqma", JinvT, g)
    Phiv = amb_vals(psi)                                        # [nq, n_full, d]
    C[:, (d + 1) * nF:, :] = np.einsum("eq,qca,eqma->emc", wq, Phiv, gphys)
    Cinv = np.linalg.inv(C)                                     # columns = dual functions
    sgn = np.ones((E_, n_full))
    for f in range(dp1):
        sgn[:, f * nF:(f + 1) * nF] = signs[:, f][:, None]
    coef = Cinv * sgn[:, None, :]                               # [E, c, r]
    U = np.einsum("qca,ecr->eqra", Phiv, coef)
    DU = np.einsum("eqcab,ecr->eqrab", amb_grads(gpsi), coef)
    divU = np.einsum("eqraa->eqr", DU)
    fU = np.stack([np.einsum("qca,ecr->eqra", amb_vals(fpsi[f]), coef) for f in range(dp1)], axis=1)

    # ---------------- pressure ---------------------------------------------
    n_p = sz["n_p"]
    P = np.broadcast_to(psi[None, :, :n_p], (E_, nq, n_p)).copy()
    if velocity_only:
        return ElementData(detJ, wq, xq, U, DU, divU, P, None, None, None, fw, fx, fn, fU, None, None)

    # ---------------- Sigma(T): null space of the nt constraints -----------
    TF = trace_free_units(d)                                    # [ns0, d, d]
    ns0 = TF.shape[0]
    n_raw = ns0 * nk
    # raw basis R_(s, i) = psi_i TF_s, index s*nk + i
    def raw_vals(psiv):
        return np.einsum("...i,sab->...siab", psiv, TF).reshape(psiv.shape[:-1] + (n_raw, d, d))

    degF = polys.degrees(d - 1, k)
    top = np.nonzero(degF == k)[0]
    cons = []
    for f in range(dp1):
        lv = facet_local_vertices(d, f)
        Ef = X[:, lv[1:], :] - X[:, lv[:1], :]                  # [E, d-1, d]
        Rf = raw_vals(fpsi[f])                                   # [nqf, n_raw, d, d]
        Rn = np.einsum("qrab,eb->eqra", Rf, fn[:, f, :])         # tau n
        for m in range(d - 1):
            comp = np.einsum("eqra,ea->eqr", Rn, Ef[:, m, :])    # (tau n).e_m = tau_nt . e_m
            cons.append(np.einsum("eq,qj,eqr->ejr", fw[:, f, :], qF[:, top], comp))
    Ccon = np.concatenate(cons, axis=1)                          # [E, n_con, n_raw]
    # scale rows to unit size before the rank decision
    Ccon = Ccon / np.linalg.norm(Ccon, axis=2, keepdims=True)
    _, sv, Vh = np.linalg.svd(Ccon)
    rank = Ccon.shape[1]
    assert np.all(sv[:, -1] > 1e-8 * sv[:, 0]), "nt constraints are dependent"
    Nsig = np.transpose(Vh[:, rank:, :], (0, 2, 1))              # [E, n_raw, n_sigma]
    Rv = raw_vals(psi)                                           # [nq, n_raw, d, d]
    S = np.einsum("qrab,ers->eqsab", Rv, Nsig)
    # div of raw: (div R)_a = sum_b TF_ab d_b psi
    divR = np.einsum("sab,eqib->eqsia", TF, gpsi).reshape(E_, nq, n_raw, d)
    divS = np.einsum("eqra,ers->eqsa", divR, Nsig)
    fS = np.stack([np.einsum("qrab,ers->eqsab", raw_vals(fpsi[f]), Nsig) for f in range(dp1)], axis=1)

    divW = None
    if sz["lowest"]:
        # ------------ k = 1 (Sec. 7): W_h in H(div), P^0(T, R^3) + x P^0(T) -----------
        # dof of facet f = flux through F with the global normal n_F, so the function of local
        # facet f is s_{T,f} (x - x_f) / (d |T|), x_f the vertex opposite f (its flux out of T
        # through F_f is 1, through the other facets 0); every occurrence of omega is kappa(omega)
        vol = np.abs(detJ) / math.factorial(d)
        W = np.zeros((E_, nq, dp1, d, d))
        divW = np.zeros((E_, nq, dp1))
        for f in range(dp1):
            phi = signs[:, f][:, None, None] * (xq - X[:, f, None, :]) / (d * vol)[:, None, None]
            W[:, :, f] = kappa(phi)
            divW[:, :, f] = (signs[:, f] / vol)[:, None]
    else:
        # ---------------- W_h = P^{k-1}(T, skew) ----------------------------
        K = skew_units(d)
        nkm1 = polys.n_poly(d, k - 1)
        W = np.einsum("qi,rab->qriab", psi[:, :nkm1], K).reshape(nq, -1, d, d)
        W = np.broadcast_to(W[None], (E_,) + W.shape).copy()

    # ---------------- Vhat_h on facets ---------------------------------------
    nFm1 = polys.n_poly(d - 1, k - 1)
    n_hatF = sz["n_hatF"]
    fH = np.zeros((E_, dp1, nqf, (d + 1) * n_hatF, d))
    for f in range(dp1):
        lv = facet_local_vertices(d, f)
        Ef = X[:, lv[1:], :] - X[:, lv[:1], :]
        for m in range(d - 1):
            for j in range(nFm1):
                col = f * n_hatF + m * nFm1 + j
                fH[:, f, :, col, :] = qF[None, :, j, None] * Ef[:, None, m, :]

    return ElementData(detJ, wq, xq, U, DU, divU, P, S, divS, W, fw, fx, fn, fU, fS, fH, divW)


def kappa(v: np.ndarray) -> np.ndarray:
    """kappa of Sec. 2 (notation) for d = 3: v[..., 3] -> 1/2 [[0, -v3, v2], [v3, 0, -v1], [-v2, v1, 0]]."""
    out = np.zeros(v.shape + (3,))
    out[..., 0, 1] = -v[..., 2]
    out[..., 0, 2] = v[..., 1]
    out[..., 1, 0] = v[..., 2]
    out[..., 1, 2] = -v[..., 0]
    out[..., 2, 0] = -v[..., 1]
    out[..., 2, 1] = v[..., 0]
    return 0.5 * out


def stabilisation_weight(X: np.ndarray, nu: float, lo_stab: int) -> np.ndarray:
    """Coefficient of (div omega, div eta)_T for k = 1, per element [E]: lo_stab = 0 takes nu (the
    printed form at nu = 1, reading R21(d)); lo_stab = 1 takes nu h_T^2 with h_T the element diameter
    (longest edge), which keeps the term within the section's norm (reading R21(d'))."""
    if lo_stab == 0:
        return np.full(X.shape[0], nu)
    diam2 = np.max([np.sum((X[:, a] - X[:, b]) ** 2, axis=1)
                    for a in range(X.shape[1]) for b in range(a + 1, X.shape[1])], axis=0)
    return nu * diam2


def element_matrices(X, signs, k, nu, lo_stab: int = 0, bubble_basis: str = "orthonormal"):
    """Local blocks of eq. (bigfemSPmat) on every element of the batch.

    Returns dict of arrays [E, rows, cols]:
      M   = nu^{-1} (phi^sigma_i, phi^sigma_j)_T
      Bw  = (phi^sigma_j : phi^omega_i)_T                 (volume integral, reading R2)
      Bu  = (div phi^sigma_j, phi^u_i)_T - (phi^sigma_j,nn, phi^u_i,n)_dT
      Bh  = -(phi^sigma_j,nt, phi^uhat_i,t)_dT
      Adiv= nu d^{-1} (div phi^u_i, div phi^u_j)_T
      Bp  = -(div phi^u_j, phi^p_i)_T                     (weak form sign, reading R18)
      Mu  = (phi^u_i, phi^u_j)_T
    """
    D = element_data(X, signs, k, bubble_basis=bubble_basis)
    d = X.shape[2]
    out = {}
    out["M"] = np.einsum("eq,eqiab,eqjab->eij", D.wq, D.S, D.S) / nu
    if D.divW is None:
        out["Bw"] = np.einsum("eq,eqjab,eqiab->eij", D.wq, D.S, D.W)
    vol = np.einsum("eq,eqja,eqia->eij", D.wq, D.divS, D.U)
    Snn = np.einsum("efqjab,efa,efb->efqj", D.fS, D.fn, D.fn)
    Un = np.einsum("efqia,efa->efqi", D.fU, D.fn)
    bnd = np.einsum("efq,efqj,efqi->eij", D.fw, Snn, Un)
    out["Bu"] = vol - bnd
    Sn = np.einsum("efqjab,efb->efqja", D.fS, D.fn)
    Snt = Sn - Snn[..., None] * D.fn[:, :, None, None, :]
    out["Bh"] = -np.einsum("efq,efqja,efqia->eij", D.fw, Snt, D.fH)
    if D.divW is not None:
        # k = 1 (Sec. 7): the rotation dofs are the third entry of each facet's hat block; they
        # couple to sigma through (phi^sigma, kappa(phi^omega))_T and carry the stabilisation
        # c_T (div omega, div eta)_T with c_T = stabilisation_weight (reading R21)
        nhF = D.fH.shape[3] // (d + 1)
        rows = [f * nhF + nhF - 1 for f in range(d + 1)]
        out["Bw"] = np.zeros((X.shape[0], 0, D.S.shape[2]))
        out["Bh"][:, rows, :] = np.einsum("eq,eqjab,eqfab->efj", D.wq, D.S, D.W)
        Sh = np.zeros((X.shape[0], len(out["Bh"][0]), len(out["Bh"][0])))
        cT = stabilisation_weight(X, nu, lo_stab)
        Sh[:, np.ix_(rows, rows)[0], np.ix_(rows, rows)[1]] = \
            cT[:, None, None] * np.einsum("eq,eqf,eqg->efg", D.wq, D.divW, D.divW)
        out["Shat"] = Sh
    out["Adiv"] = nu / d * np.einsum("eq,eqi,eqj->eij", D.wq, D.divU, D.divU)
    out["Bp"] = -np.einsum("eq,eqj,eqi->eij", D.wq, D.divU, D.P)
    out["Mu"] = np.einsum("eq,eqia,eqja->eij", D.wq, D.U, D.U)
    out["Mp"] = np.einsum("eq,eqi,eqj->eij", D.wq, D.P, D.P)
    return out


def load_vector(X, signs, k, f, q=None):
    """F_i = (f, phi^u_i)_T on each element; f(x[..., d]) -> [..., d]."""
    D = element_data(X, signs, k, q=q if q is not None else k + 8, velocity_only=True)
    fv = f(D.xq)
    return np.einsum("eq,eqa,eqia->ei", D.wq, fv, D.U)
