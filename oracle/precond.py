"""Auxiliary-space preconditioner of the MCS velocity block (oracle side, test infrastructure).

* ``p1_space``     conforming space Vbar_h = P^1 vector fields, zero on the
                   boundary (eq. fes_Vbar); dofs = interior vertices in
                   ascending id, vertex-major (rank*d + component).
* ``abar``         abar(u, v) = nu (eps u, eps v) (eq. defAhat with the scale
                   read as nu, reading R1).
* ``embedding``    E ubar = (ubar, (ubar)_t) (eq. defE), written out through the
                   dof functionals: facet flux moments, interior moments, and the
                   L2(F) projection of the tangential trace onto Vhat_h; for the
                   lowest-order variant (k = 1, Sec. 7) E ubar = (ubar,
                   Pi^0 (ubar)_t, curl ubar), the L2 projection being Pi^0 there.
* ``GMG``          geometric multigrid V-cycle used as C (reading R11): nested
                   Kuhn meshes, prolongation = P1 interpolation (2-point edge
                   average), 2 pre- and 2 post-sweeps of l1-Jacobi
                   (D = diag(sum_j |A_ij|)), exact solve on the coarsest level.
* ``FacetBlockGS`` block Gauss-Seidel on A^d with one block per interior facet
                   (Theorem aux_pc_schur, Corollary aux_pc_mult), facets swept
                   colour by colour; the adjoint sweep runs the colours backwards.
* ``ASP``          multiplicative ASP of Sec. 5.2 applied to the condensed system
                   (Sec. 6.1): s smoothing sweeps, coarse correction
                   E^d C^{-1} E^d^T on the new residual, s adjoint sweeps;
                   wrapped by the factorization eq. (factorSsigma) into
                   Ahat^ext^{-1} (bubble elimination and back substitution).
* ``FullASP``      the ASP of Theorem aux_pc on the full velocity block (bubbles not
                   condensed): overlapping facet blocks with the neighbours' bubbles,
                   additive or multiplicative (colour-ordered block Gauss-Seidel).
* ``Khat_inv``     block preconditioner eq. (mhatinvfactor) with Ahat^{-1} in
                   both factors (reading R3) and Shat_p = M_p = nu^{-1}(p, q);
                   implemented with two applications of Ahat^{-1}.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, mesh as meshmod, polys, system


# ------------------------------------------------------------------ P1 space
def p1_map(m: meshmod.Mesh):
    """vertex id -> interior rank (-1 on the boundary)."""
    iv = meshmod.interior_vertices(m)
    rank = -np.ones(m.coords.shape[0], dtype=np.int64)
    rank[iv] = np.arange(len(iv))
    return rank, len(iv)


OUTFLOW_C = 4.0   # C of Lemma outflow (reading R23)


def outflow_penalty(m: meshmod.Mesh, nu: float, k: int, C: float = OUTFLOW_C) -> sp.csr_matrix:
    """Tangential penalty of Lemma outflow on the free P1 dofs:
    sum_{F in Gamma_Ntilde} nu C k^2 / h_F int_F ubar_t . vbar_t ds, h_F the facet diameter.
    With the P1 hat functions, int_F lambda_a lambda_b = |F| (1 + delta_ab) / (d (d + 1))."""
    d = m.dim
    rank, nv = p1_map(m)
    R, Cc, V = [], [], []
    for F in np.nonzero(m.outflow)[0]:
        w = m.facets[F]
        Xf = m.coords[w]
        Ef = Xf[1:] - Xf[:1]
        meas = np.sqrt(np.linalg.det(Ef @ Ef.T)) / np.prod(np.arange(1, d))
        hF = max(np.linalg.norm(Xf[a] - Xf[b]) for a in range(d) for b in range(a + 1, d))
        n = m.normals[F]
        Pt = np.eye(d) - np.outer(n, n)
        c = nu * C * k * k / hF
        for a in range(d):
            for b in range(d):
                if rank[w[a]] < 0 or rank[w[b]] < 0:
                    continue
                mab = meas * (1.0 + (a == b)) / (d * (d + 1))
                for i in range(d):
                    for j in range(d):
                        R.append(rank[w[a]] * d + i); Cc.append(rank[w[b]] * d + j); V.append(c * mab * Pt[i, j])
    return sp.csr_matrix((V, (R, Cc)), shape=(nv * d, nv * d))


def abar(m: meshmod.Mesh, nu: float, k: int | None = None, C: float = OUTFLOW_C) -> sp.csr_matrix:
    """Abar = nu (eps(u), eps(v)) on the free P1 vector fields; with Gamma_Ntilde marked, plus the
    tangential penalty of Lemma outflow (k required)."""
    d = m.dim
    rank, nv = p1_map(m)
    X = m.coords[m.elems]
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
    vol = np.abs(np.linalg.det(J)) / np.prod(np.arange(1, d + 1))
    # gradients of barycentric coordinates
    ghat = np.vstack([-np.ones(d), np.eye(d)])                 # [d+1, d] reference
    g = np.einsum("eba,vb->eva", np.linalg.inv(J), ghat)        # J^{-T} ghat
    ne = X.shape[0]
    nl = (d + 1) * d
    # eps of basis (vertex v, comp a): sym(e_a g_v^T)
    epsb = np.zeros((ne, d + 1, d, d, d))
    for a in range(d):
        epsb[:, :, a, a, :] += 0.5 * g
        epsb[:, :, a, :, a] += 0.5 * g
    epsb = epsb.reshape(ne, nl, d, d)
    Ke = nu * vol[:, None, None] * np.einsum("eiab,ejab->eij", epsb, epsb)
    r = rank[m.elems]                                           # [ne, d+1]
    gm = np.where(r[:, :, None] >= 0, r[:, :, None] * d + np.arange(d)[None, None, :], -1)
    gm = gm.reshape(ne, nl)
    A = system.assemble(gm, gm, Ke, (nv * d, nv * d))
    if m.outflow is not None:
        A = (A + outflow_penalty(m, nu, k, C)).tocsr()
    return A


def prolongation(coarse: meshmod.Mesh, fine: meshmod.Mesh) -> sp.csr_matrix:
    """P1 interpolation from the N/2 mesh to the N mesh (interior dofs)."""
    d = fine.dim
    rc, nc = p1_map(coarse)
    rf, nf = p1_map(fine)
    idx = meshmod.mesh_index(fine)
    Nc1 = coarse.N + 1
    stride = np.array([Nc1 ** a for a in range(d)])
    R, C, V = [], [], []
    for vid in np.nonzero(rf >= 0)[0]:
        I = idx[vid]
        o = I % 2
        a = (I - o) // 2
        b = (I + o) // 2
        ends = [a] if not o.any() else [a, b]
        w = 1.0 / len(ends)
        for e in ends:
            cv = int(e @ stride)
            if rc[cv] >= 0:
                for c in range(d):
                    R.append(rf[vid] * d + c)
                    C.append(rc[cv] * d + c)
                    V.append(w)
    return sp.csr_matrix((V, (R, C)), shape=(nf * d, nc * d))


class GMG:
    """Symmetric V-cycle for Abar on the hierarchy N0, 2 N0, ..., N (C^{-1} ~ Abar^{-1})."""

    def __init__(self, dim: int, N: int, levels: int, nu: float, smooth: int = 2, outflow_k: int | None = None,
                 C: float = OUTFLOW_C):
        """outflow_k: with Gamma_Ntilde marked on every level, the degree k of the penalty."""
        self.meshes = [meshmod.structured(dim, N >> (levels - 1 - l)) for l in range(levels)]
        if outflow_k is not None:
            self.meshes = [meshmod.with_outflow(m) for m in self.meshes]
        self.A = [abar(m, nu, outflow_k, C) for m in self.meshes]
        self.P = [None] + [prolongation(self.meshes[l - 1], self.meshes[l]) for l in range(1, levels)]
        self.Dl1 = [np.asarray(abs(A).sum(axis=1)).ravel() for A in self.A]
        self.smooth = smooth
        self.coarse = np.linalg.inv(self.A[0].toarray()) if self.A[0].shape[0] else np.zeros((0, 0))

    def vcycle(self, b: np.ndarray, l: int | None = None) -> np.ndarray:
        l = len(self.A) - 1 if l is None else l
        if l == 0:
            return self.coarse @ b
        A, D = self.A[l], self.Dl1[l]
        x = np.zeros_like(b)
        for _ in range(self.smooth):
            x = x + (b - A @ x) / D
        r = b - A @ x
        x = x + self.P[l] @ self.vcycle(self.P[l].T @ r, l - 1)
        for _ in range(self.smooth):
            x = x + (b - A @ x) / D
        return x


# ------------------------------------------------------------------ embedding E
def embedding(D: system.Discretization) -> sp.csr_matrix:
    """E: P1 interior dofs -> condensed layout [u_d | u_o | uhat | p] (p rows zero)."""
    m, k = D.mesh, D.k
    d = m.dim
    sz = D.sz
    rank, nv = p1_map(m)
    R, C, V = [], [], []
    nF, nhF, ntF, nb = sz["nF"], sz["n_hatF"], sz["n_tF"], sz["n_bub"]
    s, ws = polys.quadrature(d - 1, k + 2)
    qF = polys.dubiner(d - 1, k, s)[0]
    nFm1 = polys.n_poly(d - 1, k - 1)
    ref_meas = 1.0 / np.prod(np.arange(1, d))
    # facet rows: BDM moments on every BDM-dof facet; uhat rows on interior facets only (on
    # Gamma_Ntilde, pi_0 of Lemma outflow zeroes them: there are no uhat dofs there)
    urank = m.u_rank
    for F in np.nonzero(m.udof)[0]:
        r = urank[F]
        ri = m.int_rank[F]
        w = m.facets[F]
        Xf = m.coords[w]
        Ef = Xf[1:] - Xf[:1]
        meas = np.sqrt(np.linalg.det(Ef @ Ef.T)) / np.prod(np.arange(1, d))
        wf = ws * meas / ref_meas
        lam = np.hstack([1 - s.sum(axis=1, keepdims=True), s])   # barycentrics of facet vertices
        # L2(F) Gram of the uhat basis q_j e_m
        basis = []
        for mm in range(d - 1):
            for j in range(nFm1):
                basis.append(qF[:, j, None] * Ef[mm][None, :])
        basis = np.stack(basis, axis=1)                          # [nq, nhF, d]
        G = np.einsum("q,qia,qja->ij", wf, basis, basis)
        for iv, vid in enumerate(w):
            if rank[vid] < 0:
                continue
            for a in range(d):
                col = rank[vid] * d + a
                ub = np.zeros((len(ws), d))
                ub[:, a] = lam[:, iv]
                flux = ub @ m.normals[F]
                mom = np.einsum("q,qj,q->j", wf, qF, flux)
                for j in range(nF):
                    R.append(r * nF + j); C.append(col); V.append(mom[j])
                if ri < 0:
                    continue
                rhs = np.einsum("q,qa,qia->i", wf, ub, basis)
                ch = np.linalg.solve(G, rhs)
                for j in range(ntF):
                    R.append(D.off_h + ri * nhF + j); C.append(col); V.append(ch[j])
                if sz["lowest"]:
                    # k = 1 (Sec. 7): third component curl(ubar), as its flux int_F curl(ubar).n_F;
                    # curl(lambda_v e_a) = grad(lambda_v) x e_a, taken on an adjacent element
                    T = m.facet_elems[F, 0]
                    XT = m.coords[m.elems[T]]
                    JT = (XT[1:] - XT[:1]).T
                    ghat = np.vstack([-np.ones(d), np.eye(d)])
                    gl = np.linalg.solve(JT.T, ghat[list(m.elems[T]).index(vid)])
                    ea = np.zeros(d)
                    ea[a] = 1.0
                    R.append(D.off_h + ri * nhF + ntF); C.append(col)
                    V.append(meas * float(np.cross(gl, ea) @ m.normals[F]))
    # bubble rows: interior moments I_m(ubar|T) = int_T ubar . J^{-T} g_m
    X = m.coords[m.elems]
    xv, wv = polys.quadrature(d, k + 2)
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
    JinvT = np.transpose(np.linalg.inv(J), (0, 2, 1))
    absdet = np.abs(np.linalg.det(J))
    g = fem.interior_test_functions(d, k, xv)                  # [nq, nb, d]
    lam = np.hstack([1 - xv.sum(axis=1, keepdims=True), xv])   # [nq, d+1]
    for T in range(X.shape[0]):
        gphys = np.einsum("ab,qmb->qma", JinvT[T], g)
        for iv, vid in enumerate(m.elems[T]):
            if rank[vid] < 0:
                continue
            for a in range(d):
                mom = absdet[T] * np.einsum("q,q,qm->m", wv, lam[:, iv], gphys[:, :, a])
                for b in range(nb):
                    R.append(D.off_o + T * nb + b); C.append(rank[vid] * d + a); V.append(mom[b])
    return sp.csr_matrix((V, (R, C)), shape=(D.ndof, nv * d))


# ------------------------------------------------------------------ condensed preconditioner
class ASP:
    """Ahat^{-1} on the velocity block (u_d, u_o, uhat) of the condensed layout."""

    def __init__(self, D: system.Discretization, AT: np.ndarray, gmg: GMG,
                 smooth: int = 2, multiplicative: bool = True):
        self.D = D
        m = D.mesh
        d = m.dim
        sz = D.sz
        self.Ad, self.G, self.Aoo = system.bubble_condense(D, AT)
        o, c = system.local_split(D)
        am = D.a_map
        self.cmap = am[:, c]                                    # coupling dofs (global), -1 on Dirichlet
        self.omap = am[:, o]
        n = D.ndof
        self.Ad_glob = system.assemble(self.cmap, self.cmap, self.Ad, (n, n)).tocsr()
        nF, nhF = sz["nF"], sz["n_hatF"]
        self.nint = m.n_int
        A = self.Ad_glob
        self.colour = meshmod.colouring(m)
        self.ncol = int(self.colour.max()) + 1 if len(self.colour) else 0
        if m.outflow is None:
            self.fdofs = np.array([np.concatenate([r * nF + np.arange(nF), D.off_h + r * nhF + np.arange(nhF)])
                                   for r in range(self.nint)]).reshape(self.nint, nF + nhF)
            self.Dinv = np.stack([np.linalg.inv(A[f][:, f].toarray()) for f in self.fdofs]) \
                if self.nint else np.zeros((0, nF + nhF, nF + nhF))
            self.fblocks = None
        else:
            # one block per BDM-dof facet: its nF moments, plus its uhat dofs if it is interior
            self.fblocks = []
            for F in np.nonzero(m.udof)[0]:
                r, ri = m.u_rank[F], m.int_rank[F]
                blk = list(r * nF + np.arange(nF))
                if ri >= 0:
                    blk += list(D.off_h + ri * nhF + np.arange(nhF))
                self.fblocks.append(np.array(blk, dtype=np.int64))
            self.Dinv = [np.linalg.inv(A[f][:, f].toarray()) for f in self.fblocks]
        E = embedding(D)
        cd = np.concatenate([np.arange(D.n_dd), D.off_h + np.arange(D.n_hat)])
        mask = np.zeros(n, dtype=bool)
        mask[cd] = True
        self.Ed = sp.diags(mask.astype(float)) @ E             # rows of u_d and uhat only
        self.gmg = gmg
        self.smooth = smooth
        self.multiplicative = multiplicative

    def _sweep(self, x, b, order):
        for c in order:
            if self.fblocks is not None:
                r = b - self.Ad_glob @ x
                for i in np.nonzero(self.colour == c)[0]:
                    x[self.fblocks[i]] += self.Dinv[i] @ r[self.fblocks[i]]
                continue
            fs = self.fdofs[self.colour == c]
            if len(fs) == 0:
                continue
            r = b - self.Ad_glob @ x
            x[fs] += np.einsum("fij,fj->fi", self.Dinv[self.colour == c], r[fs])
        return x

    def apply_ad(self, b: np.ndarray) -> np.ndarray:
        """Multiplicative (or additive) ASP for A^d on the coupling dofs."""
        if not self.multiplicative:
            x = np.zeros_like(b)
            if self.fblocks is not None:
                for blk, Di in zip(self.fblocks, self.Dinv):
                    x[blk] += Di @ b[blk]
            else:
                fs = self.fdofs
                x[fs] = np.einsum("fij,fj->fi", self.Dinv, b[fs])
            return x + self.Ed @ self.gmg.vcycle(self.Ed.T @ b)
        x = np.zeros_like(b)
        fwd = range(self.ncol)
        bwd = range(self.ncol - 1, -1, -1)
        for _ in range(self.smooth):
            x = self._sweep(x, b, fwd)
        r = b - self.Ad_glob @ x
        x = x + self.Ed @ self.gmg.vcycle(self.Ed.T @ r)
        for _ in range(self.smooth):
            x = self._sweep(x, b, bwd)
        return x

    def apply(self, r: np.ndarray) -> np.ndarray:
        """Ahat^ext^{-1} r for r in the condensed layout (p part ignored, zero on output)."""
        D = self.D
        cm, om = self.cmap, self.omap
        ok = cm >= 0
        ro = r[om]                                              # [ne, n_o]
        # r_d <- r_d - G^T r_o  (per element, summed into the facet dofs)
        rc = r.copy()
        rc[D.off_o:D.off_h] = 0.0
        rc[D.off_p:] = 0.0
        contrib = np.einsum("eoc,eo->ec", self.G, ro)
        np.add.at(rc, cm[ok], -contrib[ok])
        xc = self.apply_ad(rc)
        xcl = np.where(ok, xc[np.maximum(cm, 0)], 0.0)
        xo = np.linalg.solve(self.Aoo, ro[..., None])[..., 0] - np.einsum("eoc,ec->eo", self.G, xcl)
        x = xc
        x[om] = xo
        x[D.off_p:] = 0.0
        return x


class FullASP:
    """ASP on the full (sigma, omega-condensed, bubble-uncondensed) velocity block A (Theorem aux_pc):
    one overlapping block per interior facet F holding F's dofs (BDM facet moments, uhat) and the
    bubbles of both elements of F; with E (all rows, bubbles included) and C.  Additive:
    M^{-1} + E C^{-1} E^T with M the overlapping block Jacobi; multiplicative: the blocks swept colour
    by colour (facets of one colour share no element, so their blocks are disjoint), the coarse
    correction on the new residual, and the adjoint sweep (Sec. 5.2)."""

    def __init__(self, D: system.Discretization, AT: np.ndarray, gmg: GMG,
                 smooth: int = 2, multiplicative: bool = True):
        self.D = D
        m = D.mesh
        sz = D.sz
        n = D.ndof
        am = D.a_map
        self.A = system.assemble(am, am, AT, (n, n)).tocsr()
        nF, nhF, nb = sz["nF"], sz["n_hatF"], sz["n_bub"]
        ints = np.nonzero(m.interior)[0]
        blocks = []
        for r, F in enumerate(ints):
            own = [r * nF + j for j in range(nF)] + [D.off_h + r * nhF + j for j in range(nhF)]
            bub = [D.off_o + T * nb + j for T in m.facet_elems[F] for j in range(nb)]
            blocks.append(np.array(own + bub, dtype=np.int64))
        self.blocks = blocks
        self.Dinv = [np.linalg.inv(self.A[b][:, b].toarray()) for b in blocks]
        self.colour = meshmod.colouring(m)
        self.ncol = int(self.colour.max()) + 1 if len(blocks) else 0
        self.vel = np.arange(D.off_p)
        E = embedding(D)
        mask = np.zeros(n)
        mask[self.vel] = 1.0
        self.E = sp.diags(mask) @ E
        self.gmg = gmg
        self.smooth = smooth
        self.multiplicative = multiplicative

    def _sweep(self, x, b, order):
        for c in order:
            r = b - self.A @ x
            for i in np.nonzero(self.colour == c)[0]:
                blk = self.blocks[i]
                x[blk] += self.Dinv[i] @ r[blk]
        return x

    def apply(self, r: np.ndarray) -> np.ndarray:
        """Ahat^{-1} r on the velocity part of the condensed layout (p part ignored, zero on output)."""
        b = r.copy()
        b[self.D.off_p:] = 0.0
        x = np.zeros_like(b)
        if not self.multiplicative:
            for blk, Di in zip(self.blocks, self.Dinv):
                x[blk] += Di @ b[blk]
            return x + self.E @ self.gmg.vcycle(self.E.T @ b)
        for _ in range(self.smooth):
            x = self._sweep(x, b, range(self.ncol))
        x = x + self.E @ self.gmg.vcycle(self.E.T @ (b - self.A @ x))
        for _ in range(self.smooth):
            x = self._sweep(x, b, range(self.ncol - 1, -1, -1))
        x[self.D.off_p:] = 0.0
        return x


class BlockPreconditioner:
    """Khat^{-1} of eq. (mhatinvfactor), applied with two Ahat^{-1} (reading R3)."""

    def __init__(self, D: system.Discretization, asp: ASP):
        self.D = D
        self.asp = asp
        K = system.condensed_system(D, np.zeros((D.mesh.elems.shape[0], D.sz["n_A"], D.sz["n_A"])))
        self.B = K[D.off_p:, :D.off_p]                          # pressure rows, velocity cols
        Mp = D.mats["Mp"]
        self.Sp_inv_diag = np.zeros(D.n_pres)
        self.Sp_inv_diag[(D.p_map - D.off_p).ravel()] = (D.nu / np.einsum("eii->ei", Mp)).ravel()

    def apply(self, r: np.ndarray) -> np.ndarray:
        D = self.D
        np_ = D.off_p
        a = self.asp.apply(r)
        zp = self.Sp_inv_diag * (r[np_:] - self.B @ a[:np_])
        t = r.copy()
        t[np_:] = 0.0
        t[:np_] -= self.B.T @ zp
        z = self.asp.apply(t)
        z[np_:] = zp
        return z

    def dense(self) -> np.ndarray:
        """The literal triple product of eq. (mhatinvfactor) with dense Ahat^{-1}."""
        D = self.D
        n = D.ndof
        np_ = D.off_p
        Ainv = np.zeros((np_, np_))
        for j in range(np_):
            e = np.zeros(n)
            e[j] = 1.0
            Ainv[:, j] = self.asp.apply(e)[:np_]
        B = self.B.toarray()
        Sinv = np.diag(self.Sp_inv_diag)
        I_u, I_p = np.eye(np_), np.eye(n - np_)
        left = np.block([[I_u, -Ainv @ B.T], [np.zeros((n - np_, np_)), I_p]])
        mid = np.block([[Ainv, np.zeros((np_, n - np_))], [np.zeros((n - np_, np_)), Sinv]])
        right = np.block([[I_u, np.zeros((np_, n - np_))], [-B @ Ainv, I_p]])
        return left @ mid @ right
