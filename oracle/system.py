"""Global systems of the MCS method (oracle side, test infrastructure).

* ``Discretization`` holds the mesh, the dof maps of the contract and all element
  matrices (eq. bigfemSPmat), computed batch-wise over elements.
* ``full_system`` assembles the uncondensed saddle-point matrix over
  (sigma, omega, u, uhat, p) of eq. (bigfemSPmat); ``solve_full`` adds one
  Lagrange multiplier for int p = 0 (pure Dirichlet boundary, reading R6) and
  solves it with a sparse direct solver.
* ``condense`` forms, element by element, A_T = A^div - B_sigma M^{-1} B_sigma^T
  of Sec. 4.2 (static condensation of sigma, omega) literally, with a dense
  solve of the local saddle-point block; ``condensed_system`` assembles
  K = [[A, B^T], [B, 0]] of eq. (femSPmat).
* ``bubble_condense`` forms A_oo, A_od, the "double" Schur complement
  A^d = A_dd - A_do A_oo^{-1} A_od and the harmonic-extension map
  G = A_oo^{-1} A_od (eqs. Hcoeffs, factorSsigma).

Global vector layout (dof contract): [u_d | u_o | uhat | p], with u_d indexed by
(interior facet rank, mode), u_o by (element, bubble), uhat by (interior facet
rank, tangent, mode), p by (element, mode).  For the lowest-order variant (k = 1,
Sec. 7) u_o is empty and each facet's uhat block is (tangent 1, tangent 2, flux of
the H(div) rotation omega); the rotation is condensed away with sigma for k >= 2
only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, mesh as meshmod


@dataclass
class Discretization:
    mesh: meshmod.Mesh
    k: int
    nu: float
    sz: dict
    # local -> global maps (-1: Dirichlet, removed)
    u_map: np.ndarray      # [ne, n_u]
    h_map: np.ndarray      # [ne, n_hat]
    p_map: np.ndarray      # [ne, n_p]
    n_dd: int              # total facet-BDM dofs
    n_oo: int              # total bubble dofs
    n_hat: int
    n_pres: int
    mats: dict = field(default_factory=dict)

    @property
    def off_o(self):
        return self.n_dd

    @property
    def off_h(self):
        return self.n_dd + self.n_oo

    @property
    def off_p(self):
        return self.n_dd + self.n_oo + self.n_hat

    @property
    def ndof(self):
        return self.off_p + self.n_pres

    @property
    def a_map(self):
        """local (u, uhat) -> global index, [ne, n_A]."""
        return np.concatenate([self.u_map, self.h_map], axis=1)


def dof_maps(m: meshmod.Mesh, k: int):
    """Local -> global maps.  BDM facet dofs live on the interior facets and, when the mesh marks
    Gamma_Ntilde, also on its facets (u_n free there, eq. stokes_NT); uhat dofs on interior facets only
    (uhat = 0 on Gamma_D and Gamma_Ntilde)."""
    d = m.dim
    sz = fem.local_sizes(d, k)
    ne = m.elems.shape[0]
    nF, nb, nhF, npp = sz["nF"], sz["n_bub"], sz["n_hatF"], sz["n_p"]
    nint = m.n_int
    n_dd = m.n_udof * nF
    n_oo = ne * nb
    n_hat = nint * nhF
    n_pres = ne * npp
    u_map = -np.ones((ne, sz["n_u"]), dtype=np.int64)
    h_map = -np.ones((ne, sz["n_hat"]), dtype=np.int64)
    urank = m.u_rank
    for f in range(d + 1):
        ru = urank[m.elem_facets[:, f]]
        oku = ru >= 0
        for j in range(nF):
            u_map[oku, f * nF + j] = ru[oku] * nF + j
        r = m.int_rank[m.elem_facets[:, f]]
        ok = r >= 0
        for j in range(nhF):
            h_map[ok, f * nhF + j] = n_dd + n_oo + r[ok] * nhF + j
    for b in range(nb):
        u_map[:, (d + 1) * nF + b] = n_dd + np.arange(ne) * nb + b
    p_map = n_dd + n_oo + n_hat + np.arange(ne)[:, None] * npp + np.arange(npp)[None, :]
    return sz, u_map, h_map, p_map, n_dd, n_oo, n_hat, n_pres


def discretize(m: meshmod.Mesh, k: int, nu: float, batch: int = 2048, lo_stab: int = 0) -> Discretization:
    """lo_stab: weight of the k = 1 stabilisation (fem.stabilisation_weight)."""
    sz, u_map, h_map, p_map, n_dd, n_oo, n_hat, n_pres = dof_maps(m, k)
    D = Discretization(m, k, nu, sz, u_map, h_map, p_map, n_dd, n_oo, n_hat, n_pres)
    X = m.coords[m.elems]
    parts = []
    for s in range(0, X.shape[0], batch):
        parts.append(fem.element_matrices(X[s:s + batch], m.signs[s:s + batch], k, nu, lo_stab))
    D.mats = {key: np.concatenate([p[key] for p in parts]) for key in parts[0]}
    return D


def load(D: Discretization, f, batch: int = 2048) -> np.ndarray:
    """Global load vector (f, phi^u) in the condensed layout (zeros outside u)."""
    X = D.mesh.coords[D.mesh.elems]
    Floc = np.concatenate([fem.load_vector(X[s:s + batch], D.mesh.signs[s:s + batch], D.k, f)
                           for s in range(0, X.shape[0], batch)])
    F = np.zeros(D.ndof)
    ok = D.u_map >= 0
    np.add.at(F, D.u_map[ok], Floc[ok])
    return F


def _coo(rows_map, cols_map, blocks):
    """Scatter element blocks [E, r, c] with maps [E, r], [E, c] (-1 dropped)."""
    E_, r, c = blocks.shape
    R = np.broadcast_to(rows_map[:, :, None], (E_, r, c))
    C = np.broadcast_to(cols_map[:, None, :], (E_, r, c))
    ok = (R >= 0) & (C >= 0)
    return R[ok], C[ok], blocks[ok]


def assemble(rows_map, cols_map, blocks, shape):
    R, C, V = _coo(rows_map, cols_map, blocks)
    return sp.csr_matrix((V, (R, C)), shape=shape)


def _psi0(d: int) -> float:
    """Value of the constant orthonormal basis function on T_hat (|T_hat| = 1/d!)."""
    return math.sqrt(math.factorial(d))


def pressure_constraint(D: Discretization) -> np.ndarray:
    """c with c.x = int_Omega p_h dx (condensed layout).

    p_0 = psi_0 is constant, so int_T p_i = (p_i, p_0)_T / psi_0."""
    c = np.zeros(D.ndof)
    intp = D.mats["Mp"][:, :, 0] / _psi0(D.mesh.dim)
    np.add.at(c, D.p_map.ravel(), intp.ravel())
    return c


def full_system(D: Discretization):
    """Uncondensed symmetric saddle-point matrix over [sigma | omega | condensed layout]."""
    ne = D.mesh.elems.shape[0]
    ns, nw = D.sz["n_sigma"], D.sz["n_omega"]
    s_map = np.arange(ne)[:, None] * ns + np.arange(ns)[None, :]
    w_map = ne * ns + np.arange(ne)[:, None] * nw + np.arange(nw)[None, :]
    off = ne * (ns + nw)
    n = off + D.ndof
    um, hm, pm = D.u_map, D.h_map, D.p_map
    shift = lambda a: np.where(a >= 0, a + off, -1)
    R, C, V = [], [], []

    def add(rm, cm, blk, sym=True):
        r, c, v = _coo(rm, cm, blk)
        R.append(r); C.append(c); V.append(v)
        if sym:
            R.append(c); C.append(r); V.append(v)

    add(s_map, s_map, -D.mats["M"], sym=False)
    add(w_map, s_map, D.mats["Bw"])
    add(shift(um), s_map, D.mats["Bu"])
    add(shift(hm), s_map, D.mats["Bh"])
    add(shift(um), shift(um), D.mats["Adiv"], sym=False)
    if "Shat" in D.mats:                                        # k = 1: nu (div omega, div eta)
        add(shift(hm), shift(hm), D.mats["Shat"], sym=False)
    add(shift(pm), shift(um), D.mats["Bp"])
    Kf = sp.csr_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=(n, n))
    return Kf, off


def _solve_pinned(K: sp.spmatrix, rhs: np.ndarray, pin: int | None) -> np.ndarray:
    """Direct solve of the singular saddle-point system whose kernel is the constant pressure:
    the constant-mode coefficient `pin` is fixed to 0 (row and column removed); the caller
    removes the pressure mean afterwards (pure Dirichlet boundary, reading R6).  pin = None: the
    system is nonsingular (Gamma_Ntilde marked) and is solved as it is."""
    if pin is None:
        return spla.spsolve(K.tocsc(), rhs)
    n = K.shape[0]
    keep = np.ones(n, dtype=bool)
    keep[pin] = False
    idx = np.nonzero(keep)[0]
    Kr = K.tocsr()[idx][:, idx].tocsc()
    sol = np.zeros(n)
    sol[idx] = spla.spsolve(Kr, rhs[idx])
    return sol


def solve_full(D: Discretization, F: np.ndarray):
    """Direct solve of the uncondensed system; returns (x_condensed_layout, sigma, omega).
    The pressure is determined up to a constant; use mean_zero_pressure on the result."""
    Kf, off = full_system(D)
    n = Kf.shape[0]
    rhs = np.concatenate([np.zeros(off), F])
    sol = _solve_pinned(Kf, rhs, None if D.mesh.outflow is not None else off + int(D.p_map[0, 0]))
    ne = D.mesh.elems.shape[0]
    ns, nw = D.sz["n_sigma"], D.sz["n_omega"]
    sigma = sol[:ne * ns].reshape(ne, ns)
    omega = sol[ne * ns:off].reshape(ne, nw)
    return sol[off:n], sigma, omega


# ---------------------------------------------------------------- condensation
def condense(D: Discretization) -> np.ndarray:
    """A_T = A^div - B_sigma M^{-1} B_sigma^T per element, [ne, n_A, n_A] (Sec. 4.2)."""
    m = D.mats
    ns, nw, nu_, nh = D.sz["n_sigma"], D.sz["n_omega"], D.sz["n_u"], D.sz["n_hat"]
    ne = m["M"].shape[0]
    Mloc = np.zeros((ne, ns + nw, ns + nw))
    Mloc[:, :ns, :ns] = -m["M"]
    Mloc[:, :ns, ns:] = np.transpose(m["Bw"], (0, 2, 1))
    Mloc[:, ns:, :ns] = m["Bw"]
    Bs = np.zeros((ne, nu_ + nh, ns + nw))
    Bs[:, :nu_, :ns] = m["Bu"]
    Bs[:, nu_:, :ns] = m["Bh"]
    Aext = np.zeros((ne, nu_ + nh, nu_ + nh))
    Aext[:, :nu_, :nu_] = m["Adiv"]
    if "Shat" in m:
        Aext[:, nu_:, nu_:] = m["Shat"]
    return Aext - Bs @ np.linalg.solve(Mloc, np.transpose(Bs, (0, 2, 1)))


def condensed_system(D: Discretization, AT: np.ndarray | None = None):
    """K = [[A, B^T], [B, 0]] of eq. (femSPmat) in the condensed layout."""
    AT = condense(D) if AT is None else AT
    am = D.a_map
    A = assemble(am, am, AT, (D.ndof, D.ndof))
    Bp = assemble(D.p_map, D.u_map, D.mats["Bp"], (D.ndof, D.ndof))
    return (A + Bp + Bp.T).tocsr()


def solve_condensed(D: Discretization, F: np.ndarray, AT=None):
    """Direct solve of K x = F (eq. femSPmat); pressure up to a constant (see solve_full)."""
    K = condensed_system(D, AT)
    return _solve_pinned(K, F, None if D.mesh.outflow is not None else int(D.p_map[0, 0]))


def local_split(D: Discretization):
    """Index sets of the element's (u, uhat) vector: bubbles (o) and coupling dofs (d = facet BDM + uhat)."""
    d = D.mesh.dim
    nF, nb, nu_, nh = D.sz["nF"], D.sz["n_bub"], D.sz["n_u"], D.sz["n_hat"]
    o = np.arange((d + 1) * nF, nu_)
    c = np.concatenate([np.arange((d + 1) * nF), np.arange(nu_, nu_ + nh)])
    return o, c


def bubble_condense(D: Discretization, AT: np.ndarray):
    """(A^d_T, G_T = A_oo^{-1} A_od, A_oo) per element; A^d_T indexed by the coupling dofs."""
    o, c = local_split(D)
    Aoo = AT[:, o][:, :, o]
    Aoc = AT[:, o][:, :, c]
    Acc = AT[:, c][:, :, c]
    G = np.linalg.solve(Aoo, Aoc)
    Ad = Acc - np.transpose(Aoc, (0, 2, 1)) @ G
    return Ad, G, Aoo


def mean_zero_pressure(D: Discretization, x: np.ndarray) -> np.ndarray:
    """Subtract the mean value of p_h (returns a copy)."""
    x = x.copy()
    d = D.mesh.dim
    area = float(np.sum(np.abs(D.mats["Mp"][:, 0, 0])) / _psi0(d) ** 2)   # sum |T|
    mean = pressure_constraint(D) @ x / area
    x[D.p_map[:, 0]] -= mean / _psi0(d)
    return x


def recover_stress(D: Discretization, x: np.ndarray):
    """Local solves of eq. (projection): (sigma_T, omega_T) from the (u, uhat) part of x.

    Row sigma of eq. (bigfemSPmat): -M sigma + Bw^T omega + Bu^T u + Bh^T uhat = 0;
    row omega: Bw sigma = 0."""
    m = D.mats
    ns, nw = D.sz["n_sigma"], D.sz["n_omega"]
    ne = m["M"].shape[0]
    xu = np.where(D.u_map >= 0, x[np.maximum(D.u_map, 0)], 0.0)
    xh = np.where(D.h_map >= 0, x[np.maximum(D.h_map, 0)], 0.0)
    Mloc = np.zeros((ne, ns + nw, ns + nw))
    Mloc[:, :ns, :ns] = -m["M"]
    Mloc[:, :ns, ns:] = np.transpose(m["Bw"], (0, 2, 1))
    Mloc[:, ns:, :ns] = m["Bw"]
    rhs = np.zeros((ne, ns + nw))
    rhs[:, :ns] = -(np.einsum("eij,ei->ej", m["Bu"], xu) + np.einsum("eij,ei->ej", m["Bh"], xh))
    sol = np.linalg.solve(Mloc, rhs[..., None])[..., 0]
    return sol[:, :ns], sol[:, ns:]


def pattern(D: Discretization) -> sp.csr_matrix:
    """Structural sparsity of K = [[A, B^T], [B, 0]]: every element couples its (u, uhat) dofs
    with each other and its u dofs with its pressure dofs (entries of value 1, no cancellation)."""
    ne = D.mesh.elems.shape[0]
    am = D.a_map
    nA, nu_, npp = am.shape[1], D.u_map.shape[1], D.p_map.shape[1]
    A = assemble(am, am, np.ones((ne, nA, nA)), (D.ndof, D.ndof))
    B = assemble(D.p_map, D.u_map, np.ones((ne, npp, nu_)), (D.ndof, D.ndof))
    P = (A + B + B.T).tocsr()
    P.data[:] = 1.0
    P.sort_indices()
    return P
