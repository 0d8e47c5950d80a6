"""Structured simplicial meshes and the dof-numbering contract (oracle side, test infrastructure).

The paper works on a quasi-uniform simplicial triangulation with facet sets
(Sec. 2, Notation).  The synthetic workloads use the unit square / cube split
into N^d cells, each cell split into d! Kuhn simplices; such meshes are nested
under uniform refinement, which the geometric multigrid for the conforming
auxiliary space relies on.

Contract (shared in words with the CUDA library, never in code):
* vertex (i, j[, l]) in [0, N]^d has id i + (N+1)*(j + (N+1)*l), coordinates /N;
* cell (i, j[, l]) has id i + N*(j + N*l); its d! simplices are indexed by the
  permutations pi of (0..d-1) in lexicographic order; element id = cell*d! + perm;
  element vertices: v_0 = cell corner, v_{m+1} = v_m + e_{pi(m)}.  These are in
  ascending global id;
* local facet f of an element is opposite local vertex f, its vertices in
  ascending order;
* global facets are the distinct sorted vertex tuples in lexicographic order;
  interior facets (two elements) keep that relative order;
* the facet normal n_F is the unit vector with det[e_1..e_{d-1}, n_F] > 0 for the
  edge vectors e_m = x_{w_m} - x_{w_0} of the sorted facet vertices w;
* orientation sign s_{T,f} = +1 if n_F points out of T, else -1;
* facet colouring: greedy in interior-facet order, a facet takes the smallest
  colour not used by an already coloured interior facet that shares an element.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    dim: int
    N: int
    coords: np.ndarray        # [nv, d]
    elems: np.ndarray         # [ne, d+1] sorted vertex ids
    facets: np.ndarray        # [nf, d] sorted vertex ids, lexicographic
    elem_facets: np.ndarray   # [ne, d+1] global facet of local facet f
    facet_elems: np.ndarray   # [nf, 2] adjacent elements (second = -1 on the boundary)
    interior: np.ndarray      # [nf] bool
    int_rank: np.ndarray      # [nf] rank among interior facets, -1 on boundary
    normals: np.ndarray       # [nf, d] n_F
    signs: np.ndarray         # [ne, d+1] s_{T,f}
    outflow: np.ndarray | None = None   # [nf] bool, facets on Gamma_Ntilde (None: all Dirichlet)

    @property
    def n_int(self) -> int:
        return int(self.interior.sum())

    @property
    def udof(self) -> np.ndarray:
        """Facets that carry BDM (normal-flux) dofs: interior facets and facets on Gamma_Ntilde."""
        return self.interior if self.outflow is None else (self.interior | self.outflow)

    @property
    def u_rank(self) -> np.ndarray:
        """Rank of each BDM-dof facet in facet order (-1 elsewhere); equals int_rank without outflow."""
        if self.outflow is None:
            return self.int_rank
        r = -np.ones(len(self.interior), dtype=np.int64)
        r[self.udof] = np.arange(int(self.udof.sum()))
        return r

    @property
    def n_udof(self) -> int:
        return int(self.udof.sum())


def structured(dim: int, N: int, coords: np.ndarray | None = None) -> Mesh:
    """Kuhn triangulation of [0,1]^dim with N cells per direction.

    ``coords`` may override the vertex coordinates (e.g. a perturbed mesh with
    the same connectivity)."""
    d = dim
    nv1 = N + 1
    if coords is None:
        grids = np.meshgrid(*[np.arange(nv1)] * d, indexing="ij")
        # vertex id i + nv1*(j + nv1*l): first index fastest
        idx = np.stack([g.transpose(tuple(range(d))[::-1]).ravel() for g in grids], axis=1)
        coords = idx.astype(np.float64) / N
    perms = list(itertools.permutations(range(d)))
    cells = np.stack(np.meshgrid(*[np.arange(N)] * d, indexing="ij"), axis=-1)
    cells = cells.transpose(tuple(range(d))[::-1] + (d,)).reshape(-1, d)   # cell id order
    stride = np.array([nv1 ** a for a in range(d)])
    elems = []
    for c in cells:
        for p in perms:
            v = c.copy()
            ids = [int(v @ stride)]
            for m in range(d):
                v = v.copy()
                v[p[m]] += 1
                ids.append(int(v @ stride))
            elems.append(ids)
    elems = np.array(elems, dtype=np.int64)
    return build(dim, N, coords, elems)


def build(dim: int, N: int, coords: np.ndarray, elems: np.ndarray) -> Mesh:
    d = dim
    ne = elems.shape[0]
    assert np.all(np.diff(elems, axis=1) > 0), "element vertices must be ascending"
    loc = [[v for v in range(d + 1) if v != f] for f in range(d + 1)]
    ftup = np.stack([elems[:, loc[f]] for f in range(d + 1)], axis=1)  # [ne, d+1, d]
    flat = ftup.reshape(-1, d)
    facets, inv = np.unique(flat, axis=0, return_inverse=True)
    inv = inv.reshape(ne, d + 1)
    nf = facets.shape[0]
    facet_elems = -np.ones((nf, 2), dtype=np.int64)
    for T in range(ne):
        for f in range(d + 1):
            F = inv[T, f]
            if facet_elems[F, 0] < 0:
                facet_elems[F, 0] = T
            else:
                facet_elems[F, 1] = T
    interior = facet_elems[:, 1] >= 0
    int_rank = -np.ones(nf, dtype=np.int64)
    int_rank[interior] = np.arange(int(interior.sum()))
    # facet normals
    X = coords[facets]                          # [nf, d, d]
    E = X[:, 1:, :] - X[:, :1, :]               # [nf, d-1, d]
    if d == 2:
        e = E[:, 0, :]
        n = np.stack([-e[:, 1], e[:, 0]], axis=1)
    else:
        n = np.cross(E[:, 0, :], E[:, 1, :])
    n = n / np.linalg.norm(n, axis=1, keepdims=True)
    # orientation signs
    signs = np.zeros((ne, d + 1), dtype=np.int64)
    for f in range(d + 1):
        F = inv[:, f]
        out = coords[facets[F, 0]] - coords[elems[:, f]]
        signs[:, f] = np.where(np.einsum("ij,ij->i", n[F], out) > 0, 1, -1)
    return Mesh(dim, N, coords, elems, facets, inv, facet_elems, interior, int_rank, n, signs)


def colouring(mesh: Mesh) -> np.ndarray:
    """Greedy colouring of the BDM-dof facets (interior facets, plus Gamma_Ntilde facets if marked);
    returns colour per facet rank."""
    ints = np.nonzero(mesh.udof)[0]
    rank = mesh.u_rank
    colour = -np.ones(len(ints), dtype=np.int64)
    for r, F in enumerate(ints):
        used = set()
        for T in mesh.facet_elems[F]:
            if T < 0:
                continue
            for G in mesh.elem_facets[T]:
                g = rank[G]
                if g >= 0 and colour[g] >= 0:
                    used.add(int(colour[g]))
        c = 0
        while c in used:
            c += 1
        colour[r] = c
    return colour


def interior_vertices(mesh: Mesh) -> np.ndarray:
    """Ids of the free vertices of the conforming space, ascending: vertices not on the boundary of
    the unit square/cube, plus (with Gamma_Ntilde marked) those inside the face x_1 = 1."""
    N = mesh.N
    idx = np.rint(mesh_index(mesh)).astype(np.int64)
    inside = np.all((idx > 0) & (idx < N), axis=1)
    if mesh.outflow is not None:
        inside |= (idx[:, 0] == N) & np.all((idx[:, 1:] > 0) & (idx[:, 1:] < N), axis=1)
    return np.nonzero(inside)[0]


def with_outflow(m: Mesh) -> Mesh:
    """Marks the face x_1 = 1 of the unit square / cube as Gamma_Ntilde (outflow, Sec. 6.2: u_t = 0
    and ((sigma + p I) n).n = 0); the other faces stay Dirichlet."""
    idx = mesh_index(m)
    on = np.all(idx[m.facets][:, :, 0] == m.N, axis=1) & ~m.interior
    m.outflow = on
    return m


def mesh_index(mesh: Mesh) -> np.ndarray:
    """Grid multi-index (i, j[, l]) of every vertex, from its id."""
    N1 = mesh.N + 1
    ids = np.arange(mesh.coords.shape[0])
    out = []
    for _ in range(mesh.dim):
        out.append(ids % N1)
        ids = ids // N1
    return np.stack(out, axis=1)


def factorial(d: int) -> int:
    return math.factorial(d)
