"""Parity at the full sizes of the c2 and c3 workloads, in the launch configuration bench.py times
(mixed form, the same multigrid hierarchy): mesh, facets, signs, colouring and dof numbering
bit-exact; element operators and load-vector entries of sampled elements against the oracle computed
element by element; and properties of the solve that hold at any size."""
from types import SimpleNamespace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import workloads  # noqa: E402
from oracle import fem, manufactured, mesh, system  # noqa: E402

CASES = {"c2": (2, 256, 3, 1e-2, 5), "c3": (3, 32, 2, 1.0, 4), "c4k1": (3, 16, 1, 1.0, -1)}


@pytest.fixture(scope="module")
def mcs():
    from paper_2207_08481_gb300 import build
    build.build()
    import paper_2207_08481_gb300.mcs as m
    return m


def _coupling_perm(sz, n_c, mF):
    """GPU coupling order (facet-major: nF facet moments, then uhat modes) -> oracle [u_d | uhat]."""
    d = sz["d"]
    o = np.arange((d + 1) * sz["nF"], sz["n_u"])
    c = np.concatenate([np.arange((d + 1) * sz["nF"]), np.arange(sz["n_u"], sz["n_u"] + sz["n_hat"])])
    pos = {v: i for i, v in enumerate(c)}
    perm = []
    for cc in range(n_c):
        f, t = divmod(cc, mF)
        perm.append(pos[f * sz["nF"] + t if t < sz["nF"] else sz["n_u"] + f * sz["n_hatF"] + (t - sz["nF"])])
    return np.array(perm), o


@pytest.mark.parametrize("name", ["c2", "c3", "c4k1"])
def test_fullsize_numbering_and_sampled_operators(mcs, name):
    d, N, k, nu, lev = CASES[name]
    h = mcs.Handle.structured(d, N, k, nu, precision=mcs.MCS_MIXED, gmg_levels=lev)
    h.condense()
    m = mesh.structured(d, N)
    facets, ef, sg, col = h.export_mesh()
    assert np.array_equal(facets, m.facets) and np.array_equal(ef, m.elem_facets) and np.array_equal(sg, m.signs)
    if name == "c2":  # the greedy colouring in Python takes minutes at the 3D size
        assert np.array_equal(col, mesh.colouring(m))
    sz = fem.local_sizes(d, k)
    _, u_map, h_map, p_map = system.dof_maps(m, k)[:4]
    dm = h.export_dofmap()
    assert np.array_equal(dm, np.concatenate([u_map, h_map, p_map], axis=1))
    ne = m.elems.shape[0]
    T = np.unique(np.concatenate([[0, ne - 1], np.random.default_rng(0).choice(ne, 14, replace=False)]))
    X = m.coords[m.elems[T]]
    mats = fem.element_matrices(X, m.signs[T], k, nu)
    AT = system.condense(SimpleNamespace(mats=mats, sz=sz))
    Ad_o, G_o, _ = system.bubble_condense(SimpleNamespace(mesh=SimpleNamespace(dim=d), sz=sz), AT)
    perm, _ = _coupling_perm(sz, h.sizes.n_c, h.sizes.mF)
    il = np.tril_indices(AT.shape[1])
    for i, t in enumerate(T):
        P = h.element_matrices(int(t), 1)[0]
        ref = AT[i][il]
        assert np.abs(P - ref).max() < 1e-12 * np.abs(ref).max()      # float pairs: ~2^-48
        Ad, G = h.schur(int(t), 1)
        Ado = Ad_o[i][perm][:, perm]
        rows = ~np.isnan(Ad[0][:, 0])
        assert np.abs(Ad[0][rows] - Ado[rows]).max() < 2e-6 * np.abs(Ado).max()   # FP32 copies
        if sz["n_bub"]:
            assert np.abs(G[0] - G_o[i][:, perm]).max() < 2e-6 * np.abs(G_o[i]).max()
    if not sz["n_bub"]:     # k = 1: no bubbles, so no load entry is owned by a single element
        h.close()
        return
    # load vector: bubble entries (owned by one element) of the sampled elements
    s = h.sizes
    xq = torch.zeros((s.ne * s.nq_load, d), dtype=torch.float64, device="cuda")
    h.load_points(xq)
    F = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    h.load_vector(workloads.manufactured_f(d, nu, xq), F)
    Fo = fem.load_vector(X, m.signs[T], k, manufactured.Manufactured(d, nu).f)
    nfd = (d + 1) * sz["nF"]
    Fg = F.cpu().numpy()
    for i, t in enumerate(T):
        got = Fg[s.off_o + t * s.n_bub + np.arange(s.n_bub)]
        ref = Fo[i, nfd:nfd + s.n_bub]
        assert np.abs(got - ref).max() < 1e-10 * max(np.abs(Fo).max(), 1e-300)
    h.close()


def test_fullsize_c2_solve_properties(mcs):
    """c2 exactly as bench.py runs it: converged to the preconditioned tolerance within the bounded
    iteration band, pressure of zero mean (reading R6), and a small true residual."""
    d, N, k, nu, lev = CASES["c2"]
    h = mcs.Handle.structured(d, N, k, nu, precision=mcs.MCS_MIXED, gmg_levels=lev, rtol=1e-8)
    h.condense()
    s = h.sizes
    xq = torch.zeros((s.ne * s.nq_load, d), dtype=torch.float64, device="cuda")
    h.load_points(xq)
    F = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    h.load_vector(workloads.manufactured_f(d, nu, xq), F)
    x = torch.zeros_like(F)
    info = h.solve(F, x)
    assert info.status == 0 and info.rel_res_precond <= 1e-8 and info.iterations < 120
    p0 = x[s.off_p::s.n_p].cpu().numpy()          # constant pressure mode per element (equal areas)
    assert abs(p0.sum()) <= 1e-10 * np.abs(p0).sum()
    r = torch.zeros_like(F)
    h.residual(F, x, r)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(F)) < 1e-4
    h.close()


def test_fullsize_c4_lowest_order_solve_properties(mcs):
    """The k = 1 member of c4 as bench.py runs it (3D 16^3 x 6, mixed form, default hierarchy):
    converged, zero-mean pressure, small true residual; the rotation fluxes are part of x."""
    d, N, k, nu, lev = CASES["c4k1"]
    h = mcs.Handle.structured(d, N, k, nu, precision=mcs.MCS_MIXED, maxit=8000)
    h.condense()
    s = h.sizes
    assert (s.nhF, s.mF, s.n_bub) == (3, 6, 0)
    xq = torch.zeros((s.ne * s.nq_load, d), dtype=torch.float64, device="cuda")
    h.load_points(xq)
    F = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    h.load_vector(workloads.manufactured_f(d, nu, xq), F)
    x = torch.zeros_like(F)
    info = h.solve(F, x)
    assert info.status == 0 and info.rel_res_precond <= 1e-8
    p = x[s.off_p:].cpu().numpy()                 # P^0 pressure, equal volumes
    assert abs(p.sum()) <= 1e-10 * np.abs(p).sum()
    r = torch.zeros_like(F)
    h.residual(F, x, r)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(F)) < 1e-4
    h.close()
