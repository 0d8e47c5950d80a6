"""GPU path (libmcs through its C-ABI) against the CPU oracle, element by element."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import workloads  # noqa: E402
from oracle import fem, manufactured, mesh, precond, system  # noqa: E402


@pytest.fixture(scope="module")
def mcs():
    from paper_2207_08481_gb300 import build
    build.build()
    import paper_2207_08481_gb300.mcs as m
    return m


def _handle(mcs, d, N, k, nu, **kw):
    h = mcs.Handle.structured(d, N, k, nu, **kw)
    h.condense()
    return h


def _oracle(d, N, k, nu):
    D = system.discretize(mesh.structured(d, N), k, nu)
    return D, system.condense(D)


CASES = [(2, 4, 2, 0.7), (2, 3, 3, 1.3), (2, 2, 4, 0.3), (3, 2, 2, 0.7), (3, 1, 3, 1.0), (3, 1, 4, 0.5)]


@pytest.mark.parametrize("d,N,k,nu", CASES)
def test_mesh_dofs_pattern_bit_exact(mcs, d, N, k, nu):
    h = _handle(mcs, d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=1)
    m = mesh.structured(d, N)
    facets, ef, sg, col = h.export_mesh()
    assert np.array_equal(facets, m.facets)
    assert np.array_equal(ef, m.elem_facets)
    assert np.array_equal(sg, m.signs)
    assert np.array_equal(col, mesh.colouring(m))
    D = system.discretize(m, k, nu)
    dm = h.export_dofmap()
    assert np.array_equal(dm[:, :D.sz["n_u"]], D.u_map)
    assert np.array_equal(dm[:, D.sz["n_u"]:D.sz["n_A"]], D.h_map)
    assert np.array_equal(dm[:, D.sz["n_A"]:], D.p_map)
    rp, cl = h.export_pattern()
    Kp = system.pattern(D)
    assert np.array_equal(rp, Kp.indptr) and np.array_equal(cl, Kp.indices)
    h.close()


@pytest.mark.parametrize("d,N,k,nu", CASES)
def test_condensed_element_matrices(mcs, d, N, k, nu):
    """A_T (eq. femSPmat), A^d_T and G_T (eq. Hcoeffs) against the literal oracle condensation."""
    h = _handle(mcs, d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=1)
    D, AT = _oracle(d, N, k, nu)
    ne, nA = AT.shape[0], AT.shape[1]
    P = h.element_matrices(0, ne)
    il = np.tril_indices(nA)
    ref = AT[:, il[0], il[1]]
    err = np.abs(P - ref).max(axis=1) / np.abs(ref).max(axis=1)
    assert err.max() < 1e-12, err.max()
    Ad_o, G_o, _ = system.bubble_condense(D, AT)
    Ad, G = h.schur(0, ne)
    # GPU coupling order is facet-major; map to the oracle's [u_d | uhat] order
    sz = D.sz
    o, c = system.local_split(D)
    pos = {v: i for i, v in enumerate(c)}
    perm = []
    for cc in range(h.sizes.n_c):
        f, t = divmod(cc, h.sizes.mF)
        perm.append(pos[f * sz["nF"] + t if t < sz["nF"] else sz["n_u"] + f * sz["n_hatF"] + (t - sz["nF"])])
    Ado = Ad_o[:, perm][:, :, perm]
    Go = G_o[:, :, perm]
    # rows of boundary facets are not kept (Dirichlet); every row of an interior facet is
    interior = np.repeat(D.mesh.int_rank[D.mesh.elem_facets] >= 0, h.sizes.mF, axis=1)
    assert np.array_equal(~np.isnan(Ad[:, :, 0]), interior)
    rows = np.broadcast_to(interior[:, :, None], Ad.shape)
    assert (np.abs(Ad[rows] - Ado[rows]).max() / np.abs(Ado).max()) < 1e-11
    assert (np.abs(G - Go).max() / np.abs(Go).max()) < 1e-10
    h.close()


@pytest.mark.parametrize("d,N,k,nu", CASES)
def test_apply_matches_oracle(mcs, d, N, k, nu):
    h = _handle(mcs, d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=1)
    D, AT = _oracle(d, N, k, nu)
    K = system.condensed_system(D, AT)
    rng = np.random.default_rng(11)
    for _ in range(2):
        x = rng.standard_normal(D.ndof)
        xt = torch.tensor(x, device="cuda")
        y = torch.zeros_like(xt)
        h.apply(xt, y)
        yo = K @ x
        assert np.abs(y.cpu().numpy() - yo).max() < 1e-12 * np.abs(yo).max()
    h.close()


@pytest.mark.parametrize("d,N,k,nu", [(2, 4, 2, 0.7), (2, 3, 3, 1.3), (2, 2, 4, 0.3), (3, 2, 2, 0.7), (3, 1, 3, 1.0),
                                     (3, 1, 4, 0.5)])
def test_apply_mixed_double_float(mcs, d, N, k, nu):
    """Mixed form: A_T as float pairs with double-float arithmetic, within 1e-12 of the FP64 K x."""
    h = _handle(mcs, d, N, k, nu, precision=mcs.MCS_MIXED, gmg_levels=1)
    D, AT = _oracle(d, N, k, nu)
    K = system.condensed_system(D, AT)
    x = np.random.default_rng(2).standard_normal(D.ndof)
    y = torch.zeros(D.ndof, dtype=torch.float64, device="cuda")
    h.apply(torch.tensor(x, device="cuda"), y)
    yo = K @ x
    assert np.abs(y.cpu().numpy() - yo).max() < 1e-12 * np.abs(yo).max()
    # the stored float pairs reconstruct A_T to the parity of the FP64 condensation (1e-12 relative per
    # element; the pairs themselves hold A_T to about 2^-48)
    P = h.element_matrices(0, AT.shape[0])
    il = np.tril_indices(AT.shape[1])
    ref = AT[:, il[0], il[1]]
    assert (np.abs(P - ref).max(axis=1) / np.abs(ref).max(axis=1)).max() < 1e-12
    h.close()


@pytest.mark.parametrize("d,N,k,nu,lev", [(2, 8, 2, 0.7, 2), (2, 4, 3, 1.0, 1), (2, 8, 2, 1.0, 3), (2, 2, 4, 0.3, 1),
                                          (2, 4, 4, 1.0, 2), (3, 2, 2, 1.0, 1), (3, 4, 2, 0.5, 2), (3, 1, 3, 1.0, 1),
                                          (3, 2, 3, 1.0, 1), (3, 1, 4, 0.5, 1)])
def test_precond_fp64_matches_oracle(mcs, d, N, k, nu, lev):
    """Khat^{-1} (eq. mhatinvfactor with the multiplicative ASP of Sec. 6.1) step for step."""
    h = _handle(mcs, d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=lev)
    D, AT = _oracle(d, N, k, nu)
    bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, precond.GMG(d, N, lev, nu)))
    rng = np.random.default_rng(5)
    r = rng.standard_normal(D.ndof)
    z = torch.zeros(D.ndof, dtype=torch.float64, device="cuda")
    h.precond(torch.tensor(r, device="cuda"), z)
    zo = bp.apply(r)
    assert np.abs(z.cpu().numpy() - zo).max() < 1e-11 * np.abs(zo).max()
    h.close()


@pytest.mark.parametrize("d,N,k,lev", [(2, 8, 2, 2), (3, 4, 2, 2), (3, 2, 3, 1)])
def test_precond_mixed_close_to_oracle(mcs, d, N, k, lev):
    """FP32 preconditioner (3D k = 2 runs the warp-per-facet smoother kernel) against the FP64 oracle."""
    h = _handle(mcs, d, N, k, 1.0, precision=mcs.MCS_MIXED, gmg_levels=lev)
    D, AT = _oracle(d, N, k, 1.0)
    bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, precond.GMG(d, N, lev, 1.0)))
    r = np.random.default_rng(5).standard_normal(D.ndof)
    z = torch.zeros(D.ndof, dtype=torch.float64, device="cuda")
    h.precond(torch.tensor(r, device="cuda"), z)
    zo = bp.apply(r)
    assert np.abs(z.cpu().numpy() - zo).max() < 1e-4 * np.abs(zo).max()
    h.close()


def _manufactured_rhs(h, d, nu):
    s = h.sizes
    xq = torch.zeros((s.ne * s.nq_load, d), dtype=torch.float64, device="cuda")
    h.load_points(xq)
    F = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    h.load_vector(workloads.manufactured_f(d, nu, xq), F)
    return F


@pytest.mark.parametrize("d,N,k,nu", [(2, 8, 2, 1.0), (2, 4, 3, 0.01), (3, 2, 2, 1.0), (3, 1, 4, 0.5)])
def test_load_vector(mcs, d, N, k, nu):
    """F = (f, phi^u) with the load rule of the dof contract (collapsed Gauss-Jacobi, k + 8 points per
    direction) on both sides: equal to rounding (of the dual BDM basis, about 1e-12 at k = 4), one cube
    included (reading R12)."""
    h = _handle(mcs, d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=1)
    D = system.discretize(mesh.structured(d, N), k, nu)
    Fo = system.load(D, manufactured.Manufactured(d, nu).f)
    F = _manufactured_rhs(h, d, nu).cpu().numpy()
    assert np.abs(F - Fo).max() < 3e-12 * np.abs(Fo).max()
    h.close()


def test_mass_velocity(mcs):
    d, N, k = 2, 4, 3
    h = _handle(mcs, d, N, k, 1.0, precision=mcs.MCS_FP64, gmg_levels=1)
    D = system.discretize(mesh.structured(d, N), k, 1.0)
    Mu = system.assemble(D.u_map, D.u_map, D.mats["Mu"], (D.ndof, D.ndof))
    c = np.zeros(D.ndof)
    c[:D.off_h] = workloads.random_coefficients(D.off_h, 3)
    F = torch.zeros(D.ndof, dtype=torch.float64, device="cuda")
    h.mass_velocity(torch.tensor(c, device="cuda"), F)
    Fo = Mu @ c
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-12 * np.abs(Fo).max()
    h.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_solve_c1_matches_oracle(mcs, prec, tol):
    """c1: 2D 8x8, k=2, nu=1, manufactured solution; relative error vs the oracle's direct solve."""
    d, N, k, nu = 2, 8, 2, 1.0
    p = mcs.MCS_FP64 if prec == "fp64" else mcs.MCS_MIXED
    h = _handle(mcs, d, N, k, nu, precision=p, rtol=1e-12 if prec == "fp64" else 1e-10)
    F = _manufactured_rhs(h, d, nu)
    x = torch.zeros_like(F)
    info = h.solve(F, x)
    D = system.discretize(mesh.structured(d, N), k, nu)
    Fo = system.load(D, manufactured.Manufactured(d, nu).f)
    xo, _, _ = system.solve_full(D, Fo)
    xo = system.mean_zero_pressure(D, xo)
    xg = x.cpu().numpy()
    n = D.off_p
    eu = np.linalg.norm(xg[:n] - xo[:n]) / np.linalg.norm(xo[:n])
    ep = np.linalg.norm(xg[n:] - xo[n:]) / np.linalg.norm(xo[n:])
    assert eu < tol and ep < tol, (eu, ep, info.iterations)
    assert info.status == 0 and info.iterations < 300
    h.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
@pytest.mark.parametrize("d,N,k,nu", [(2, 2, 4, 0.3), (2, 4, 4, 1.0), (3, 1, 4, 0.5), (3, 2, 3, 1.0), (3, 1, 2, 1.0)])
def test_solve_small_meshes_all_degrees(mcs, d, N, k, nu, prec, tol):
    """Solve against the oracle's direct solve for k = 3, 4 and the smallest meshes (one cube;
    2x2 squares), with the default multigrid hierarchy.  Both sides take the same right-hand side
    (the library's load vector, equal to the oracle's to rounding as tested above).  For k = 4 the
    error is about 100 times the preconditioned residual, so the tolerances of the solves are set
    below the plain-FP64 residual floor; the double-double refinement residual reaches them."""
    p = mcs.MCS_FP64 if prec == "fp64" else mcs.MCS_MIXED
    h = _handle(mcs, d, N, k, nu, precision=p, rtol=1e-13 if prec == "fp64" else 1e-12)
    F = _manufactured_rhs(h, d, nu)
    x = torch.zeros_like(F)
    info = h.solve(F, x, check=False)
    D = system.discretize(mesh.structured(d, N), k, nu)
    xo, _, _ = system.solve_full(D, F.cpu().numpy())
    xo = system.mean_zero_pressure(D, xo)
    xg = x.cpu().numpy()
    n = D.off_p
    eu = np.linalg.norm(xg[:n] - xo[:n]) / np.linalg.norm(xo[:n])
    ep = np.linalg.norm(xg[n:] - xo[n:]) / np.linalg.norm(xo[n:])
    assert info.status == 0, (info.status, info.iterations, info.refinements, info.rel_res_precond, eu, ep)
    assert eu < tol and ep < tol, (eu, ep, info.iterations)
    h.close()


def test_residual_double_double_is_exact_to_rounding(mcs):
    """mcs_residual: F - K x to within a few ulp of the exact value even where F and K x cancel.
    F is K x itself rounded to double, so the exact residual is only the rounding error of F; a
    residual formed in FP64 would be wrong in every digit.  The velocity rows are checked in
    exact rational arithmetic against the library's own stored A_T (x_p = 0)."""
    from fractions import Fraction
    d, N, k = 2, 2, 3
    h = _handle(mcs, d, N, k, 1.0, precision=mcs.MCS_FP64, gmg_levels=1)
    D = system.discretize(mesh.structured(d, N), k, 1.0)
    ne, nA = D.mesh.elems.shape[0], D.sz["n_A"]
    P = h.element_matrices(0, ne)
    AT = np.zeros((ne, nA, nA))
    il = np.tril_indices(nA)
    AT[:, il[0], il[1]] = P
    AT[:, il[1], il[0]] = P
    rng = np.random.default_rng(3)
    x = rng.standard_normal(D.ndof)
    x[D.off_p:] = 0.0
    xf = [Fraction(v) for v in x]
    Kx = [Fraction(0)] * D.ndof
    scale = [Fraction(0)] * D.ndof
    for T in range(ne):
        g = D.a_map[T]
        for i in range(nA):
            if g[i] < 0:
                continue
            acc, sc = Fraction(0), Fraction(0)
            for j in range(nA):
                if g[j] >= 0:
                    acc += Fraction(AT[T, i, j]) * xf[g[j]]
                    sc += abs(Fraction(AT[T, i, j]) * xf[g[j]])
            Kx[g[i]] += acc
            scale[g[i]] += sc
    F = np.array([float(v) for v in Kx])
    r = torch.zeros(D.ndof, dtype=torch.float64, device="cuda")
    h.residual(torch.tensor(F, device="cuda"), torch.tensor(x, device="cuda"), r)
    rg = r.cpu().numpy()
    nu_ = D.off_p
    for g in range(nu_):
        exact = Fraction(F[g]) - Kx[g]
        err = abs(Fraction(rg[g]) - exact)
        assert err <= 2 * abs(exact) * Fraction(2) ** -52 + Fraction(2) ** -100 * scale[g], (g, float(exact), rg[g])
    # pressure rows against the oracle's B (FP64 tables on both sides: rounding-level agreement)
    K = system.condensed_system(D)
    rp = (F - K @ x)[nu_:]
    assert np.abs(rg[nu_:] - rp).max() <= 1e-14 * np.abs(x).max() * np.abs(K[nu_:]).max() * 50
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_condense_batch_equals_per_problem(mcs, prec):
    """Several meshes and degrees in one persistent condensation launch give the same operators,
    bit for bit, as one launch per problem; a solve after the batched condensation is correct."""
    p = mcs.MCS_FP64 if prec == "fp64" else mcs.MCS_MIXED
    cases = [(3, 2, 2, 1.0), (2, 4, 3, 0.5), (3, 1, 4, 0.7), (2, 2, 4, 1.0)]
    ref = [_handle(mcs, d, N, k, nu, precision=p, gmg_levels=1) for d, N, k, nu in cases]
    bat = [mcs.Handle.structured(d, N, k, nu, precision=p, gmg_levels=1) for d, N, k, nu in cases]
    mcs.condense_batch(bat)
    for (d, N, k, nu), a, b in zip(cases, ref, bat):
        ne = a.sizes.ne
        assert np.array_equal(a.element_matrices(0, ne), b.element_matrices(0, ne))
        Ada, Ga = a.schur(0, ne)
        Adb, Gb = b.schur(0, ne)
        assert np.array_equal(np.nan_to_num(Ada, nan=7.0), np.nan_to_num(Adb, nan=7.0))
        assert np.array_equal(Ga, Gb)
        r = torch.tensor(np.random.default_rng(4).standard_normal(a.sizes.ndof), device="cuda")
        za, zb = torch.zeros_like(r), torch.zeros_like(r)
        a.precond(r, za)
        b.precond(r, zb)
        assert torch.equal(za, zb)
    d, N, k, nu = cases[1]
    h = bat[1]
    F = _manufactured_rhs(h, d, nu)
    x = torch.zeros_like(F)
    info = h.solve(F, x, check=False)
    assert info.status == 0
    D = system.discretize(mesh.structured(d, N), k, nu)
    xo, _, _ = system.solve_full(D, F.cpu().numpy())
    xo = system.mean_zero_pressure(D, xo)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-6
    for hh in ref + bat:
        hh.close()


@pytest.mark.parametrize("d,N,k,nu,lev", [(2, 8, 2, 0.7, 2), (3, 2, 2, 1.0, 1), (2, 4, 3, 1.0, 2)])
def test_precond_additive_matches_oracle(mcs, d, N, k, nu, lev):
    """Additive ASP (facet-block Jacobi plus E^d C^{-1} E^d^T, Sec. 6.1) inside eq. (mhatinvfactor)."""
    h = _handle(mcs, d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=lev, asp=1)
    D, AT = _oracle(d, N, k, nu)
    bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, precond.GMG(d, N, lev, nu), multiplicative=False))
    r = np.random.default_rng(6).standard_normal(D.ndof)
    z = torch.zeros(D.ndof, dtype=torch.float64, device="cuda")
    h.precond(torch.tensor(r, device="cuda"), z)
    zo = bp.apply(r)
    assert np.abs(z.cpu().numpy() - zo).max() < 1e-11 * np.abs(zo).max()
    h.close()


def test_solve_additive_c1(mcs):
    """c1 with the additive ASP: same solution as the oracle's direct solve, more iterations than the
    multiplicative ASP (as in the paper's comparison of the two)."""
    d, N, k, nu = 2, 8, 2, 1.0
    its = {}
    for asp in (0, 1):
        h = _handle(mcs, d, N, k, nu, precision=mcs.MCS_FP64, rtol=1e-12, asp=asp)
        F = _manufactured_rhs(h, d, nu)
        x = torch.zeros_like(F)
        info = h.solve(F, x)
        its[asp] = info.iterations
        D = system.discretize(mesh.structured(d, N), k, nu)
        xo, _, _ = system.solve_full(D, F.cpu().numpy())
        xo = system.mean_zero_pressure(D, xo)
        xg = x.cpu().numpy()
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-10
        h.close()
    assert its[1] > its[0]


class _ExactC:
    """C = Abar^{-1} on the mesh's own P1 space (what a single-level hierarchy solves)."""

    def __init__(self, m, nu):
        A = precond.abar(m, nu).toarray()
        self.inv = np.linalg.inv(A) if A.shape[0] else np.zeros((0, 0))

    def vcycle(self, b):
        return self.inv @ b


@pytest.mark.parametrize("d,N,k,nu", [(2, 4, 3, 0.8), (3, 2, 2, 1.0)])
def test_general_mesh_perturbed(mcs, d, N, k, nu):
    """mcs_setup_mesh on a mesh with displaced interior vertices (general affine simplices):
    numbering bit-exact, A_T, K^-1-preconditioner and solve against the oracle on the same mesh."""
    m0 = mesh.structured(d, N)
    coords = m0.coords.copy()
    inner = mesh.interior_vertices(m0)
    coords[inner] += np.random.default_rng(9).uniform(-0.2, 0.2, (len(inner), d)) / N
    m = mesh.structured(d, N, coords=coords)
    h = mcs.Handle.from_mesh(d, coords, m.elems, k, nu, precision=mcs.MCS_FP64, rtol=1e-13)
    h.condense()
    facets, ef, sg, col = h.export_mesh()
    assert np.array_equal(facets, m.facets) and np.array_equal(ef, m.elem_facets) and np.array_equal(sg, m.signs)
    D = system.discretize(m, k, nu)
    AT = system.condense(D)
    il = np.tril_indices(AT.shape[1])
    P = h.element_matrices(0, AT.shape[0])
    assert np.abs(P - AT[:, il[0], il[1]]).max() < 1e-12 * np.abs(AT).max()
    bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, _ExactC(m, nu)))
    r = np.random.default_rng(2).standard_normal(D.ndof)
    z = torch.zeros(D.ndof, dtype=torch.float64, device="cuda")
    h.precond(torch.tensor(r, device="cuda"), z)
    zo = bp.apply(r)
    assert np.abs(z.cpu().numpy() - zo).max() < 1e-11 * np.abs(zo).max()
    c = np.zeros(D.ndof)
    c[:D.off_h] = workloads.random_coefficients(D.off_h, 5)
    F = torch.zeros(D.ndof, dtype=torch.float64, device="cuda")
    h.mass_velocity(torch.tensor(c, device="cuda"), F)
    x = torch.zeros_like(F)
    info = h.solve(F, x, check=False)
    xo, _, _ = system.solve_full(D, F.cpu().numpy())
    xo = system.mean_zero_pressure(D, xo)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-10, (info.status, info.iterations)
    h.close()


@pytest.mark.parametrize("d,N,k,nu", [(2, 3, 2, 0.7), (2, 2, 4, 1.3), (3, 1, 3, 0.5), (3, 2, 2, 1.0)])
def test_recover_stress_matches_oracle(mcs, d, N, k, nu):
    """sigma_h and omega_h of the local problems (eq. projection) for the same coefficient vector,
    evaluated at the oracle's quadrature points of every element."""
    h = _handle(mcs, d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=1)
    m = mesh.structured(d, N)
    D = system.discretize(m, k, nu)
    x = np.random.default_rng(8).standard_normal(D.ndof)
    sig, om = system.recover_stress(D, x)
    X = m.coords[m.elems]
    E = fem.element_data(X, m.signs, k)
    so = np.einsum("ej,eqjab->eqab", sig, E.S)
    wo = np.einsum("ej,eqjab->eqab", om, E.W)
    J0 = (X[0, 1:, :] - X[0, :1, :]).T
    xhat = np.linalg.solve(J0, (E.xq[0] - X[0, 0]).T).T
    ne, nq = X.shape[0], xhat.shape[0]
    sg = torch.zeros((ne, nq, d, d), dtype=torch.float64, device="cuda")
    om_g = torch.zeros_like(sg)
    h.recover_stress(torch.tensor(x, device="cuda"), xhat, sg, om_g)
    assert np.abs(sg.cpu().numpy() - so).max() < 1e-11 * np.abs(so).max()
    assert np.abs(om_g.cpu().numpy() - wo).max() < 1e-10 * np.abs(wo).max()
    h.close()
