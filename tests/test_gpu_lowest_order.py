"""Lowest-order variant (k = 1, Sec. 7, three dimensions) through the C-ABI against the oracle.

The rotation lives in H(div) with one flux dof per facet (the third entry of each facet's uhat
block), is kept after condensation, couples through kappa(omega) and carries nu (div omega,
div eta); the embedding adds curl(ubar).  Every step of the path is compared element by element."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import workloads  # noqa: E402
from oracle import fem, manufactured, mesh, precond, system  # noqa: E402

K = 1


@pytest.fixture(scope="module")
def mcs():
    from paper_2207_08481_gb300 import build
    build.build()
    import paper_2207_08481_gb300.mcs as m
    return m


def _handle(mcs, N, nu, **kw):
    h = mcs.Handle.structured(3, N, K, nu, **kw)
    h.condense()
    return h


def _oracle(N, nu):
    D = system.discretize(mesh.structured(3, N), K, nu)
    return D, system.condense(D)


def test_two_dimensional_lowest_order_is_unsupported(mcs):
    with pytest.raises(mcs.McsError) as e:
        mcs.Handle.structured(2, 4, 1, 1.0)
    assert e.value.code == mcs.MCS_ERR_UNSUPPORTED


@pytest.mark.parametrize("N", [1, 2, 3])
def test_dofs_pattern_bit_exact(mcs, N):
    h = _handle(mcs, N, 1.0, precision=mcs.MCS_FP64, gmg_levels=1)
    m = mesh.structured(3, N)
    D = system.discretize(m, K, 1.0)
    s = h.sizes
    assert (s.nF, s.nhF, s.n_bub, s.ndof) == (3, 3, 0, D.ndof)
    dm = h.export_dofmap()
    assert np.array_equal(dm[:, :D.sz["n_u"]], D.u_map)
    assert np.array_equal(dm[:, D.sz["n_u"]:D.sz["n_A"]], D.h_map)
    assert np.array_equal(dm[:, D.sz["n_A"]:], D.p_map)
    rp, cl = h.export_pattern()
    Kp = system.pattern(D)
    assert np.array_equal(rp, Kp.indptr) and np.array_equal(cl, Kp.indices)
    h.close()


@pytest.mark.parametrize("N,nu", [(2, 0.7), (3, 1.3)])
def test_condensed_element_matrices(mcs, N, nu):
    """A_T over (u, uhat, omega) against the literal oracle condensation; with no bubbles the
    facet blocks of the stream are A_T itself in facet-major order."""
    h = _handle(mcs, N, nu, precision=mcs.MCS_FP64, gmg_levels=1)
    D, AT = _oracle(N, nu)
    ne, nA = AT.shape[0], AT.shape[1]
    P = h.element_matrices(0, ne)
    il = np.tril_indices(nA)
    ref = AT[:, il[0], il[1]]
    assert (np.abs(P - ref).max(axis=1) / np.abs(ref).max(axis=1)).max() < 1e-12
    Ad, G = h.schur(0, ne)
    assert G.shape[1] == 0
    perm = [f * 3 + t if t < 3 else 12 + f * 3 + (t - 3) for f in range(4) for t in range(6)]
    Ado = AT[:, perm][:, :, perm]
    interior = np.repeat(D.mesh.int_rank[D.mesh.elem_facets] >= 0, 6, axis=1)
    assert np.array_equal(~np.isnan(Ad[:, :, 0]), interior)
    rows = np.broadcast_to(interior[:, :, None], Ad.shape)
    assert np.abs(Ad[rows] - Ado[rows]).max() < 1e-11 * np.abs(Ado).max()
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_apply_matches_oracle(mcs, prec):
    p = mcs.MCS_FP64 if prec == "fp64" else mcs.MCS_MIXED
    h = _handle(mcs, 3, 0.7, precision=p, gmg_levels=1)
    D, AT = _oracle(3, 0.7)
    Kc = system.condensed_system(D, AT)
    x = np.random.default_rng(11).standard_normal(D.ndof)
    y = torch.zeros(D.ndof, dtype=torch.float64, device="cuda")
    h.apply(torch.tensor(x, device="cuda"), y)
    yo = Kc @ x
    assert np.abs(y.cpu().numpy() - yo).max() < 1e-12 * np.abs(yo).max()
    h.close()


@pytest.mark.parametrize("N,nu,lev", [(2, 1.0, 1), (4, 0.5, 2)])
def test_precond_fp64_matches_oracle(mcs, N, nu, lev):
    """Khat^{-1} with facet blocks of 6 (3 BDM^1, 2 tangential, 1 rotation flux), E^d with the curl
    rows and the GMG V-cycle, step for step."""
    h = _handle(mcs, N, nu, precision=mcs.MCS_FP64, gmg_levels=lev)
    D, AT = _oracle(N, nu)
    bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, precond.GMG(3, N, lev, nu)))
    r = np.random.default_rng(5).standard_normal(D.ndof)
    z = torch.zeros(D.ndof, dtype=torch.float64, device="cuda")
    h.precond(torch.tensor(r, device="cuda"), z)
    zo = bp.apply(r)
    assert np.abs(z.cpu().numpy() - zo).max() < 1e-11 * np.abs(zo).max()
    h.close()


def test_precond_mixed_and_additive(mcs):
    N, lev = 4, 2
    D, AT = _oracle(N, 1.0)
    r = np.random.default_rng(7).standard_normal(D.ndof)
    for asp, tol, prec in [(0, 1e-4, mcs.MCS_MIXED), (1, 1e-11, mcs.MCS_FP64)]:
        h = _handle(mcs, N, 1.0, precision=prec, gmg_levels=lev, asp=asp)
        bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, precond.GMG(3, N, lev, 1.0),
                                                        multiplicative=(asp == 0)))
        z = torch.zeros(D.ndof, dtype=torch.float64, device="cuda")
        h.precond(torch.tensor(r, device="cuda"), z)
        zo = bp.apply(r)
        assert np.abs(z.cpu().numpy() - zo).max() < tol * np.abs(zo).max()
        h.close()


def _rhs(h, nu):
    s = h.sizes
    xq = torch.zeros((s.ne * s.nq_load, 3), dtype=torch.float64, device="cuda")
    h.load_points(xq)
    F = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    h.load_vector(workloads.manufactured_f(3, nu, xq), F)
    return F


def test_load_vector(mcs):
    h = _handle(mcs, 2, 0.8, precision=mcs.MCS_FP64, gmg_levels=1)
    D = system.discretize(mesh.structured(3, 2), K, 0.8)
    Fo = system.load(D, manufactured.Manufactured(3, 0.8).f)
    F = _rhs(h, 0.8).cpu().numpy()
    # both sides integrate f with the load rule of the dof contract (k + 8 points per direction)
    assert np.abs(F - Fo).max() < 1e-13 * np.abs(Fo).max()
    h.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
@pytest.mark.parametrize("N,nu", [(2, 1.0), (4, 0.6)])
def test_solve_matches_oracle(mcs, N, nu, prec, tol):
    p = mcs.MCS_FP64 if prec == "fp64" else mcs.MCS_MIXED
    h = _handle(mcs, N, nu, precision=p, rtol=1e-13 if prec == "fp64" else 1e-12, maxit=4000)
    F = _rhs(h, nu)
    x = torch.zeros_like(F)
    info = h.solve(F, x, check=False)
    D = system.discretize(mesh.structured(3, N), K, nu)
    xo = system.mean_zero_pressure(D, system.solve_condensed(D, F.cpu().numpy()))
    xg = x.cpu().numpy()
    n = D.off_p
    eu = np.linalg.norm(xg[:n] - xo[:n]) / np.linalg.norm(xo[:n])
    ep = np.linalg.norm(xg[n:] - xo[n:]) / np.linalg.norm(xo[n:])
    assert info.status == 0, (info.status, info.iterations, info.rel_res_precond)
    assert eu < tol and ep < tol, (eu, ep, info.iterations)
    h.close()


def test_recover_stress(mcs):
    """sigma_h of the local problems (eq. projection) with the rotation flux dofs taken from x."""
    N, nu = 2, 0.9
    h = _handle(mcs, N, nu, precision=mcs.MCS_FP64, gmg_levels=1)
    m = mesh.structured(3, N)
    D = system.discretize(m, K, nu)
    x = np.random.default_rng(8).standard_normal(D.ndof)
    sig, _ = system.recover_stress(D, x)
    X = m.coords[m.elems]
    E = fem.element_data(X, m.signs, K)
    so = np.einsum("ej,eqjab->eqab", sig, E.S)
    J0 = (X[0, 1:, :] - X[0, :1, :]).T
    xhat = np.linalg.solve(J0, (E.xq[0] - X[0, 0]).T).T
    sg = torch.zeros((X.shape[0], xhat.shape[0], 3, 3), dtype=torch.float64, device="cuda")
    xt = torch.tensor(x, device="cuda")
    h.recover_stress(xt, xhat, sg)
    assert np.abs(sg.cpu().numpy() - so).max() < 1e-11 * np.abs(so).max()
    with pytest.raises(mcs.McsError) as e:
        h.recover_stress(xt, xhat, sg, torch.zeros_like(sg))
    assert e.value.code == mcs.MCS_ERR_UNSUPPORTED
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_condense_batch_with_lowest_order(mcs, prec):
    """k = 1 and k = 2, 3 problems in one persistent condensation launch: bit-identical operators."""
    p = mcs.MCS_FP64 if prec == "fp64" else mcs.MCS_MIXED
    cases = [(3, 2, 1, 1.0), (3, 2, 2, 0.7), (3, 1, 3, 1.0), (3, 3, 1, 0.4)]
    ref = [mcs.Handle.structured(d, N, k, nu, precision=p, gmg_levels=1) for d, N, k, nu in cases]
    for a in ref:
        a.condense()
    bat = [mcs.Handle.structured(d, N, k, nu, precision=p, gmg_levels=1) for d, N, k, nu in cases]
    mcs.condense_batch(bat)
    for a, b in zip(ref, bat):
        ne = a.sizes.ne
        assert np.array_equal(a.element_matrices(0, ne), b.element_matrices(0, ne))
        r = torch.tensor(np.random.default_rng(4).standard_normal(a.sizes.ndof), device="cuda")
        za, zb = torch.zeros_like(r), torch.zeros_like(r)
        a.precond(r, za)
        b.precond(r, zb)
        assert torch.equal(za, zb)
    for hh in ref + bat:
        hh.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_h2_stabilisation_parity(mcs, prec, tol):
    """lo_stab = 1: coefficient nu h_T^2 of (div omega, div eta)_T (reading R21(d')); A_T and the
    solve against the oracle with the same weight."""
    p = mcs.MCS_FP64 if prec == "fp64" else mcs.MCS_MIXED
    N, nu = 4, 0.8
    h = _handle(mcs, N, nu, precision=p, lo_stab=1, rtol=1e-13 if prec == "fp64" else 1e-12, maxit=4000)
    D = system.discretize(mesh.structured(3, N), K, nu, lo_stab=1)
    AT = system.condense(D)
    P = h.element_matrices(0, AT.shape[0])
    il = np.tril_indices(AT.shape[1])
    ref = AT[:, il[0], il[1]]
    assert (np.abs(P - ref).max(axis=1) / np.abs(ref).max(axis=1)).max() < (1e-12 if prec == "fp64" else 1e-13)
    F = _rhs(h, nu)
    x = torch.zeros_like(F)
    info = h.solve(F, x, check=False)
    xo = system.mean_zero_pressure(D, system.solve_condensed(D, F.cpu().numpy(), AT))
    xg = x.cpu().numpy()
    n = D.off_p
    assert info.status == 0, (info.status, info.iterations)
    assert np.linalg.norm(xg[:n] - xo[:n]) / np.linalg.norm(xo[:n]) < tol
    assert np.linalg.norm(xg[n:] - xo[n:]) / np.linalg.norm(xo[n:]) < tol
    h.close()
