"""Outflow boundary Gamma_Ntilde (eq. stokes_NT, Lemma outflow) through the C-ABI against the oracle.

The library numbers the coupling facets (interior and outflow) in facet order and keeps phantom uhat
slots on outflow facets (identity rows, zero); the oracle has no uhat there.  Every comparison maps
the oracle's layout into the library's and checks that the phantom slots stay zero."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import workloads  # noqa: E402
from oracle import mesh, precond, system  # noqa: E402


@pytest.fixture(scope="module")
def mcs():
    from paper_2207_08481_gb300 import build
    build.build()
    import paper_2207_08481_gb300.mcs as m
    return m


def _oracle(d, N, k, nu):
    D = system.discretize(mesh.with_outflow(mesh.structured(d, N)), k, nu)
    return D, system.condense(D)


def _dev_index(D, h):
    """Library index of every oracle dof, and the library's phantom uhat slots."""
    m, sz, s = D.mesh, D.sz, h.sizes
    nhF = sz["n_hatF"]
    idx = np.arange(D.ndof)
    assert (s.n_dd, s.n_oo, s.off_h) == (D.n_dd, D.n_oo, D.off_h)
    phantom = []
    for F in np.nonzero(m.udof)[0]:
        r, ri = m.u_rank[F], m.int_rank[F]
        if ri >= 0:
            idx[D.off_h + ri * nhF + np.arange(nhF)] = s.off_h + r * nhF + np.arange(nhF)
        else:
            phantom += list(s.off_h + r * nhF + np.arange(nhF))
    idx[D.off_p:] = s.off_p + np.arange(D.n_pres)
    return idx, np.array(phantom, dtype=np.int64)


def _phantom_mask(D, AT):
    """The oracle's A_T with the rows and columns of the outflow facets' uhat replaced by the identity."""
    m, sz = D.mesh, D.sz
    A = AT.copy()
    nu_, nhF = sz["n_u"], sz["n_hatF"]
    for T in range(A.shape[0]):
        for f in range(m.dim + 1):
            if m.outflow[m.elem_facets[T, f]]:
                loc = nu_ + f * nhF + np.arange(nhF)
                A[T, loc, :] = 0.0
                A[T, :, loc] = 0.0
                A[T, loc, loc] = 1.0
    return A


CASES = [(2, 4, 2, 0.7, 2), (2, 4, 3, 1.3, 1), (3, 2, 2, 1.0, 1)]


@pytest.mark.parametrize("d,N,k,nu,lev", CASES)
def test_outflow_numbering_and_element_matrices(mcs, d, N, k, nu, lev):
    h = mcs.Handle.structured(d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=lev, outflow=1)
    h.condense()
    D, AT = _oracle(d, N, k, nu)
    idx, phantom = _dev_index(D, h)
    assert h.sizes.ndof == D.ndof + len(phantom)
    dm = h.export_dofmap()
    sz = D.sz
    assert np.array_equal(dm[:, :sz["n_u"]], D.u_map)
    hm = D.h_map
    assert np.array_equal(dm[:, sz["n_u"]:sz["n_A"]][hm >= 0], idx[hm[hm >= 0]])
    assert np.isin(dm[:, sz["n_u"]:sz["n_A"]][hm < 0], np.concatenate([phantom, [-1]])).all()
    assert np.array_equal(dm[:, sz["n_A"]:], idx[D.p_map])
    P = h.element_matrices(0, AT.shape[0])
    ref = _phantom_mask(D, AT)
    il = np.tril_indices(AT.shape[1])
    assert np.abs(P - ref[:, il[0], il[1]]).max() < 1e-12 * np.abs(AT).max()
    h.close()


@pytest.mark.parametrize("d,N,k,nu,lev", CASES + [(2, 8, 2, 1.0, 3), (3, 4, 2, 0.5, 2)])
def test_outflow_apply_and_precond(mcs, d, N, k, nu, lev):
    """K x and Khat^{-1} r (ASP with facet blocks on the outflow facets, E^d with pi_0, GMG on the
    penalised Abar) step for step, FP64."""
    h = mcs.Handle.structured(d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=lev, outflow=1)
    h.condense()
    D, AT = _oracle(d, N, k, nu)
    idx, phantom = _dev_index(D, h)
    Kc = system.condensed_system(D, AT)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(D.ndof)
    xd = torch.zeros(h.sizes.ndof, dtype=torch.float64, device="cuda")
    xd[torch.tensor(idx, device="cuda")] = torch.tensor(x, device="cuda")
    y = torch.zeros_like(xd)
    h.apply(xd, y)
    yo = Kc @ x
    yg = y.cpu().numpy()
    assert np.abs(yg[idx] - yo).max() < 1e-12 * np.abs(yo).max()
    assert np.abs(yg[phantom]).max(initial=0.0) == 0.0
    bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, precond.GMG(d, N, lev, nu, outflow_k=k)))
    z = torch.zeros_like(xd)
    h.precond(xd, z)
    zo = bp.apply(x)
    zg = z.cpu().numpy()
    assert np.abs(zg[idx] - zo).max() < 1e-11 * np.abs(zo).max()
    assert np.abs(zg[phantom]).max(initial=0.0) == 0.0
    h.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
@pytest.mark.parametrize("d,N,k,nu", [(2, 8, 2, 1.0), (3, 4, 2, 0.8)])
def test_outflow_solve(mcs, d, N, k, nu, prec, tol):
    """F = M_u c (c ~ N(0, 1) on the velocity dofs): the solve against the oracle's direct solve, with
    no pressure mean removed on either side."""
    p = mcs.MCS_FP64 if prec == "fp64" else mcs.MCS_MIXED
    h = mcs.Handle.structured(d, N, k, nu, precision=p, outflow=1, rtol=1e-12, maxit=3000)
    h.condense()
    D, AT = _oracle(d, N, k, nu)
    idx, phantom = _dev_index(D, h)
    c = np.zeros(D.ndof)
    c[:D.off_h] = workloads.random_coefficients(D.off_h, 5)
    cd = torch.zeros(h.sizes.ndof, dtype=torch.float64, device="cuda")
    cd[torch.tensor(idx, device="cuda")] = torch.tensor(c, device="cuda")
    F = torch.zeros_like(cd)
    h.mass_velocity(cd, F)
    x = torch.zeros_like(F)
    info = h.solve(F, x, check=False)
    assert info.status == 0, (info.status, info.iterations)
    xo = system.solve_condensed(D, F.cpu().numpy()[idx], AT)
    xg = x.cpu().numpy()
    n = D.off_p
    assert np.linalg.norm(xg[idx][:n] - xo[:n]) / np.linalg.norm(xo[:n]) < tol
    assert np.linalg.norm(xg[idx][n:] - xo[n:]) / np.linalg.norm(xo[n:]) < tol
    assert np.abs(xg[phantom]).max(initial=0.0) < 1e-14 * np.abs(xg).max()
    h.close()
