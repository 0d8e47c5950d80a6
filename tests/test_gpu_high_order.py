"""Degrees k = 5, 6 (the top of the batched degree sweep of 3D 16^3 x 6 tetrahedra, k = 1..6) through
the C-ABI against the oracle, on meshes small enough for its dense element algebra.

At these degrees one element's data no longer fits in shared memory (3D k = 6: 6 MB of condensation
workspace, 707 KB of packed operator, 176 KB of facet stream per facet), so the library runs its
unstaged kernels: condensation in a global workspace, the facet step reading the facet stream from
global memory, the chunked double-float apply and double-double residual, and the element prologue and
epilogue reading G and A_oo^{-1} from global memory.  The interior BDM moments of the dof contract are
L2-orthonormal, which keeps the element matrices well scaled at these degrees."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import workloads  # noqa: E402
from oracle import manufactured, mesh, precond, system  # noqa: E402

CASES = [(2, 2, 5, 0.7), (2, 2, 6, 1.0), (3, 1, 5, 0.8), (3, 1, 6, 1.0)]
_ORACLE = {}


@pytest.fixture(scope="module")
def mcs():
    from paper_2207_08481_gb300 import build
    build.build()
    import paper_2207_08481_gb300.mcs as m
    return m


def _oracle(d, N, k, nu):
    key = (d, N, k, nu)
    if key not in _ORACLE:
        D = system.discretize(mesh.structured(d, N), k, nu)
        _ORACLE[key] = (D, system.condense(D))
    return _ORACLE[key]


def _tol(k):
    return 1e-10      # rounding of the element algebra at 3D k = 6 reaches a few 1e-11


@pytest.mark.parametrize("d,N,k,nu", CASES)
def test_numbering_and_element_matrices(mcs, d, N, k, nu):
    h = mcs.Handle.structured(d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=1)
    h.condense()
    D, AT = _oracle(d, N, k, nu)
    dm = h.export_dofmap()
    assert np.array_equal(dm[:, :D.sz["n_u"]], D.u_map)
    assert np.array_equal(dm[:, D.sz["n_u"]:D.sz["n_A"]], D.h_map)
    ne, nA = AT.shape[0], AT.shape[1]
    P = h.element_matrices(0, ne)
    il = np.tril_indices(nA)
    ref = AT[:, il[0], il[1]]
    assert (np.abs(P - ref).max(axis=1) / np.abs(ref).max(axis=1)).max() < _tol(k)
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("d,N,k,nu", CASES)
def test_apply_and_residual(mcs, d, N, k, nu, prec):
    """K x (FP64, or the chunked double-float apply) and the double-double residual F - K x."""
    h = mcs.Handle.structured(d, N, k, nu, precision=mcs.MCS_FP64 if prec == "fp64" else mcs.MCS_MIXED,
                              gmg_levels=1)
    h.condense()
    D, AT = _oracle(d, N, k, nu)
    K = system.condensed_system(D, AT)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(D.ndof)
    xt = torch.tensor(x, device="cuda")
    y = torch.zeros_like(xt)
    h.apply(xt, y)
    yo = K @ x
    assert np.abs(y.cpu().numpy() - yo).max() < _tol(k) * np.abs(yo).max()
    F = torch.tensor(rng.standard_normal(D.ndof), device="cuda")
    r = torch.zeros_like(F)
    h.residual(F, xt, r)
    ro = F.cpu().numpy() - yo
    assert np.abs(r.cpu().numpy() - ro).max() < _tol(k) * np.abs(yo).max()
    h.close()


@pytest.mark.parametrize("d,N,k,nu", CASES)
def test_precond_fp64_matches_oracle(mcs, d, N, k, nu):
    """Khat^{-1} step for step (unstaged facet step, prologue and epilogue)."""
    h = mcs.Handle.structured(d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=1)
    h.condense()
    D, AT = _oracle(d, N, k, nu)
    bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, precond.GMG(d, N, 1, nu)))
    r = np.random.default_rng(5).standard_normal(D.ndof)
    z = torch.zeros(D.ndof, dtype=torch.float64, device="cuda")
    h.precond(torch.tensor(r, device="cuda"), z)
    zo = bp.apply(r)
    assert np.abs(z.cpu().numpy() - zo).max() < _tol(k) * np.abs(zo).max()
    h.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
@pytest.mark.parametrize("d,N,k,nu", CASES)
def test_solve_matches_oracle(mcs, d, N, k, nu, prec, tol):
    """Manufactured solve (tight tolerance, double-double residual) against the oracle's direct solve of
    the condensed system; both sides take the library's load vector."""
    h = mcs.Handle.structured(d, N, k, nu, precision=mcs.MCS_FP64 if prec == "fp64" else mcs.MCS_MIXED,
                              gmg_levels=1, rtol=1e-13 if prec == "fp64" else 1e-12, maxit=4000)
    h.condense()
    s = h.sizes
    xq = torch.zeros((s.ne * s.nq_load, d), dtype=torch.float64, device="cuda")
    h.load_points(xq)
    F = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    h.load_vector(workloads.manufactured_f(d, nu, xq), F)
    D, AT = _oracle(d, N, k, nu)
    Fo = system.load(D, manufactured.Manufactured(d, nu).f)
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-11 * np.abs(Fo).max()
    x = torch.zeros_like(F)
    info = h.solve(F, x, check=False)
    xo = system.mean_zero_pressure(D, system.solve_condensed(D, F.cpu().numpy(), AT))
    xg = x.cpu().numpy()
    n = D.off_p
    eu = np.linalg.norm(xg[:n] - xo[:n]) / np.linalg.norm(xo[:n])
    ep = np.linalg.norm(xg[n:] - xo[n:]) / np.linalg.norm(xo[n:])
    assert info.status == 0, (info.status, info.iterations, eu, ep)
    assert eu < tol and ep < tol, (eu, ep, info.iterations)
    h.close()
