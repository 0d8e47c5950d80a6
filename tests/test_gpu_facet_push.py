"""The forward facet sweeps with a maintained residual (mcs_options.facet_push = 1): the sweeps before the
coarse correction keep, per facet and side, the partial residual of that side's element and push each
block update into the facets of both elements, so that the residual for E^d^T needs no pass of its own.
It is the same block Gauss-Seidel sweep (Corollary aux_pc_mult) as the row-product form
(facet_push = 0), summed in another order: the two agree to rounding, and the FP64 form matches the
oracle's K-hat^{-1} step for step."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

from oracle import mesh, precond, system  # noqa: E402


@pytest.fixture(scope="module")
def mcs():
    from paper_2207_08481_gb300 import build
    build.build()
    import paper_2207_08481_gb300.mcs as m
    return m


def _precond(h, r):
    z = torch.zeros_like(r)
    h.precond(r, z)
    torch.cuda.synchronize()
    return z.cpu().numpy()


# (dim, N, k, nu, precision, GMG levels, outflow): every case runs the maintained-residual sweep
CASES = [(3, 2, 2, 0.7, "fp64", 2, 0), (3, 4, 2, 1.0, "fp64", 3, 0), (3, 2, 2, 1.0, "fp64", 2, 1),
         (2, 4, 4, 0.3, "fp64", 2, 0), (2, 4, 5, 1.0, "fp64", 2, 0), (2, 2, 6, 1.0, "fp64", 1, 0),
         (3, 4, 2, 1.0, "mixed", 3, 0), (3, 2, 2, 1.0, "mixed", 2, 1), (2, 2, 6, 0.5, "mixed", 1, 0)]


@pytest.mark.parametrize("d,N,k,nu,prec,lev,out", CASES)
def test_push_equals_row_products(mcs, d, N, k, nu, prec, lev, out):
    p = mcs.MCS_FP64 if prec == "fp64" else mcs.MCS_MIXED
    hp = mcs.Handle.structured(d, N, k, nu, precision=p, gmg_levels=lev, outflow=out)
    hr = mcs.Handle.structured(d, N, k, nu, precision=p, gmg_levels=lev, outflow=out, facet_push=0)
    for h in (hp, hr):
        h.condense()
    assert hp.sizes.push_warps > 0 and hr.sizes.push_warps == 0
    rng = np.random.default_rng(11)
    r = torch.tensor(rng.standard_normal(hp.sizes.ndof), device="cuda")
    zp, zr = _precond(hp, r), _precond(hr, r)
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert np.abs(zp - zr).max() <= tol * np.abs(zr).max()
    # deterministic: one writer per (facet, side) slot and launch
    assert np.array_equal(zp, _precond(hp, r))
    hp.close()
    hr.close()


@pytest.mark.parametrize("d,N,k,nu,lev", [(3, 2, 2, 0.7, 2), (3, 4, 2, 1.3, 3), (2, 4, 4, 0.3, 2)])
def test_push_fp64_matches_oracle(mcs, d, N, k, nu, lev):
    """K-hat^{-1} (eq. mhatinvfactor, multiplicative ASP of Sec. 6.1) step for step against the oracle."""
    h = mcs.Handle.structured(d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=lev)
    h.condense()
    assert h.sizes.push_warps > 0
    D = system.discretize(mesh.structured(d, N), k, nu)
    AT = system.condense(D)
    bp = precond.BlockPreconditioner(D, precond.ASP(D, AT, precond.GMG(d, N, lev, nu)))
    r = np.random.default_rng(5).standard_normal(D.ndof)
    z = _precond(h, torch.tensor(r, device="cuda"))
    zo = bp.apply(r)
    assert np.abs(z - zo).max() < 1e-11 * np.abs(zo).max()
    h.close()


def test_push_solve_same_iterations(mcs):
    """A full mixed solve on 3D 8^3 x 6, k = 2: both forms of the sweep converge alike."""
    its = {}
    for fp in (1, 0):
        h = mcs.Handle.structured(3, 8, 2, 1.0, precision=mcs.MCS_MIXED, rtol=1e-8, etol=1e-8, facet_push=fp)
        h.condense()
        s = h.sizes
        c = torch.tensor(np.random.default_rng(2).standard_normal(s.off_p), device="cuda")
        F = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
        h.mass_velocity(c, F)
        x = torch.zeros_like(F)
        info = h.solve(F, x, check=False)
        assert info.status == 0
        its[fp] = (info.iterations, x.cpu().numpy())
        h.close()
    assert abs(its[1][0] - its[0][0]) <= 8
    xa, xb = its[1][1], its[0][1]
    assert np.linalg.norm(xa - xb) <= 1e-8 * np.linalg.norm(xb)
