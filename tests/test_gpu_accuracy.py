"""Accuracy of the timed solves: both forms, with exactly the options bench.py times, against the
oracle's direct solve of the condensed system (eq. femSPmat), on meshes of the benchmark's element
types that the oracle finishes in seconds; and at full size, properties that hold at any size.

The bars are those of the two forms: relative L2 error of u and of p <= 1e-8 (mixed: FP32
preconditioner, FP64 outer Krylov) and <= 1e-10 (FP64 form).  The stopping rule is the relative
preconditioned residual 1e-8 together with the error bound of mcs_options.etol: with nu = 1e-2 and a
pressure-dominated right-hand side the residual test alone leaves velocity errors near 5e-6.
Both sides take the library's load vector (its own parity is tested separately), so the comparison is
that of the solver.

Where nu << 1 the discrete problem itself is only defined to a few 1e-10 (k = 3, nu = 1e-2) or 1e-9
(k = 4, nu = 1e-3) in FP64: the oracle's two routes to the same solution, the direct solve of the
condensed system and that of the full system of eq. (bigfemSPmat), differ by that much.  There the
bar is the larger of the form's bar and four times that oracle-internal difference."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import bench  # noqa: E402  (the timed options; bench.py imports only the standard library at load)
import workloads  # noqa: E402
from oracle import mesh, system  # noqa: E402


@pytest.fixture(scope="module")
def mcs():
    from paper_2207_08481_gb300 import build
    build.build()
    import paper_2207_08481_gb300.mcs as m
    return m


def _rhs(h, d, nu):
    s = h.sizes
    xq = torch.zeros((s.ne * s.nq_load, d), dtype=torch.float64, device="cuda")
    h.load_points(xq)
    F = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    h.load_vector(workloads.manufactured_f(d, nu, xq), F)
    return F


CASES = list(bench.ORACLE_CASES.values()) + [
    dict(dim=2, N=16, k=4, nu=1e-3, levels=1),    # strongest velocity amplification measured (6,400x)
    dict(dim=3, N=4, k=3, nu=0.1, levels=2),
]

_FLOORS = {}


def _oracle_floor(c, F):
    """Relative difference (u, p) between the oracle's condensed and full direct solves of the case."""
    key = tuple(sorted(c.items()))
    if key not in _FLOORS:
        D = system.discretize(mesh.structured(c["dim"], c["N"]), c["k"], c["nu"])
        Fh = F.cpu().numpy()
        xc = system.mean_zero_pressure(D, system.solve_condensed(D, Fh))
        xf, _, _ = system.solve_full(D, Fh)
        xf = system.mean_zero_pressure(D, xf)
        n = D.off_p
        _FLOORS[key] = (np.linalg.norm(xc[:n] - xf[:n]) / np.linalg.norm(xf[:n]),
                        np.linalg.norm(xc[n:] - xf[n:]) / np.linalg.norm(xf[n:]))
    return _FLOORS[key]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=lambda i: "{dim}D-N{N}-k{k}-nu{nu}".format(**CASES[i]))
def oracle_case(request, mcs):
    c = CASES[request.param]
    h = mcs.Handle.structured(c["dim"], c["N"], c["k"], c["nu"], precision=mcs.MCS_FP64, gmg_levels=c["levels"])
    h.condense()
    F = _rhs(h, c["dim"], c["nu"])
    h.close()
    D = system.discretize(mesh.structured(c["dim"], c["N"]), c["k"], c["nu"])
    xo = system.mean_zero_pressure(D, system.solve_condensed(D, F.cpu().numpy()))
    return c, F, xo, D.off_p


@pytest.mark.parametrize("form", ["mixed", "fp64"])
def test_timed_solve_meets_the_bar(mcs, oracle_case, form):
    c, F, xo, n = oracle_case
    h = mcs.Handle.structured(c["dim"], c["N"], c["k"], c["nu"], gmg_levels=c["levels"], **bench.FORMS[form])
    h.condense()
    x = torch.zeros_like(F)
    info = h.solve(F, x)
    xg = x.cpu().numpy()
    eu = np.linalg.norm(xg[:n] - xo[:n]) / np.linalg.norm(xo[:n])
    ep = np.linalg.norm(xg[n:] - xo[n:]) / np.linalg.norm(xo[n:])
    bar = bench.ERR_BAR[form]
    assert info.status == 0 and info.rel_res_precond <= bench.FORMS[form]["rtol"]
    assert 0 < info.err_est <= bar
    bar_u = bar_p = bar
    if eu > bar or ep > bar:
        fu, fp = _oracle_floor(c, F)
        bar_u, bar_p = max(bar, 4 * fu), max(bar, 4 * fp)
    assert eu <= bar_u and ep <= bar_p, (eu, ep, bar_u, bar_p, info.err_est, info.iterations, info.refinements)
    h.close()


def test_residual_alone_misses_the_velocity_bar(mcs, oracle_case):
    """Why the timed rule carries the error bound: rtol 1e-8 alone gives velocity errors far above 1e-8
    for the nu = 1e-2 and 1e-3 cases (the error bound then has work to do)."""
    c, F, xo, n = oracle_case
    if c["nu"] >= 1.0:
        pytest.skip("nu = 1: the residual test alone nearly meets the bar")
    h = mcs.Handle.structured(c["dim"], c["N"], c["k"], c["nu"], gmg_levels=c["levels"],
                              **dict(bench.FORMS["mixed"], etol=0.0))
    h.condense()
    x = torch.zeros_like(F)
    h.solve(F, x)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg[:n] - xo[:n]) / np.linalg.norm(xo[:n]) > 1e-7
    h.close()


def test_full_size_forms_agree(mcs):
    """The headline workload as bench.py runs it: both forms converge with their error bounds met, and
    their solutions agree within the mixed form's bar (the FP64 form's bar is 100 times smaller)."""
    w = bench.WORKLOADS[bench.HEADLINE]
    xs = {}
    for form in ("fp64", "mixed"):
        h = mcs.Handle.structured(w["dim"], w["N"], w["k"], w["nu"], gmg_levels=w["levels"], **bench.FORMS[form])
        h.condense()
        if form == "fp64":
            F = _rhs(h, w["dim"], w["nu"])
            n = h.sizes.off_p
        x = torch.zeros_like(F)
        info = h.solve(F, x)
        assert info.status == 0 and info.err_est <= bench.ERR_BAR[form], (form, info.err_est)
        xs[form] = x
        h.close()
    for sl in (slice(0, n), slice(n, None)):
        a, b = xs["mixed"][sl], xs["fp64"][sl]
        assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) <= bench.ERR_BAR["mixed"]
