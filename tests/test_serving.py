"""Serving loop: scheduler logic on the CPU (fake backend), determinism on the GPU."""
import threading
import time

import numpy as np
import pytest

from paper_2207_08481_gb300 import serve


class FakeBackend:
    """Records calls; a 'solve' takes a little time and returns a value derived from the request."""

    def __init__(self, nbytes=10):
        self.nbytes = nbytes
        self.setups, self.closes = [], []
        self.active = {}
        self.lock = threading.Lock()
        self.max_concurrent = 0
        self.overlap_same_key = False
        self._running = 0

    def new_stream(self):
        return object()

    def setup(self, key, stream):
        with self.lock:
            self.setups.append(key)
        return {"key": key}

    def resident_bytes(self, h):
        return self.nbytes

    def solve(self, h, req, stream, keep_x):
        with self.lock:
            self._running += 1
            self.max_concurrent = max(self.max_concurrent, self._running)
            if self.active.get(h["key"]):
                self.overlap_same_key = True
            self.active[h["key"]] = True
        time.sleep(0.002)
        with self.lock:
            self.active[h["key"]] = False
            self._running -= 1
        return 5, 0, float(req.seed % 97), None

    def close(self, h):
        with self.lock:
            self.closes.append(h["key"])


def test_trace_is_seeded_and_well_formed():
    a = serve.make_trace(200, 50.0, seed=7)
    b = serve.make_trace(200, 50.0, seed=7)
    assert [(r.dim, r.e, r.k, r.nu, r.seed) for r in a] == [(r.dim, r.e, r.k, r.nu, r.seed) for r in b]
    assert all(np.diff([r.arrival for r in a]) > 0)
    rate = len(a) / a[-1].arrival
    assert 35 < rate < 70
    assert {r.k for r in a} <= {2, 3, 4} and {r.dim for r in a} == {2, 3}
    assert all(1e-3 <= r.nu <= 1.0 and 3 <= r.e <= 17 for r in a)
    # mesh size rule: about 2^e elements, at most 2^e
    for r in a:
        ne = r.N ** r.dim * (2 if r.dim == 2 else 6)
        assert ne <= 2 ** r.e


def test_scheduler_completes_all_and_serialises_per_handle():
    fb = FakeBackend()
    srv = serve.SolveServer(fb, slots=4, budget_bytes=1e12, estimator=lambda *k: 10)
    reqs = serve.make_trace(60, 1000.0, seed=1, e_range=(3, 5))
    res = srv.run(reqs, realtime=False)
    assert [r.rid for r in res] == list(range(60))
    assert all(r.status == 0 for r in res)
    assert fb.max_concurrent > 1            # work of several requests overlaps
    assert not fb.overlap_same_key          # one request at a time per handle
    assert len(fb.setups) == len(set(fb.setups))   # operators are cached, never set up twice
    srv.close()


def test_admission_respects_the_budget_and_evicts_lru():
    fb = FakeBackend(nbytes=40)
    srv = serve.SolveServer(fb, slots=2, budget_bytes=100, estimator=lambda *k: 40)
    reqs = serve.make_trace(40, 1000.0, seed=3, e_range=(3, 9))
    res = srv.run(reqs, realtime=False)
    assert len(res) == 40
    assert srv.peak_bytes <= 100
    assert srv.evictions > 0 and len(fb.closes) == srv.evictions
    srv.close()


def test_request_larger_than_budget_is_refused():
    fb = FakeBackend()
    srv = serve.SolveServer(fb, slots=1, budget_bytes=5, estimator=lambda *k: 40)
    with pytest.raises(MemoryError):
        srv._acquire(serve.Request(0, 0.0, 2, 5, 2, 0.1, 1), None)


@pytest.mark.gpu
def test_results_identical_alone_and_in_the_mix():
    """Each request's solution is the same when served alone and among concurrent requests."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2207_08481_gb300 import build
    build.build()
    reqs = serve.make_trace(16, 1000.0, seed=11, e_range=(5, 11), ks=(2, 3))
    mixed = serve.SolveServer(serve.GpuBackend(), slots=4, keep_x=True)
    rm = mixed.run(reqs, realtime=False)
    mixed.close()
    alone = serve.SolveServer(serve.GpuBackend(), slots=1, keep_x=True)
    ra = alone.run(reqs, realtime=False)
    alone.close()
    for a, b in zip(rm, ra):
        assert a.status == 0 and b.status == 0
        assert np.abs(a.x - b.x).max() <= 1e-12 * np.abs(b.x).max()


@pytest.mark.gpu
@pytest.mark.parametrize("dim,e,k,nu", [(3, 4, 2, 0.05), (2, 3, 4, 0.3), (2, 9, 3, 2e-3)])
def test_served_solution_matches_oracle_at_nu(dim, e, k, nu):
    """A request solved with the cached nu = 1 operators and rescaled equals the oracle's direct
    solve at its own nu (smallest meshes of the trace included: 3D with one cell, 2D with 2x2)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from oracle import mesh, system
    from paper_2207_08481_gb300 import build
    build.build()
    req = serve.Request(0, 0.0, dim, e, k, nu, 1234)
    be = serve.GpuBackend(rtol=1e-10)
    h = be.setup(req.key, torch.cuda.current_stream())
    its, status, _, x = be.solve(h, req, None, True)
    be_sizes = h.sizes
    be.close(h)
    assert status == 0, (status, its)
    D = system.discretize(mesh.structured(dim, req.N), k, nu)
    Mu = system.assemble(D.u_map, D.u_map, D.mats["Mu"], (D.ndof, D.ndof))
    c = be.coefficients(req, be_sizes).cpu().numpy()
    xo, _, _ = system.solve_full(D, Mu @ c)
    xo = system.mean_zero_pressure(D, xo)
    n = D.off_p
    eu = np.linalg.norm(x[:n] - xo[:n]) / np.linalg.norm(xo[:n])
    ep = np.linalg.norm(x[n:] - xo[n:]) / max(np.linalg.norm(xo[n:]), 1e-300)
    assert eu < 1e-8 and ep < 1e-8, (eu, ep, its)
