"""Continuous-batching solve server on top of libmcs.

Requests (dim, mesh exponent e, k, nu, seed) arrive over time.  A fixed number of slots
(worker threads, each with its own CUDA stream) take admitted requests from the queue in
arrival order, so the work of several requests overlaps on the device.  Condensed
operators and multigrid hierarchies stay resident in an operator cache keyed by
(dim, N, k).  They are kept at nu = 1: the MCS operators scale exactly with nu
(A(nu) = nu A(1), Shat_p(nu) = Shat_p(1)/nu), so a request with viscosity nu is solved
with the nu = 1 operators and its velocity divided by nu (the pressure is unchanged).

Admission: a request whose operators are not resident is admitted only when the
estimated device bytes of its handle fit in the budget (default 120 GB) next to
everything resident; least-recently-used idle operators are evicted to make room.

The scheduler is independent of the GPU: `GpuBackend` runs the library, tests use a
backend that only records calls.
"""
from __future__ import annotations

import heapq
import math
import threading
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float          # seconds since the start of the trace
    dim: int
    e: int                  # mesh size exponent: about 2^e elements
    k: int
    nu: float
    seed: int

    @property
    def N(self) -> int:
        """Cells per direction of the structured mesh with about 2^e elements."""
        if self.dim == 2:
            return max(1, 2 ** ((self.e - 1) // 2))
        n = 1
        while 6 * (2 * n) ** 3 <= 2 ** self.e:
            n *= 2
        return n

    @property
    def key(self):
        return (self.dim, self.N, self.k)


@dataclass
class Result:
    rid: int
    start: float
    end: float
    latency: float
    iterations: int
    status: int
    checksum: float
    cache_hit: bool
    x: np.ndarray | None = None


def make_trace(n: int, rate: float, seed: int, dims=(2, 3), e_range=(3, 17), ks=(2, 3, 4),
               nu_range=(1e-3, 1.0)) -> list[Request]:
    """Poisson arrivals at `rate` per second; each request a seeded draw (c5 workload)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        dim = int(rng.choice(dims))
        e = int(rng.integers(e_range[0], e_range[1] + 1))
        k = int(rng.choice(ks))
        nu = float(math.exp(rng.uniform(math.log(nu_range[0]), math.log(nu_range[1]))))
        out.append(Request(i, t, dim, e, k, nu, int(rng.integers(0, 2 ** 31 - 1))))
    return out


def estimate_bytes(dim: int, N: int, k: int) -> int:
    """Conservative device bytes of one handle (mixed form), from the space dimensions."""
    from math import comb
    ne = (N ** dim) * (2 if dim == 2 else 6)
    nf = ne * (dim + 1) // 2 + dim * N ** (dim - 1) * (2 if dim == 2 else 4)
    nk = comb(k + dim, dim)
    nF, nFm1 = comb(k + dim - 1, dim - 1), comb(k + dim - 2, dim - 1)
    nu_ = dim * nk
    nbub = nu_ - (dim + 1) * nF
    mF = nF + (dim - 1) * nFm1
    nc = (dim + 1) * mF
    nA = nu_ + (dim + 1) * (dim - 1) * nFm1
    npres = comb(k - 1 + dim, dim)
    ndof = nf * mF + ne * (nbub + npres)
    per_elem = 8 * (nA * (nA + 1) // 2) + 4 * ((dim + 1) * (nc * mF + 3) + nbub * nc + nbub * nbub + 8)
    per_facet = 4 * (mF * mF + 4 + mF * dim * dim) + 64 + 64
    vectors = 8 * ndof * 12 + 4 * ndof * 5
    gmg = 2 * (N + 1) ** dim * dim * 4 * 60
    return int(1.3 * (ne * per_elem + nf * per_facet + vectors + gmg)) + (64 << 20)


class GpuBackend:
    """Runs requests with libmcs on the current CUDA device."""

    def __init__(self, precision=None, rtol=1e-8, etol=1e-8):
        import torch

        import paper_2207_08481_gb300.mcs as mcs
        self.torch = torch
        self.mcs = mcs
        self.precision = mcs.MCS_MIXED if precision is None else precision
        self.rtol = rtol
        self.etol = etol

    def new_stream(self):
        return self.torch.cuda.Stream()

    def setup(self, key, stream):
        """New operators on a stream of their own (work on different handles overlaps)."""
        dim, N, k = key
        hs = self.torch.cuda.Stream()
        hs.wait_stream(stream)
        with self.torch.cuda.stream(hs):
            h = self.mcs.Handle.structured(dim, N, k, 1.0, stream=hs, precision=self.precision, rtol=self.rtol,
                                           etol=self.etol)
            h.condense()
        return h

    def resident_bytes(self, h) -> int:
        return int(h.sizes.bytes_resident)

    def coefficients(self, req: Request, s):
        """c ~ N(0,1) on the velocity dofs (u_d, u_o), zero elsewhere: drawn on the device by
        torch's generator seeded with the request's seed (the same c for the same request)."""
        torch = self.torch
        g = torch.Generator(device="cuda")
        g.manual_seed(req.seed)
        c = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
        c[:s.off_h] = torch.randn(s.off_h, dtype=torch.float64, device="cuda", generator=g)
        return c

    def solve(self, h, req: Request, stream, keep_x: bool):
        """Random body force f = sum c_j phi_j (c ~ N(0,1), seeded), F = M_u c, solve, scale by 1/nu.
        Everything runs on the handle's stream (requests on one handle are serialised)."""
        torch = self.torch
        s = h.sizes
        with torch.cuda.stream(h.stream):
            ct = self.coefficients(req, s)
            F = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
            h.mass_velocity(ct, F)
            x = torch.zeros_like(F)
            info = h.solve(F, x, check=False)
            x[:s.off_p] /= req.nu          # velocity of the nu problem; pressure unchanged
            xh = x.cpu().numpy()
        return info.iterations, info.status, float(np.sum(xh)), (xh if keep_x else None)

    def close(self, h):
        h.close()


class SolveServer:
    def __init__(self, backend, slots: int = 4, budget_bytes: float = 120e9, keep_x: bool = False,
                 estimator=estimate_bytes):
        self.backend = backend
        self.slots = slots
        self.budget = budget_bytes
        self.keep_x = keep_x
        self.estimator = estimator
        self.cache: OrderedDict = OrderedDict()      # key -> handle (LRU order)
        self.cache_bytes: dict = {}
        self.in_use: dict = {}                       # key -> number of requests running on it
        self.key_lock: dict = {}
        self.lock = threading.Condition()
        self.evictions = 0
        self.peak_bytes = 0

    # ---------------------------------------------------------------- memory accounting
    def resident(self) -> int:
        return sum(self.cache_bytes.values())

    def _make_room(self, need: int) -> bool:
        """Evict idle LRU operators until `need` more bytes fit; False if impossible now."""
        while self.resident() + need > self.budget:
            victim = None
            for key in self.cache:
                if self.in_use.get(key, 0) == 0 and self.cache[key] is not None:
                    victim = key
                    break
            if victim is None:
                return False
            h = self.cache.pop(victim)
            self.cache_bytes.pop(victim, None)
            self.backend.close(h)
            self.evictions += 1
        return True

    def _acquire(self, req: Request, stream):
        """Operators for req (cached or new); blocks until the budget admits them."""
        key = req.key
        with self.lock:
            while True:
                if key in self.cache:
                    self.cache.move_to_end(key)
                    self.in_use[key] = self.in_use.get(key, 0) + 1
                    lk = self.key_lock.setdefault(key, threading.Lock())
                    h = self.cache[key]
                    hit = h is not None
                    if h is not None:
                        break
                    # another slot is setting it up: wait
                    self.in_use[key] -= 1
                    self.lock.wait(0.05)
                    continue
                need = self.estimator(*key)
                if need > self.budget:
                    raise MemoryError(f"request {req.rid} needs {need} bytes, more than the budget")
                if self._make_room(need):
                    self.cache[key] = None                   # placeholder while setting up
                    self.cache_bytes[key] = need
                    self.in_use[key] = 1
                    lk = self.key_lock.setdefault(key, threading.Lock())
                    hit = False
                    h = None
                    break
                self.lock.wait(0.05)
        if h is None:
            h = self.backend.setup(key, stream)
            with self.lock:
                self.cache[key] = h
                self.cache_bytes[key] = self.backend.resident_bytes(h)
                self.peak_bytes = max(self.peak_bytes, self.resident())
                self.lock.notify_all()
        return h, lk, hit

    def _release(self, key):
        with self.lock:
            self.in_use[key] -= 1
            self.lock.notify_all()

    # ---------------------------------------------------------------- trace replay
    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Replays the trace: request i becomes available at its arrival time."""
        queue = deque()
        results: list[Result] = []
        done = threading.Event()
        qlock = threading.Condition()
        t0 = time.perf_counter()
        pending = sorted(requests, key=lambda r: r.arrival)

        def feeder():
            for r in pending:
                if realtime:
                    dt = r.arrival - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                with qlock:
                    queue.append(r)
                    qlock.notify()
            with qlock:
                done.set()
                qlock.notify_all()

        def worker():
            stream = self.backend.new_stream()
            while True:
                with qlock:
                    while not queue and not done.is_set():
                        qlock.wait(0.05)
                    if not queue and done.is_set():
                        return
                    req = queue.popleft()
                start = time.perf_counter() - t0
                h, lk, hit = self._acquire(req, stream)
                try:
                    with lk:                       # one request at a time per handle
                        its, status, chk, x = self.backend.solve(h, req, stream, self.keep_x)
                finally:
                    self._release(req.key)
                end = time.perf_counter() - t0
                arrival = req.arrival if realtime else 0.0
                res = Result(req.rid, start, end, end - arrival, its, status, chk, hit, x)
                with qlock:
                    results.append(res)

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.slots)]
        feed = threading.Thread(target=feeder, daemon=True)
        feed.start()
        for t in threads:
            t.start()
        feed.join()
        for t in threads:
            t.join()
        results.sort(key=lambda r: r.rid)
        return results

    def close(self):
        with self.lock:
            for h in self.cache.values():
                if h is not None:
                    self.backend.close(h)
            self.cache.clear()
            self.cache_bytes.clear()


def summarize(results: list[Result], wall: float) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    return {"requests": len(results), "throughput_solves_per_s": len(results) / wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "not_converged": int(sum(1 for r in results if r.status != 0)),
            "cache_hits": int(sum(1 for r in results if r.cache_hit))}
