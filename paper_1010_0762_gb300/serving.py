"""Serving loop for streams of dual-pair requests over the continuous-batching engine.

A request names a sequence family and a precision.  Each family is one slowly changing
operator (the convection drifts by a fixed relative step per request) whose recycle space stays
on the device between its requests, in a resident handle.  The loop admits arrived requests as
engine slots and device memory allow, advances all requests in flight one cycle per engine step
(one launch per iteration phase for all of them), and retires finished ones.  Admission is by
an HBM budget: idle families are evicted least recently used (their handle, and with it the
recycle space, is dropped; correctness is unaffected, only the next solve's iteration count).

Host logic only: every solve step runs in the library's kernels (rbicg_engine_*).
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import inputs as I


@dataclasses.dataclass
class FamilySpec:
    fid: int
    N: int                 # grid side (n = N^2)
    c0: tuple              # initial convection
    k: int                 # recycle dimension
    drift: float = 0.01    # relative drift of the convection per request
    seed: int = 0


@dataclasses.dataclass
class Request:
    rid: int
    fid: int
    precision: str         # "fp64" or "fp32_refined"
    t_arrival: float       # seconds after the start of the run
    t_admit: float = -1.0
    t_done: float = -1.0
    result: dict | None = None
    x: object = None       # device solution (kept when requested)


def footprint_bytes(n, nnz, k, s, w=8):
    """Device bytes a resident handle holds for order n (FP64): residual rings of two cycles,
    bases U, Ut, C, Ct and the per-cycle U_j, C_j (double-buffered), vectors, A^H values and
    the family's own copies of A and of the current right-hand sides and solutions."""
    ldk = ((k + 3) // 4) * 4
    rings = 2 * (2 * (s + 2)) * n * w
    bases = 12 * n * ldk * w
    vectors = 12 * n * w
    matrix = 2 * nnz * (w + 4) + 2 * 4 * (n + 1)
    return rings + bases + vectors + matrix


class Family:
    """A family's problems: A_j = convdiff(N, c_j) with c_j drifting, b_j, bt_j ~ N(0, 1)."""

    def __init__(self, spec: FamilySpec):
        self.spec = spec
        self.count = 0
        self.c = np.array(spec.c0, dtype=float)
        self.rng = np.random.default_rng(spec.seed)

    def next_problem(self):
        if self.count > 0:
            self.c = self.c * (1.0 + self.spec.drift * self.rng.uniform(-1.0, 1.0, size=self.c.shape))
        self.count += 1
        A = I.convdiff(self.spec.N, list(self.c))
        n = A.n
        b = self.rng.standard_normal(n)
        bt = self.rng.standard_normal(n)
        return A, b, bt


class Server:
    """Admission, residency and the step loop.  `backend` supplies the device side:

    backend.make_handle(spec, precision) -> handle     (a resident solver)
    backend.free_handle(handle)
    backend.submit(handle, A, b, bt, tag) -> None      (starts the request on the engine)
    backend.step() -> in_flight                        (one cycle for every request in flight)
    backend.poll() -> [(tag, result_dict, x)]          (finished requests)
    """

    def __init__(self, specs, backend, hbm_budget, s=40, max_in_flight=32, keep_x=False):
        self.specs = {sp.fid: sp for sp in specs}
        self.families = {sp.fid: Family(sp) for sp in specs}
        self.backend = backend
        self.hbm_budget = hbm_budget
        self.s = s
        self.max_in_flight = max_in_flight
        self.keep_x = keep_x
        self.resident = collections.OrderedDict()   # (fid, precision) -> handle, LRU order
        self.bytes_resident = 0
        self.busy = set()                             # (fid, precision) with a request in flight
        self.evictions = 0

    def _footprint(self, fid):
        sp = self.specs[fid]
        n = sp.N * sp.N
        return footprint_bytes(n, I.convdiff_nnz(sp.N, 2), sp.k, self.s)

    def _acquire(self, key):
        """The resident handle for key, creating it (and evicting idle LRU families) if needed;
        None if the budget cannot hold it now."""
        if key in self.resident:
            self.resident.move_to_end(key)
            return self.resident[key]
        need = self._footprint(key[0])
        if need > self.hbm_budget:
            raise ValueError("family %d does not fit the HBM budget at all" % key[0])
        while self.bytes_resident + need > self.hbm_budget:
            idle = [k for k in self.resident if k not in self.busy]
            if not idle:
                return None
            victim = idle[0]
            self.backend.free_handle(self.resident.pop(victim))
            self.bytes_resident -= self._footprint(victim[0])
            self.evictions += 1
        h = self.backend.make_handle(self.specs[key[0]], key[1])
        self.resident[key] = h
        self.bytes_resident += need
        return h

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep):
        """Serve `requests` (sorted by t_arrival, in seconds from the start).  Returns stats."""
        pending = collections.deque(sorted(requests, key=lambda r: r.t_arrival))
        queue = collections.deque()      # arrived, not yet admitted (FIFO)
        by_tag = {}
        t0 = clock()
        done = 0
        in_flight = 0
        while done < len(requests):
            now = clock() - t0
            while pending and pending[0].t_arrival <= now:
                queue.append(pending.popleft())
            # admission: FIFO, skipping requests whose family is busy (per-family order is kept)
            skipped = collections.deque()
            while queue and in_flight < self.max_in_flight:
                rq = queue.popleft()
                key = (rq.fid, rq.precision)
                if any(k[0] == rq.fid for k in self.busy) or any(q.fid == rq.fid for q in skipped):
                    skipped.append(rq)
                    continue
                h = self._acquire(key)
                if h is None:
                    skipped.append(rq)
                    break
                A, b, bt = self.families[rq.fid].next_problem()
                rq.t_admit = clock() - t0
                self.busy.add(key)
                by_tag[rq.rid] = rq
                self.backend.submit(h, A, b, bt, rq.rid)
                in_flight += 1
            queue.extendleft(reversed(skipped))
            if in_flight:
                self.backend.step()
            elif pending:
                sleep(max(0.0, min(pending[0].t_arrival - (clock() - t0), 0.01)))
            for tag, res, x in self.backend.poll():
                rq = by_tag.pop(tag)
                rq.t_done = clock() - t0
                rq.result = res
                if self.keep_x:
                    rq.x = x
                self.busy.discard((rq.fid, rq.precision))
                in_flight -= 1
                done += 1
        wall = clock() - t0
        # a solve counts only when it met the tolerance (status OK, or OK with an empty recycle
        # space); breakdowns and exhausted iteration budgets are reported beside it
        ok = [r for r in requests if r.result["status"] in (0, 4)]
        lat_ok = np.array([(r.t_done - r.t_arrival) * 1e3 for r in ok]) if ok else np.zeros(1)
        lat_all = np.array([(r.t_done - r.t_arrival) * 1e3 for r in requests])
        return {
            "requests": len(requests),
            "converged": len(ok),
            "failed": len(requests) - len(ok),
            "wall_s": wall,
            "solves_per_s": len(ok) / wall if wall > 0 else None,
            "requests_per_s": len(requests) / wall if wall > 0 else None,
            "p50_ms": float(np.percentile(lat_ok, 50)),
            "p99_ms": float(np.percentile(lat_ok, 99)),
            "mean_ms": float(lat_ok.mean()),
            "p99_ms_all_requests": float(np.percentile(lat_all, 99)),
            "evictions": self.evictions,
            "all_converged": len(ok) == len(requests),
            "statuses": dict(collections.Counter(int(r.result["status"]) for r in requests)),
            "fp64_fallbacks": sum(1 for r in requests if r.result.get("fallback") == 2),
            "guard_fallbacks": sum(1 for r in requests if r.result.get("fallback") == 1),
            "mean_iters": float(np.mean([r.result["iters"] for r in requests])),
        }


def poisson_arrivals(count, rate, families, seed, p_fp32=0.5):
    """`count` requests with exponential inter-arrival times (rate per second), uniform family
    choice and precision fp32_refined with probability p_fp32."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for i in range(count):
        fid = int(rng.integers(len(families)))
        prec = "fp32_refined" if rng.random() < p_fp32 else "fp64"
        out.append(Request(i, families[fid].fid, prec, float(t[i])))
    return out


def random_families(count, seed, side_lo=64, side_hi=1024, k_lo=10, k_hi=20, c_hi=50.0):
    """Families with log-uniform grid sides, U[1, c_hi]^2 convection and k ~ U{k_lo..k_hi}."""
    rng = np.random.default_rng(seed)
    out = []
    for f in range(count):
        N = int(round(np.exp(rng.uniform(np.log(side_lo), np.log(side_hi)))))
        c = tuple(rng.uniform(1.0, c_hi, size=2))
        k = int(rng.integers(k_lo, k_hi + 1))
        out.append(FamilySpec(f, N, c, k, 0.01, seed * 1000 + f))
    return out


class GpuBackend:
    """The device side of Server: resident rbicg handles and one rbicg engine."""

    def __init__(self, s=40, tol=1e-8, stream=None, restarts=0):
        import torch

        from . import rbicg as R
        self.R, self.torch = R, torch
        self.s, self.tol, self.restarts = s, tol, restarts
        self.engine = R.Engine(stream)
        self.inflight = {}   # tag -> (op, b, bt, x, xt)
        self.patterns = {}   # (N) -> (row_ptr, col_idx) on the device

    def make_handle(self, spec, precision):
        n = spec.N * spec.N
        return self.R.Solver(n, k=spec.k, s=self.s, tol=self.tol, precision=precision, restarts=self.restarts)

    def free_handle(self, h):
        h.destroy()

    def submit(self, h, A, b, bt, tag):
        torch, R = self.torch, self.R
        key = A.n
        if key not in self.patterns:
            self.patterns[key] = (torch.as_tensor(A.row_ptr, device="cuda"), torch.as_tensor(A.col_idx, device="cuda"))
        rp, ci = self.patterns[key]
        op = R.Operator(rp, ci, torch.as_tensor(A.val, device="cuda"))
        bd = torch.as_tensor(b, device="cuda")
        btd = torch.as_tensor(bt, device="cuda")
        x = torch.zeros_like(bd)
        xt = torch.zeros_like(bd)
        self.inflight[tag] = (op, bd, btd, x, xt)
        self.engine.submit(h, op, bd, btd, x, xt, tag)

    def step(self):
        return self.engine.step()

    def poll(self):
        out = []
        for tag, res in self.engine.poll():
            op, bd, btd, x, xt = self.inflight.pop(tag)
            out.append((tag, res, x))
        return out
