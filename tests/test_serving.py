"""Serving loop: admission, per-family order, HBM-budget eviction (CPU, fake device side) and
the GPU engine's batch invariance under continuous batching."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1010_0762_gb300 import serving as SV  # noqa: E402


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, d):
        self.t += max(d, 1e-4)


class FakeBackend:
    """Requests need a fixed number of steps (by family); one step advances the clock 1 ms."""

    def __init__(self, clock, steps_by_fid):
        self.clock = clock
        self.steps_by_fid = steps_by_fid
        self.left = {}
        self.fid_of = {}
        self.handles = 0
        self.freed = []
        self.max_in_flight_seen = 0

    def make_handle(self, spec, precision):
        self.handles += 1
        return (spec.fid, precision, self.handles)

    def free_handle(self, h):
        self.freed.append(h)

    def submit(self, h, A, b, bt, tag):
        assert A.n == len(b) == len(bt)
        self.left[tag] = self.steps_by_fid[h[0]]
        self.max_in_flight_seen = max(self.max_in_flight_seen, len(self.left))

    def step(self):
        self.clock.t += 1e-3
        for t in list(self.left):
            self.left[t] -= 1
        return len(self.left)

    def poll(self):
        out = []
        for t in [t for t, v in self.left.items() if v <= 0]:
            del self.left[t]
            out.append((t, {"status": 0, "iters": 1}, None))
        return out


def _specs(sides):
    return [SV.FamilySpec(f, N, (3.0, 1.0), 8, 0.01, 7 + f) for f, N in enumerate(sides)]


def test_serving_admits_in_family_order_and_retires_everything():
    specs = _specs([8, 10, 12])
    clk = FakeClock()
    be = FakeBackend(clk, {0: 3, 1: 5, 2: 2})
    srv = SV.Server(specs, be, hbm_budget=10**12, s=10, max_in_flight=4)
    reqs = SV.poisson_arrivals(30, rate=2000.0, families=specs, seed=3, p_fp32=0.0)
    st = srv.run(reqs, clock=clk, sleep=clk.sleep)
    assert st["requests"] == 30 and st["all_converged"]
    assert be.max_in_flight_seen <= 3          # at most one request per family in flight
    for f in range(3):
        mine = [r for r in reqs if r.fid == f]
        admits = [r.t_admit for r in mine]
        assert admits == sorted(admits)        # a family's requests are served in arrival order
        for a, b in zip(mine, mine[1:]):
            assert b.t_admit >= a.t_done       # ... one after another
    assert st["p99_ms"] >= st["p50_ms"] > 0
    assert srv.evictions == 0


def test_serving_evicts_idle_families_lru_under_the_hbm_budget():
    specs = _specs([16, 16, 16])
    one = SV.footprint_bytes(256, 1216, 8, 10)
    clk = FakeClock()
    be = FakeBackend(clk, {0: 2, 1: 2, 2: 2})
    srv = SV.Server(specs, be, hbm_budget=int(2.5 * one), s=10, max_in_flight=8)
    reqs = [SV.Request(i, i % 3, "fp64", 0.001 * i) for i in range(12)]
    st = srv.run(reqs, clock=clk, sleep=clk.sleep)
    assert st["all_converged"]
    assert srv.evictions > 0 and len(be.freed) == srv.evictions
    assert srv.bytes_resident <= srv.hbm_budget
    # never more than two families resident at a time
    assert len(srv.resident) <= 2


class FailingBackend(FakeBackend):
    """Family 1's requests end in a BiCG breakdown (status 2) after their steps."""

    def poll(self):
        out = []
        for t, res, x in super().poll():
            fid = self.fid_of_tag[t]
            out.append((t, {"status": 2 if fid == 1 else 0, "iters": 1}, x))
        return out

    def submit(self, h, A, b, bt, tag):
        self.fid_of_tag = getattr(self, "fid_of_tag", {})
        self.fid_of_tag[tag] = h[0]
        super().submit(h, A, b, bt, tag)


def test_breakdowns_are_reported_and_not_counted_as_solves():
    # throughput and latency percentiles count converged solves only; the failed ones are
    # reported by status beside them
    specs = _specs([8, 10])
    clk = FakeClock()
    be = FailingBackend(clk, {0: 2, 1: 4})
    srv = SV.Server(specs, be, hbm_budget=10**12, s=10, max_in_flight=4)
    reqs = [SV.Request(i, i % 2, "fp64", 0.0) for i in range(10)]
    st = srv.run(reqs, clock=clk, sleep=clk.sleep)
    assert st["requests"] == 10 and st["converged"] == 5 and st["failed"] == 5
    assert st["statuses"] == {0: 5, 2: 5} and not st["all_converged"]
    assert abs(st["solves_per_s"] - 5 / st["wall_s"]) < 1e-9
    assert abs(st["requests_per_s"] - 10 / st["wall_s"]) < 1e-9
    ok_lat = [(r.t_done - r.t_arrival) * 1e3 for r in reqs if r.fid == 0]
    assert abs(st["p50_ms"] - float(np.percentile(ok_lat, 50))) < 1e-9
    assert st["p99_ms_all_requests"] >= st["p99_ms"]


def test_family_that_cannot_fit_is_rejected():
    specs = _specs([64])
    srv = SV.Server(specs, FakeBackend(FakeClock(), {0: 1}), hbm_budget=1000, s=10)
    with pytest.raises(ValueError):
        srv.run([SV.Request(0, 0, "fp64", 0.0)], clock=FakeClock(), sleep=lambda d: None)


def test_footprint_grows_with_n_k_and_s():
    base = SV.footprint_bytes(1000, 5000, 10, 40)
    assert SV.footprint_bytes(2000, 10000, 10, 40) > base
    assert SV.footprint_bytes(1000, 5000, 20, 40) > base
    assert SV.footprint_bytes(1000, 5000, 10, 60) > base


@pytest.mark.gpu
def test_served_results_equal_solo_solves():
    # continuous batching: requests of several families join and leave the engine at cycle
    # boundaries; each family's results equal a solo, in-order solve of its sequence bit for bit
    import torch

    from paper_1010_0762_gb300 import rbicg as R

    torch.cuda.set_device(0)
    specs = [SV.FamilySpec(0, 20, (10.0, 10.0), 6, 0.01, 11), SV.FamilySpec(1, 24, (3.0, 1.0), 8, 0.01, 12),
             SV.FamilySpec(2, 16, (5.0, 2.0), 8, 0.01, 13), SV.FamilySpec(3, 28, (2.0, 2.0), 10, 0.01, 14)]
    be = SV.GpuBackend(s=20, tol=1e-9)
    srv = SV.Server(specs, be, hbm_budget=8 * 2**30, s=20, max_in_flight=8, keep_x=True)
    reqs = SV.poisson_arrivals(14, rate=400.0, families=specs, seed=5, p_fp32=0.0)
    st = srv.run(reqs)
    assert st["all_converged"], [r.result for r in reqs]
    for sp in specs:
        fam = SV.Family(sp)
        h = R.Solver(sp.N * sp.N, k=sp.k, s=20, tol=1e-9)
        for rq in [r for r in reqs if r.fid == sp.fid]:
            A, b, bt = fam.next_problem()
            x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
            xt = torch.zeros_like(x)
            res = h.solve_pair(R.Operator.from_csr(A), torch.as_tensor(b, device="cuda"),
                               torch.as_tensor(bt, device="cuda"), x, xt)
            assert res["iters"] == rq.result["iters"], (sp.fid, rq.rid)
            assert torch.equal(x, rq.x), (sp.fid, rq.rid)


@pytest.mark.gpu
def test_served_fp32_refined_requests_overlap_and_equal_solo_solves():
    # FP32-refined requests step through the engine (their inner FP32 solves are batched with the
    # other requests' cycles, the FP64 refinement steps run between engine steps): each result
    # equals a solo solve on a handle of the same precision, bit for bit
    import torch

    from paper_1010_0762_gb300 import rbicg as R

    torch.cuda.set_device(0)
    specs = [SV.FamilySpec(0, 20, (10.0, 10.0), 6, 0.01, 21), SV.FamilySpec(1, 24, (3.0, 1.0), 8, 0.01, 22),
             SV.FamilySpec(2, 16, (5.0, 2.0), 8, 0.01, 23)]
    be = SV.GpuBackend(s=20, tol=1e-10)
    srv = SV.Server(specs, be, hbm_budget=8 * 2**30, s=20, max_in_flight=8, keep_x=True)
    reqs = SV.poisson_arrivals(12, rate=400.0, families=specs, seed=7, p_fp32=0.5)
    assert {r.precision for r in reqs} == {"fp64", "fp32_refined"}
    st = srv.run(reqs)
    assert st["all_converged"], [r.result for r in reqs]
    assert any(r.result["refine_steps"] >= 1 and r.result["fallback"] == 0 for r in reqs
               if r.precision == "fp32_refined")
    for sp in specs:
        fam = SV.Family(sp)
        hs = {p: R.Solver(sp.N * sp.N, k=sp.k, s=20, tol=1e-10, precision=p) for p in ("fp64", "fp32_refined")}
        for rq in [r for r in reqs if r.fid == sp.fid]:
            A, b, bt = fam.next_problem()
            x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
            xt = torch.zeros_like(x)
            res = hs[rq.precision].solve_pair(R.Operator.from_csr(A), torch.as_tensor(b, device="cuda"),
                                              torch.as_tensor(bt, device="cuda"), x, xt)
            assert res["iters"] == rq.result["iters"], (sp.fid, rq.rid, rq.precision)
            assert res["refine_steps"] == rq.result["refine_steps"]
            assert torch.equal(x, rq.x), (sp.fid, rq.rid, rq.precision)
