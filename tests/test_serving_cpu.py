"""Host logic of the request loop (paper_1811_03557_gb300/serving.py) on the
CPU, with a fake backend that sleeps instead of running kernels: admission by
memory footprint, LRU eviction, continuous batching, one operation per
factorisation at a time, PKS runs interleaved step by step, and failures
reported on the requests they belong to."""
import threading
import time

import numpy as np
import pytest

from paper_1811_03557_gb300.serving import ServingEngine
from paper_1811_03557_gb300.workloads import (Geometry, PksRunModel, ServingModel, ServingRequest,
                                              pks_run_catalog, poly_gauss_coeffs, poly_gauss_rhs,
                                              serving_catalog, serving_stream)


class FakeBackend:
    fixed_bytes = 0

    def __init__(self, sizes, solve_s=0.002, build_s=0.01, fail_build=()):
        self.sizes = sizes                 # model key -> bytes
        self.solve_s, self.build_s = solve_s, build_s
        self.fail_build = set(fail_build)
        self.lock = threading.Lock()
        self.in_use = set()
        self.live = {}                     # handle -> bytes
        self.peak = 0
        self.log = []                      # (op, key, batch size)
        self.overlap = 0
        self.active = 0
        self.next = 0

    def _key(self, m):
        return (m.N, m.K, m.sigma) if isinstance(m, ServingModel) else ("pks", m.N, m.K)

    def estimate_bytes(self, m, max_batch, pks=False):
        return self.sizes[self._key(m)]

    def _enter(self, h):
        with self.lock:
            assert h not in self.in_use, "two operations on one handle at once"
            self.in_use.add(h)
            self.active += 1
            self.overlap = max(self.overlap, self.active)

    def _leave(self, h):
        with self.lock:
            self.in_use.discard(h)
            self.active -= 1

    def _alloc(self, m):
        with self.lock:
            h = self.next
            self.next += 1
            self.live[h] = self.sizes[self._key(m)]
            self.peak = max(self.peak, sum(self.live.values()))
        return h

    def build(self, slot, m):
        if self._key(m) in self.fail_build:
            raise RuntimeError("build refused")
        h = self._alloc(m)
        self._enter(h)
        time.sleep(self.build_s)
        self._leave(h)
        self.log.append(("build", self._key(m), 0))
        return h, self.live[h]

    def destroy(self, h):
        with self.lock:
            assert h not in self.in_use
            del self.live[h]

    def solve(self, slot, h, m, rhs, deliver):
        self._enter(h)
        time.sleep(self.solve_s)
        self._leave(h)
        self.log.append(("solve", self._key(m), len(rhs)))
        for i, f in enumerate(rhs):
            deliver(i, f * 2.0)
        return {"h2d_ms": 0.1, "solve_ms": self.solve_s * 1e3, "d2h_ms": 0.1}

    def pks_create(self, slot, pm):
        h = self._alloc(pm)
        return h, self.live[h]

    def pks_step(self, slot, h):
        self._enter(h)
        time.sleep(self.solve_s)
        self._leave(h)
        self.log.append(("pks_step", h, 0))
        return {"step": 1}

    def pks_destroy(self, h):
        self.destroy(h)


def _catalog(n):
    return [ServingModel(Geometry.sphere(1.0), 32, -1.25, 1.25, 4, 100.0 + i) for i in range(n)]


def _sizes(cat, each):
    return {(m.N, m.K, m.sigma): each for m in cat}


def _reqs(times, models):
    return [ServingRequest(t, "solve", m, 10 * i) for i, (t, m) in enumerate(zip(times, models))]


def test_all_requests_served_and_results_routed():
    cat = _catalog(3)
    be = FakeBackend(_sizes(cat, 100))
    got = {}
    eng = ServingEngine(be, cat, n_slots=2, max_batch=4, hbm_budget=1000,
                        rhs=lambda seed, m: np.full(3, float(seed)),
                        on_result=lambda r, u: got.__setitem__(r, u.copy()))
    reqs = _reqs(np.linspace(0, 0.02, 30), [i % 3 for i in range(30)])
    rep = eng.run(reqs)
    assert rep.ok == 30 and rep.failed == 0
    for i, q in enumerate(reqs):
        np.testing.assert_array_equal(got[i], np.full(3, 2.0 * q.rhs_seed))
    assert rep.builds == 3 and rep.evictions == 0
    assert all(r.done >= r.dispatch >= r.arrival for r in eng.rec)


def test_continuous_batching_joins_waiting_requests():
    # one model, a slow solve: requests that arrive during it form the next batch
    cat = _catalog(1)
    be = FakeBackend(_sizes(cat, 100), solve_s=0.03)
    eng = ServingEngine(be, cat, n_slots=1, max_batch=8, hbm_budget=1000,
                        rhs=lambda s, m: np.zeros(1))
    reqs = _reqs([0.0] + list(np.linspace(0.045, 0.055, 6)), [0] * 7)
    rep = eng.run(reqs)
    sizes = [b for op, _, b in be.log if op == "solve"]
    assert sum(sizes) == 7
    assert max(sizes) >= 2, sizes          # later arrivals batched together
    assert all(s <= 8 for s in sizes)
    assert rep.mean_batch > 1.0


def test_max_batch_respected_and_fifo_within_model():
    cat = _catalog(1)
    be = FakeBackend(_sizes(cat, 100))
    order = []
    eng = ServingEngine(be, cat, n_slots=1, max_batch=3, hbm_budget=1000,
                        rhs=lambda s, m: np.zeros(1), on_result=lambda r, u: order.append(r))
    eng.run(_reqs([0.0] * 10, [0] * 10), realtime=False)
    assert [b for op, _, b in be.log if op == "solve"] == [3, 3, 3, 1]
    assert order == list(range(10))


def test_admission_by_footprint_and_lru_eviction():
    cat = _catalog(4)
    be = FakeBackend(_sizes(cat, 400))
    eng = ServingEngine(be, cat, n_slots=2, max_batch=4, hbm_budget=1000,
                        rhs=lambda s, m: np.zeros(1))
    # models 0,1 first (both fit), then 2 (evicts the least recently used), then 0 again
    reqs = _reqs([0.0, 0.001, 0.06, 0.12, 0.18], [0, 1, 2, 0, 3])
    rep = eng.run(reqs)
    assert rep.ok == 5
    assert be.peak <= 1000
    assert rep.evictions >= 2
    ev = [e for e in eng.events if e[1] == "evict"]
    assert ev[0][2] == 0                      # model 0 was least recently used at t=0.06
    assert eng.peak_bytes <= 1000


def test_model_larger_than_budget_fails_its_requests_only():
    cat = _catalog(2)
    sizes = _sizes(cat, 100)
    sizes[(32, 4, 101.0)] = 5000
    be = FakeBackend(sizes)
    eng = ServingEngine(be, cat, n_slots=2, max_batch=4, hbm_budget=1000,
                        rhs=lambda s, m: np.zeros(1))
    rep = eng.run(_reqs([0, 0, 0.001, 0.002], [0, 1, 0, 1]))
    assert rep.ok == 2 and rep.failed == 2
    assert all((r.model == 1) != r.ok for r in eng.rec)
    assert "budget" in rep.errors[0]


def test_failed_build_reported_and_loop_continues():
    cat = _catalog(2)
    be = FakeBackend(_sizes(cat, 100), fail_build={(32, 4, 100.0)})
    eng = ServingEngine(be, cat, n_slots=2, max_batch=4, hbm_budget=1000,
                        rhs=lambda s, m: np.zeros(1))
    rep = eng.run(_reqs([0, 0.001, 0.002], [0, 1, 0]))
    assert rep.failed == 2 and rep.ok == 1
    assert "build refused" in rep.errors[0]


def test_waits_for_memory_instead_of_evicting_busy_models():
    # budget for one model; two models with queued work: the second waits
    cat = _catalog(2)
    be = FakeBackend(_sizes(cat, 600), solve_s=0.01)
    eng = ServingEngine(be, cat, n_slots=2, max_batch=2, hbm_budget=1000,
                        rhs=lambda s, m: np.zeros(1))
    rep = eng.run(_reqs([0.0] * 6, [0, 1, 0, 1, 0, 1]), realtime=False)
    assert rep.ok == 6
    assert be.peak <= 1000


def test_pks_runs_interleave_with_solves():
    cat = _catalog(1)
    pm = PksRunModel(32, 4, steps=5)
    sizes = _sizes(cat, 100)
    sizes[("pks", 32, 4)] = 200
    be = FakeBackend(sizes, solve_s=0.004)
    eng = ServingEngine(be, cat, [pm], n_slots=1, max_batch=4, hbm_budget=1000,
                        rhs=lambda s, m: np.zeros(1))
    reqs = [ServingRequest(0.0, "pks", 0, 0)] + _reqs(np.linspace(0.001, 0.03, 8), [0] * 8)
    rep = eng.run(reqs)
    assert rep.ok == 9 and rep.pks_runs == 1
    ops = [op for op, _, _ in be.log]
    first, last = ops.index("pks_step"), len(ops) - 1 - ops[::-1].index("pks_step")
    assert "solve" in ops[first:last]          # solves ran between the run's steps
    assert ops.count("pks_step") == 5
    assert not be.live or all(v == 100 for v in be.live.values())  # the run's memory was freed


def test_overlap_uses_several_slots():
    cat = _catalog(3)
    be = FakeBackend(_sizes(cat, 100), solve_s=0.02)
    eng = ServingEngine(be, cat, n_slots=3, max_batch=2, hbm_budget=1000,
                        rhs=lambda s, m: np.zeros(1))
    rep = eng.run(_reqs([0.0] * 9, [i % 3 for i in range(9)]), realtime=False)
    assert rep.ok == 9
    assert be.overlap >= 2 and rep.max_busy_slots >= 2


def test_stream_generators_are_seeded_and_shaped():
    cat = serving_catalog(0, 64)
    assert cat == serving_catalog(0, 64)
    assert {m.N for m in cat} <= {32, 64, 128, 256} and len({m.N for m in cat}) == 4
    assert all(4 <= m.K <= 12 and 1e2 <= m.sigma <= 1e5 for m in cat)
    assert all(0.5 <= max(m.geom.axes) <= 1.0 and m.hi == -m.lo == 1.25 * max(m.geom.axes)
               for m in cat)
    s = serving_stream(0, 2000, 500.0, 64, 4, 0.01)
    t = np.array([q.t for q in s])
    assert np.all(np.diff(t) > 0)
    assert abs(len(s) / t[-1] - 500.0) < 50.0           # Poisson rate
    assert 5 <= sum(q.kind == "pks" for q in s) <= 40
    assert len(pks_run_catalog(1, 4)) == 4


def test_poly_gauss_rhs_matches_pointwise_definition():
    m = ServingModel(Geometry.ellipsoid(0.8, 0.6, 0.5), 9, -1.0, 1.0, 4, 100.0)
    f = poly_gauss_rhs(7, m, dtype=np.float64)
    c, w = poly_gauss_coeffs(7)
    h = 2.0 / 10
    r = 0.8
    for (i, j, k) in [(0, 0, 0), (4, 5, 6), (8, 1, 3)]:
        x, y, z = (-1.0 + h * (i + 1)) / r, (-1.0 + h * (j + 1)) / r, (-1.0 + h * (k + 1)) / r
        p = sum(c[a, b, d] * x ** a * y ** b * z ** d for a in range(4) for b in range(4)
                for d in range(4))
        assert abs(f[i, j, k] - p * np.exp(-w * (x * x + y * y + z * z))) < 1e-12
    assert np.all(c[np.add.outer(np.add.outer(np.arange(4), np.arange(4)), np.arange(4)) > 3] == 0)


def test_latency_breakdown_splits_queueing_and_service():
    """A cold factorisation: the first requests wait for its build, later ones
    only for a slot; service holds the backend's device times; for every request
    build wait + slot wait + service = latency."""
    cat = _catalog(1)
    be = FakeBackend(_sizes(cat, 100), build_s=0.05, solve_s=0.01)
    eng = ServingEngine(be, cat, n_slots=1, max_batch=2, hbm_budget=1000, rhs=lambda s, m: np.ones(4))
    reqs = _reqs(np.linspace(0, 0.022, 12), [0] * 12)
    rep = eng.run(reqs)
    assert rep.ok == 12
    b = rep.breakdown
    assert set(b) == {"build_wait_ms", "slot_wait_ms", "service_ms", "h2d_ms", "solve_ms", "d2h_ms", "host_ms"}
    assert b["build_wait_ms"]["p99"] > 30.0          # the first requests waited for the 50 ms build
    assert b["solve_ms"]["p50"] == pytest.approx(10.0)
    assert b["service_ms"]["p50"] >= 10.0
    for r in eng.rec:
        q = r.dispatch - r.arrival
        assert 0.0 <= r.build_wait <= q + 1e-9
        assert r.latency == pytest.approx(q + (r.done - r.dispatch))

