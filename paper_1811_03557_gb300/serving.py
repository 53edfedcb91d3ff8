"""Request loop: continuous batching of DPM elliptic solves and PKS runs on
one GPU, with boundary-equation factorisations kept resident in HBM.

The paper solves one problem at a time; a service answers a stream of them.
What makes that cheap is the split the method already has: Steps 1-2 (point
sets, gamma geometry, the BEP matrix of eq. BEP_recast and its factorisation)
depend only on (body, grid, K, sigma), while a solve (Step 4a particular
solution, Step 5 least squares and extension, Steps 6-7 Green's formula) is
two auxiliary problems and a small dense solve per right-hand side.  So the
loop keeps each factorisation resident, admits new ones by their HBM
footprint (evicting the least recently used idle one when the budget is
full), and sends every request waiting on a resident factorisation to the
GPU as one batch the moment a slot frees up (dpm_solve_batched).  Requests
that arrive while a batch is on the GPU join the next one.  A PKS run holds
its own factorisation and fields for its lifetime and advances one time step
per dispatch, so long runs interleave with short solves.

Concurrency: `n_slots` worker threads, each owning one CUDA stream and its
staging buffers.  The C library releases the GIL while it runs (ctypes), so
slots overlap on the device: copies of one batch run beside the kernels of
another.  A factorisation is used by one slot at a time (the library's
handles are single-threaded); batches of different factorisations overlap.

Each request's result is computed by the same per-request arithmetic whether
it is alone or in a batch (the batched call runs the single-request kernels
over independent right-hand sides), which tests/test_gpu_serving.py checks.

The scheduler itself only needs a backend with the methods of
LibraryBackend; tests drive it on the CPU with a fake one.
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

GiB = 1 << 30


# ---------------------------------------------------------------------------
# Backend on libdpm (GPU)
# ---------------------------------------------------------------------------
class LibraryBackend:
    """Runs the loop's work items through the C library on one GPU.

    Every slot owns a stream, device buffers for `max_batch` right-hand sides
    and solutions of up to max_N^3 values, and a pinned host buffer the
    solutions come back to.  Storage is FP32: N = 128 problems use the
    tensor-core solver, N = 256 the FFT-style solver, others the FP32 SIMT
    solver; the least squares and the extension run in FP64 as in dpm_solve.
    """

    def __init__(self, ctx, n_slots: int, max_batch: int, max_N: int, device: int = 0,
                 tc: bool = True):
        import torch
        from . import abi
        self.abi, self.torch = abi, torch
        self.ctx, self.device, self.tc = ctx, device, tc
        self.max_batch, self.max_N = max_batch, max_N
        cube = max_N ** 3
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_slots)]
        self.f_dev = [torch.empty(max_batch, cube, dtype=torch.float32, device=f"cuda:{device}")
                      for _ in range(n_slots)]
        self.u_dev = [torch.empty_like(x) for x in self.f_dev]
        self.out_host = [torch.empty(max_batch, cube, dtype=torch.float32).pin_memory()
                         for _ in range(n_slots)]
        self.fixed_bytes = 2 * n_slots * max_batch * cube * 4

    # -- sizes ----------------------------------------------------------------
    def precision(self, model) -> int:
        a = self.abi
        if self.tc and model.N == 128:
            return a.DPM_PREC_TC32
        if self.tc and model.N == 256:
            return a.DPM_PREC_FFT32
        return a.DPM_PREC_FP32

    @staticmethod
    def estimate_bytes(model, max_batch: int, pks: bool = False) -> int:
        """Upper estimate of the device bytes a factorisation holds while it is
        built (the build workspace is the largest part)."""
        N, ncol, nsh = model.N, (getattr(model, "beta", 1) + 1) * (model.K + 1) ** 2, (model.K + 1) ** 2
        cube = N ** 3 * 4
        r = max(model.geom.axes)
        h = (model.hi - model.lo) / (N + 1)
        ng = int(2.0 * 4.0 * np.pi * (r / h) ** 2) + 1024   # |gamma| (two layers of the surface)
        m = ng // 2 + 512                                    # |gamma_in|
        per_rhs = cube                                           # one cube per right-hand side
        build_cubes = min(ncol + 4, (8 << 30) // per_rhs)
        b = build_cubes * per_rhs + 2 * max_batch * per_rhs      # AP workspace
        b += N ** 3 + 16 * N * N + 64 * ng                   # labels, row pointers, index lists
        b += ng * nsh * 12 + ng * 56                         # harmonic tables, foot points, normals
        b += ncol * ng * 4 + ncol * m * 8 + (ncol + 4) * m * 4
        b += 3 * m * ncol * 8 + 3 * ncol * ncol * 8 + 64 * (m + ncol) * 8 * 3
        if pks:
            b += 4 * cube + 8 * N ** 3
        return int(1.15 * b)

    # -- elliptic factorisations --------------------------------------------------
    def build(self, slot: int, model):
        a = self.abi
        s = self.streams[slot]
        h = a.dpm_bep_build(self.ctx, model.geom, model.N, model.lo, model.hi, model.sigma, model.K,
                            model.beta, self.precision(model), s)
        try:
            a.dpm_bep_reserve(h, self.max_batch)
        except Exception:
            a.dpm_bep_destroy(h)
            raise
        return h, a.dpm_bep_device_bytes(h)

    def destroy(self, handle):
        self.abi.dpm_bep_destroy(handle)

    def solve(self, slot: int, handle, model, rhs: list, deliver):
        """Solve len(rhs) requests (host FP32 arrays or tensors of N^3 values) in
        one batch; deliver(i, u_host) is called for each before returning (the
        view is reused by the slot afterwards).  Returns the batch's device times
        in ms (CUDA events on the slot's stream): host->device copy, solve,
        device->host copy."""
        torch = self.torch
        n3 = model.N ** 3
        s = self.streams[slot]
        fd, ud, oh = self.f_dev[slot], self.u_dev[slot], self.out_host[slot]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(s):
            ev[0].record(s)
            for i, f in enumerate(rhs):
                src = f if isinstance(f, torch.Tensor) else torch.from_numpy(f)
                fd[i, :n3].copy_(src.reshape(-1), non_blocking=True)
            ev[1].record(s)
            self.abi.dpm_solve_batched(handle, [fd[i, :n3] for i in range(len(rhs))],
                                       [ud[i, :n3] for i in range(len(rhs))], stream=s)
            ev[2].record(s)
            for i in range(len(rhs)):
                oh[i, :n3].copy_(ud[i, :n3], non_blocking=True)
            ev[3].record(s)
        ev[3].synchronize()
        for i in range(len(rhs)):
            deliver(i, oh[i, :n3])
        return {"h2d_ms": ev[0].elapsed_time(ev[1]), "solve_ms": ev[1].elapsed_time(ev[2]),
                "d2h_ms": ev[2].elapsed_time(ev[3])}

    # -- PKS runs ---------------------------------------------------------------------
    def pks_create(self, slot: int, pm):
        a = self.abi
        from .workloads import TEST_A_C0, TEST_A_RHO0
        prm = a.pks_params(pm.geom, pm.N, pm.lo, pm.hi, 1.0, pm.dt_max, pm.K, 1,
                           self.precision(pm), dt_mode=1, rebuild=1, clamp=1)
        h = a.dpm_pks_create(self.ctx, prm, TEST_A_RHO0, TEST_A_C0, self.streams[slot])
        return h, a.dpm_pks_device_bytes(h)

    def pks_step(self, slot: int, handle) -> dict:
        st = self.abi.dpm_pks_step(handle, 1, True, self.streams[slot])
        return {"t": st.t, "dt": st.dt, "step": int(st.step), "mass": st.mass,
                "max_rho": st.max_rho, "min_rho": st.min_rho}

    def pks_destroy(self, handle):
        self.abi.dpm_pks_destroy(handle)


# ---------------------------------------------------------------------------
# Scheduler
# ---------------------------------------------------------------------------
@dataclass
class _Model:
    spec: object
    state: str = "absent"        # absent | building | ready | busy
    handle: object = None
    bytes: int = 0
    last_used: float = 0.0
    ready_at: float = 0.0        # when the factorisation last became resident
    pending: collections.deque = field(default_factory=collections.deque)
    builds: int = 0


@dataclass
class _Run:
    req: int
    spec: object
    state: str = "waiting"       # waiting | creating | ready | busy | done
    handle: object = None
    bytes: int = 0
    est: int = 0
    steps: int = 0
    ready_since: float = 0.0
    last: dict = field(default_factory=dict)


@dataclass
class RequestRecord:
    kind: str
    model: int
    arrival: float
    dispatch: float = float("nan")
    done: float = float("nan")
    batch: int = 0
    ok: bool = False
    error: str = ""
    result: dict = field(default_factory=dict)
    build_wait: float = 0.0      # of the queueing time: waiting for the factorisation to be built
    gpu: dict = field(default_factory=dict)   # the batch's device times (copies, solve), ms

    @property
    def latency(self):
        return self.done - self.arrival


class ServingEngine:
    """Continuous-batching request loop over a catalog of elliptic problems
    (ServingModel) and of PKS runs (PksRunModel)."""

    def __init__(self, backend, catalog, pks_catalog=(), n_slots: int = 4, max_batch: int = 8,
                 hbm_budget: int | None = None, rhs=None, on_result=None):
        self.be, self.n_slots, self.max_batch = backend, n_slots, max_batch
        self.models = [_Model(m) for m in catalog]
        self.pks_catalog = list(pks_catalog)
        fixed = getattr(backend, "fixed_bytes", 0)
        if hbm_budget is None:
            import torch
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = int(0.85 * free)
        self.budget = int(hbm_budget) - fixed     # for factorisations and PKS runs
        if self.budget <= 0:
            raise ValueError("the HBM budget does not cover the slots' staging buffers")
        self.rhs = rhs                 # rhs(seed, model) -> host array of N^3 values
        self.on_result = on_result     # on_result(request index, u_host) for solves
        self.events = []               # (time, what, detail) for tests and reports
        self.peak_bytes = 0

    # -- memory accounting ----------------------------------------------------------------
    def _used(self):
        u = sum(m.bytes for m in self.models if m.state != "absent")
        u += sum(r.bytes for r in self.runs.values() if r.state in ("creating", "ready", "busy"))
        return u

    def _estimate(self, spec, pks=False):
        return self.be.estimate_bytes(spec, self.max_batch, pks=pks)

    def _make_room(self, need, now):
        """Evict idle factorisations (least recently used first, none with waiting
        requests) until `need` more bytes fit.  Returns False if they cannot."""
        if self._used() + need <= self.budget:
            return True
        idle = sorted((m for m in self.models if m.state == "ready" and not m.pending),
                      key=lambda m: m.last_used)
        free_able = sum(m.bytes for m in idle)
        if self._used() - free_able + need > self.budget:
            return False
        for m in idle:
            if self._used() + need <= self.budget:
                break
            self.be.destroy(m.handle)
            self.events.append((now, "evict", self.models.index(m)))
            m.state, m.handle, m.bytes = "absent", None, 0
        return self._used() + need <= self.budget

    # -- workers ------------------------------------------------------------------------------
    def _worker(self, slot):
        while True:
            item = self.inbox[slot].get()
            if item is None:
                return
            kind, payload = item
            try:
                res = self._execute(slot, kind, payload)
                err = None
            except Exception as e:  # reported on the requests; the loop goes on
                res, err = None, f"{type(e).__name__}: {e}"
            self.done_q.put((slot, kind, payload, res, err, time.perf_counter()))

    def _execute(self, slot, kind, payload):
        be = self.be
        if kind == "build":
            return be.build(slot, self.models[payload].spec)
        if kind == "solve":
            mi, reqs = payload
            m = self.models[mi]
            rhs = [self.rhs(self.requests[r].rhs_seed, m.spec) for r in reqs]

            def deliver(i, u):
                if self.on_result is not None:
                    self.on_result(reqs[i], u)
            return be.solve(slot, m.handle, m.spec, rhs, deliver)
        if kind == "pks_create":
            return be.pks_create(slot, self.runs[payload].spec)
        if kind == "pks_step":
            return be.pks_step(slot, self.runs[payload].handle)
        raise ValueError(kind)

    # -- dispatch -------------------------------------------------------------------------------
    def _candidates(self):
        c = []
        for i, m in enumerate(self.models):
            if not m.pending:
                continue
            head = self.rec[m.pending[0]].arrival
            if m.state == "ready":
                c.append((head, 0, "solve", i))
            elif m.state == "absent":
                c.append((head, 1, "build", i))
        for k, r in self.runs.items():
            if r.state == "ready":
                c.append((r.ready_since, 0, "pks_step", k))
            elif r.state == "waiting":
                c.append((self.rec[k].arrival, 1, "pks_create", k))
        c.sort()
        return c

    def _fail(self, reqs, msg, now):
        for r in reqs:
            rec = self.rec[r]
            rec.ok, rec.error, rec.done = False, msg, now
            self.n_done += 1

    def _dispatch(self, now):
        sent = False
        while self.free_slots:
            chosen = None
            for head, _, kind, key in self._candidates():
                if kind in ("solve", "pks_step"):
                    chosen = (kind, key)
                    break
                if kind == "build":
                    m = self.models[key]
                    need = self._estimate(m.spec)
                    if need > self.budget:
                        self._fail(list(m.pending), "factorisation exceeds the HBM budget", now)
                        m.pending.clear()
                        continue
                    if self._make_room(need, now):
                        chosen = (kind, key)
                        break
                else:  # pks_create
                    r = self.runs[key]
                    r.est = self._estimate(r.spec, pks=True)
                    if r.est > self.budget:
                        self._fail([key], "PKS run exceeds the HBM budget", now)
                        r.state = "done"
                        continue
                    if self._make_room(r.est, now):
                        chosen = (kind, key)
                        break
            if chosen is None:
                break
            kind, key = chosen
            slot = self.free_slots.pop()
            if kind == "solve":
                m = self.models[key]
                reqs = [m.pending.popleft() for _ in range(min(self.max_batch, len(m.pending)))]
                for r in reqs:
                    rec = self.rec[r]
                    rec.dispatch, rec.batch = now, len(reqs)
                    # the part of the wait spent on the factorisation's build
                    rec.build_wait = max(0.0, m.ready_at - rec.arrival)
                m.state = "busy"
                self.inbox[slot].put(("solve", (key, reqs)))
                self.events.append((now, "solve", (key, len(reqs))))
            elif kind == "build":
                m = self.models[key]
                m.state, m.bytes = "building", self._estimate(m.spec)
                self.inbox[slot].put(("build", key))
                self.events.append((now, "build", key))
            elif kind == "pks_create":
                r = self.runs[key]
                r.state, r.bytes = "creating", r.est
                self.rec[key].dispatch = now
                self.inbox[slot].put(("pks_create", key))
                self.events.append((now, "pks_create", key))
            else:
                r = self.runs[key]
                r.state = "busy"
                self.inbox[slot].put(("pks_step", key))
            self.busy_max = max(self.busy_max, self.n_slots - len(self.free_slots))
            self.peak_bytes = max(self.peak_bytes, self._used())
            sent = True
        return sent

    def _complete(self, slot, kind, payload, res, err, t):
        now = t - self.t0
        self.free_slots.append(slot)
        if kind == "build":
            m = self.models[payload]
            if err:
                m.state, m.bytes = "absent", 0
                self._fail(list(m.pending), err, now)
                m.pending.clear()
            else:
                m.handle, m.bytes = res
                m.state, m.last_used, m.ready_at = "ready", now, now
                m.builds += 1
        elif kind == "solve":
            mi, reqs = payload
            m = self.models[mi]
            m.state, m.last_used = "ready", now
            for r in reqs:
                rec = self.rec[r]
                rec.done, rec.ok, rec.error = now, err is None, err or ""
                rec.gpu = dict(res) if isinstance(res, dict) else {}
                self.n_done += 1
        elif kind == "pks_create":
            r = self.runs[payload]
            if err:
                r.state, r.bytes = "done", 0
                self._fail([payload], err, now)
            else:
                r.handle, r.bytes = res
                r.state, r.ready_since = "ready", now
        else:
            r = self.runs[payload]
            if err:
                self.be.pks_destroy(r.handle)
                r.state, r.bytes, r.handle = "done", 0, None
                self._fail([payload], err, now)
                return
            r.steps += 1
            r.last = res
            if r.steps >= r.spec.steps:
                self.be.pks_destroy(r.handle)
                r.state, r.bytes, r.handle = "done", 0, None
                rec = self.rec[payload]
                rec.done, rec.ok, rec.result = now, True, dict(res)
                self.n_done += 1
            else:
                r.state, r.ready_since = "ready", now

    # -- the loop --------------------------------------------------------------------------------
    def run(self, requests, realtime: bool = True) -> "ServingReport":
        """Serve `requests` (ServingRequest list sorted by arrival).  With
        realtime=False every request is present at t = 0."""
        self.requests = list(requests)
        n = len(self.requests)
        self.rec = [RequestRecord(q.kind, q.model, q.t if realtime else 0.0) for q in self.requests]
        self.runs = {}
        self.n_done = 0
        self.busy_max = 0
        self.free_slots = list(range(self.n_slots - 1, -1, -1))
        self.inbox = [queue.Queue() for _ in range(self.n_slots)]
        self.done_q = queue.Queue()
        workers = [threading.Thread(target=self._worker, args=(s,), daemon=True)
                   for s in range(self.n_slots)]
        for w in workers:
            w.start()
        nxt = 0
        self.t0 = time.perf_counter()
        try:
            while self.n_done < n:
                now = time.perf_counter() - self.t0
                while nxt < n and self.rec[nxt].arrival <= now:
                    q = self.requests[nxt]
                    if q.kind == "solve":
                        self.models[q.model].pending.append(nxt)
                    else:
                        self.runs[nxt] = _Run(nxt, self.pks_catalog[q.model])
                    nxt += 1
                while True:
                    try:
                        self._complete(*self.done_q.get_nowait())
                    except queue.Empty:
                        break
                now = time.perf_counter() - self.t0
                self._dispatch(now)
                if self.n_done >= n:
                    break
                wait = 0.05
                if nxt < n:
                    wait = max(0.0, min(wait, self.rec[nxt].arrival - now))
                try:
                    self._complete(*self.done_q.get(timeout=wait if wait > 0 else 1e-4))
                except queue.Empty:
                    pass
        finally:
            for q in self.inbox:
                q.put(None)
            for w in workers:
                w.join()
        t_end = time.perf_counter() - self.t0
        return ServingReport.from_records(self.rec, t_end, self)

    def shutdown(self):
        """Free every resident factorisation."""
        for m in self.models:
            if m.handle is not None:
                self.be.destroy(m.handle)
                m.handle, m.state, m.bytes = None, "absent", 0

    def warm(self, model_ids=None):
        """Build and reserve factorisations ahead of traffic (as many as the
        budget holds, in the given order).  Returns how many are resident."""
        ids = range(len(self.models)) if model_ids is None else model_ids
        self.runs = {}
        k = 0
        for i in ids:
            m = self.models[i]
            if m.state != "absent":
                k += 1
                continue
            need = self._estimate(m.spec)
            if self._used() + need > self.budget:
                continue
            m.handle, m.bytes = self.be.build(0, m.spec)
            m.state, m.builds = "ready", m.builds + 1
            k += 1
        return k


@dataclass
class ServingReport:
    n: int
    ok: int
    failed: int
    elapsed_s: float
    solve_p50_ms: float
    solve_p99_ms: float
    solve_mean_ms: float
    solve_max_ms: float
    solves_per_s: float
    pks_runs: int
    pks_p50_ms: float
    pks_p99_ms: float
    batches: int
    mean_batch: float
    builds: int
    evictions: int
    max_busy_slots: int
    peak_bytes: int
    by_N: dict
    breakdown: dict
    errors: list

    @staticmethod
    def from_records(rec, t_end, eng) -> "ServingReport":
        sol = [r for r in rec if r.kind == "solve" and r.ok]
        pks = [r for r in rec if r.kind == "pks" and r.ok]
        lat = np.array([r.latency for r in sol]) * 1e3
        plat = np.array([r.latency for r in pks]) * 1e3

        def pct(a, q):
            return float(np.percentile(a, q)) if a.size else float("nan")
        first = min((r.arrival for r in rec), default=0.0)
        last = max((r.done for r in sol), default=first)
        span = max(last - first, 1e-9)
        solves = [e for e in eng.events if e[1] == "solve"]
        by_N = {}
        for r in sol:
            by_N.setdefault(eng.models[r.model].spec.N, []).append(r.latency * 1e3)
        by_N = {str(k): {"n": len(v), "p50_ms": pct(np.array(v), 50), "p99_ms": pct(np.array(v), 99)}
                for k, v in sorted(by_N.items())}
        # where a solve's latency goes: queueing (waiting for the factorisation's
        # build, then for a slot) and service (the batch's copies and solve on the
        # device, the rest host work), for all solves and for the slowest 1 %
        comp = {"build_wait_ms": [], "slot_wait_ms": [], "service_ms": [], "h2d_ms": [], "solve_ms": [],
                "d2h_ms": [], "host_ms": []}
        for r in sol:
            q = (r.dispatch - r.arrival) * 1e3
            bw = min(r.build_wait * 1e3, q)
            sv = (r.done - r.dispatch) * 1e3
            g = r.gpu
            dev = g.get("h2d_ms", 0.0) + g.get("solve_ms", 0.0) + g.get("d2h_ms", 0.0)
            for k, v in (("build_wait_ms", bw), ("slot_wait_ms", q - bw), ("service_ms", sv),
                         ("h2d_ms", g.get("h2d_ms", float("nan"))), ("solve_ms", g.get("solve_ms", float("nan"))),
                         ("d2h_ms", g.get("d2h_ms", float("nan"))), ("host_ms", sv - dev)):
                comp[k].append(v)
        breakdown = {}
        if sol:
            tail = lat >= np.percentile(lat, 99)
            for k, v in comp.items():
                a = np.array(v)
                breakdown[k] = {"p50": pct(a, 50), "p99": pct(a, 99),
                                "mean_in_p99_tail": float(np.nanmean(a[tail])) if tail.any() else float("nan")}
        return ServingReport(
            n=len(rec), ok=sum(r.ok for r in rec), failed=sum(not r.ok for r in rec),
            elapsed_s=t_end, solve_p50_ms=pct(lat, 50), solve_p99_ms=pct(lat, 99),
            solve_mean_ms=float(lat.mean()) if lat.size else float("nan"),
            solve_max_ms=float(lat.max()) if lat.size else float("nan"),
            solves_per_s=len(sol) / span, pks_runs=len(pks), pks_p50_ms=pct(plat, 50),
            pks_p99_ms=pct(plat, 99), batches=len(solves),
            mean_batch=float(np.mean([e[2][1] for e in solves])) if solves else 0.0,
            builds=sum(1 for e in eng.events if e[1] == "build"),
            evictions=sum(1 for e in eng.events if e[1] == "evict"),
            max_busy_slots=eng.busy_max, peak_bytes=eng.peak_bytes, by_N=by_N, breakdown=breakdown,
            errors=sorted({r.error for r in rec if not r.ok})[:5])

    def as_dict(self):
        return dict(self.__dict__)


# ---------------------------------------------------------------------------
# Command line: a seeded Poisson stream over a catalog of resident problems
# ---------------------------------------------------------------------------
def main(argv=None):
    import argparse
    import json

    import torch

    from . import abi
    from .workloads import pks_run_catalog, poly_gauss_rhs, serving_catalog, serving_stream

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=400.0, help="mean arrivals per second")
    ap.add_argument("--models", type=int, default=32, help="elliptic catalog size")
    ap.add_argument("--pks-models", type=int, default=4)
    ap.add_argument("--pks-fraction", type=float, default=0.005)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=8)
    ap.add_argument("--budget-gib", type=float, default=0.0, help="0: 85%% of free HBM")
    ap.add_argument("--Ns", default="32,64,128,256")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-warm", action="store_true")
    a = ap.parse_args(argv)
    Ns = tuple(int(x) for x in a.Ns.split(","))
    cat = serving_catalog(a.seed, a.models, Ns=Ns)
    pcat = pks_run_catalog(a.seed + 1, a.pks_models) if a.pks_models else []
    reqs = serving_stream(a.seed, a.requests, a.rate, len(cat), len(pcat), a.pks_fraction)
    pool = {}
    for q in reqs:
        if q.kind == "solve" and q.rhs_seed not in pool:
            pool[q.rhs_seed] = torch.from_numpy(poly_gauss_rhs(q.rhs_seed, cat[q.model])).pin_memory()
    ctx = abi.dpm_ctx_create(0)
    be = LibraryBackend(ctx, a.slots, a.max_batch, max(Ns))
    eng = ServingEngine(be, cat, pcat, n_slots=a.slots, max_batch=a.max_batch,
                        hbm_budget=int(a.budget_gib * GiB) if a.budget_gib else None,
                        rhs=lambda seed, m: pool[seed])
    t = time.perf_counter()
    warm = 0 if a.no_warm else eng.warm()
    t_warm = time.perf_counter() - t
    rep = eng.run(reqs)
    eng.shutdown()
    abi.dpm_ctx_destroy(ctx)
    out = rep.as_dict()
    out.update(warm_models=warm, warm_s=t_warm, rate_hz=a.rate, catalog=a.models)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
