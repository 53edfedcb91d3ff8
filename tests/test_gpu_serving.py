"""The request loop on the GPU: each result served in a mixed, continuously
batched stream equals the same request solved alone (dpm_solve on the same
factorisation) within the FP32 tolerance, and agrees with the FP64 oracle
within the elliptic FP32 bound; a PKS run served in the mix ends in the same
state as the run advanced alone; eviction under a small HBM budget changes
no result."""
import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.serving import LibraryBackend, ServingEngine
from paper_1811_03557_gb300.workloads import (TEST_A_C0, TEST_A_RHO0, Geometry, PksRunModel,
                                              ServingModel, ServingRequest, poly_gauss_rhs)

pytestmark = pytest.mark.gpu

CATALOG = [
    ServingModel(Geometry.sphere(0.8), 32, -1.0, 1.0, 4, 1.0e3),
    ServingModel(Geometry.ellipsoid(0.9, 0.7, 0.6), 32, -1.125, 1.125, 6, 3.0e4),
    ServingModel(Geometry.sphere(0.6), 48, -0.75, 0.75, 5, 2.0e2),
    ServingModel(Geometry.sphere(1.0), 128, -1.25, 1.25, 4, 1.0e4),   # tensor-core solver
]
PKS = [PksRunModel(32, 4, steps=3)]


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _stream(n, seed=0):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, 0.03, size=n))
    return [ServingRequest(float(t[i]), "solve", int(rng.integers(0, len(CATALOG))), 100 + i)
            for i in range(n)]


def _serve(ctx, reqs, budget=None, n_slots=2, max_batch=4):
    pool = {}
    for q in reqs:
        if q.kind == "solve":
            pool[q.rhs_seed] = torch.from_numpy(poly_gauss_rhs(q.rhs_seed, CATALOG[q.model])).pin_memory()
    got = {}
    be = LibraryBackend(ctx, n_slots, max_batch, max(m.N for m in CATALOG))
    eng = ServingEngine(be, CATALOG, PKS, n_slots=n_slots, max_batch=max_batch,
                        hbm_budget=budget, rhs=lambda s, m: pool[s],
                        on_result=lambda r, u: got.__setitem__(r, u.numpy().copy()))
    rep = eng.run(reqs)
    return eng, rep, got, pool


def _alone(eng, mi, f):
    """The same request solved by itself on the engine's resident factorisation."""
    m = CATALOG[mi]
    fd = f.to("cuda").reshape(-1)
    u = torch.empty_like(fd)
    abi.dpm_solve(eng.models[mi].handle, fd, u)
    torch.cuda.synchronize()
    return u.cpu().numpy()


def test_mixed_stream_matches_alone_and_oracle(ctx):
    reqs = _stream(24) + [ServingRequest(0.004, "pks", 0, 0)]
    reqs.sort(key=lambda q: q.t)
    eng, rep, got, pool = _serve(ctx, reqs)
    assert rep.failed == 0, rep.errors
    assert rep.batches < 24 and rep.mean_batch > 1.0      # requests were batched
    bitwise = 0
    for i, q in enumerate(reqs):
        if q.kind != "solve":
            continue
        u_alone = _alone(eng, q.model, pool[q.rhs_seed])
        assert rel(got[i], u_alone) <= 1e-5, (i, q)
        bitwise += int(np.array_equal(got[i], u_alone))
    print(f"served == alone bit for bit: {bitwise} of {len(got)}")
    # FP32 elliptic bound against the FP64 oracle, one request per N=32 model
    for mi in (0, 1):
        i = next(k for k, q in enumerate(reqs) if q.kind == "solve" and q.model == mi)
        m = CATALOG[mi]
        s = O.DPMSetup(m.geom, m.N, m.lo, m.hi, m.K, m.beta, m.sigma)
        f = pool[reqs[i].rhs_seed].numpy().astype(np.float64)
        u_ref, _, _ = O.dpm_elliptic_solve(s, f)
        u = got[i].reshape(m.N, m.N, m.N).astype(np.float64)
        assert rel(np.where(s.sets["Np"], u, 0), np.where(s.sets["Np"], u_ref, 0)) < 1e-5
    # the PKS run served between the solves ends where the run alone does
    k = next(i for i, q in enumerate(reqs) if q.kind == "pks")
    pm = PKS[0]
    prm = abi.pks_params(pm.geom, pm.N, pm.lo, pm.hi, 1.0, pm.dt_max, pm.K, 1, abi.DPM_PREC_FP32,
                         dt_mode=1, rebuild=1, clamp=1)
    h = abi.dpm_pks_create(ctx, prm, TEST_A_RHO0, TEST_A_C0)
    for _ in range(pm.steps):
        st = abi.dpm_pks_step(h, 1, True)
    abi.dpm_pks_destroy(h)
    res = eng.rec[k].result
    assert res["step"] == st.step
    assert abs(res["mass"] - st.mass) <= 1e-5 * abs(st.mass)
    assert abs(res["max_rho"] - st.max_rho) <= 1e-5 * abs(st.max_rho)
    eng.shutdown()


def test_eviction_under_small_budget_keeps_results(ctx):
    # the N=128 factorisation's build only fits once the others are evicted
    order = [(0.0, 0), (0.001, 1), (0.06, 3), (0.07, 0), (0.08, 2), (0.09, 3), (0.1, 1)]
    reqs = [ServingRequest(t, "solve", m, 500 + i) for i, (t, m) in enumerate(order)]
    probe = LibraryBackend.estimate_bytes(CATALOG[3], 2)
    fixed = 2 * 1 * 2 * 128 ** 3 * 4
    eng, rep, got, pool = _serve(ctx, reqs, budget=fixed + probe + (1 << 20), n_slots=1, max_batch=2)
    assert rep.failed == 0, rep.errors
    assert rep.evictions >= 1
    for i, q in enumerate(reqs):
        if eng.models[q.model].handle is not None:
            assert rel(got[i], _alone(eng, q.model, pool[q.rhs_seed])) <= 1e-5
    eng.shutdown()
