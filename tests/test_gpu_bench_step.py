"""The step bench.py times, end to end against the oracle.

The N = 128, K = 8 PKS workload (unit sphere in [-1.25, 1.25]^3, off-centre
Gaussians 1200 exp(-120|x - x0|^2), 600 exp(-60|x - x0|^2), x0 = (0.3, 0, 0)),
on the tensor-core solver, with Step 3's CFL time step (dt = min(dt_prev,
CFL bound, h^2/4)), the BEP and its least-squares factor rebuilt on every step
(Step 4b), and the whole step replayed as one CUDA graph: exactly the
configuration of the benchmark.  Every output of each step -- rho and c on
N^+, t, dt and the diagnostics of Section 4 -- is compared with
oracle.PKSState, started from the GPU's (FP32) initial state, at the FP32
tolerance 1e-5 relative L-inf.  The minima are compared on the scale of the
field (their exact value is ~0)."""
import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import WORKLOADS

pytestmark = pytest.mark.gpu
TOL = 1e-5
STEPS = 3


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_benchmarked_step_matches_oracle(ctx):
    w = WORKLOADS["pks_sphere_N128_K8"]
    N = w.N
    assert (N, w.K, w.beta) == (128, 8, 1)
    prm = abi.pks_params(w.geom, N, w.lo, w.hi, 1.0, w.dt, w.K, w.beta, abi.DPM_PREC_TC32,
                         dt_mode=1, rebuild=1, clamp=1)
    s = torch.cuda.Stream()
    pk = abi.dpm_pks_create(ctx, prm, w.rho0, w.c0, stream=s)
    r = torch.empty(N, N, N, device="cuda")
    c = torch.empty_like(r)
    try:
        abi.dpm_pks_get_state(pk, r, c, stream=s)
        torch.cuda.synchronize()
        o = O.PKSState(w.geom, N, w.lo, w.hi, w.K, w.beta, 1.0, w.dt,
                       rho=r.cpu().double().numpy(), c=c.cpu().double().numpy(),
                       dt_mode="cfl", clamp=True)
        Np = o.sets["Np"]
        abi.dpm_pks_set_graph(pk, True, stream=s)
        for i in range(STEPS):
            st = abi.dpm_pks_step(pk, 1, True, stream=s)
            dt = o.step()
            d = O.diagnostics(o.rho, o.c, o.sets, o.h, N, w.lo, w.hi)
            abi.dpm_pks_get_state(pk, r, c, stream=s)
            torch.cuda.synchronize()
            er = rel(r.cpu().double().numpy()[Np], o.rho[Np])
            ec = rel(c.cpu().double().numpy()[Np], o.c[Np])
            print(f"bench step {i + 1}: dt {st.dt:.6e} (oracle {dt:.6e}), rel err rho {er:.3e} c {ec:.3e}")
            assert st.step == i + 1
            assert abs(st.dt - dt) <= TOL * dt, (st.dt, dt)
            assert abs(st.t - o.t) <= TOL * o.t, (st.t, o.t)
            assert er < TOL and ec < TOL, (er, ec)
            for key in ("mass", "max_rho", "m2", "free_energy"):
                assert abs(getattr(st, key) - d[key]) <= TOL * abs(d[key]), (key, getattr(st, key), d[key])
            assert abs(st.min_rho - d["min_rho"]) <= TOL * d["max_rho"], (st.min_rho, d["min_rho"])
            assert abs(st.min_c - d["min_c"]) <= TOL * float(np.max(np.abs(o.c[Np]))), (st.min_c, d["min_c"])
    finally:
        abi.dpm_pks_destroy(pk)
