"""GPU parity of the PKS time step (Steps 3-7) against the oracle, plus the
invariants the paper states: positivity under the CFL step, decreasing free
energy, approximate mass conservation."""
import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import TEST_A_C0, TEST_A_RHO0, OFFC_C0, OFFC_RHO0, Geometry

pytestmark = pytest.mark.gpu


def gpu_pks(ctx, geom, N, lo, hi, K, dt, prec, dt_mode=0, rho0=TEST_A_RHO0, c0=TEST_A_C0, rebuild=0):
    p = abi.pks_params(geom, N, lo, hi, 1.0, dt, K, 1, prec, dt_mode=dt_mode, rebuild=rebuild, clamp=1)
    return abi.dpm_pks_create(ctx, p, rho0, c0)


def state(pks, N, prec):
    dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
    r = torch.empty(N, N, N, dtype=dt, device="cuda")
    c = torch.empty_like(r)
    abi.dpm_pks_get_state(pks, r, c)
    torch.cuda.synchronize()
    return r.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("prec,tol", [(abi.DPM_PREC_FP64, 1e-11), (abi.DPM_PREC_FP32, 1e-5)])
def test_initial_state_and_one_step_match_oracle(ctx, prec, tol):
    geom, N, lo, hi, K = Geometry.sphere(1.0), 32, -1.25, 1.25, 4
    dt = 5e-6
    pks = gpu_pks(ctx, geom, N, lo, hi, K, dt, prec)
    r0, c0 = state(pks, N, prec)
    o = O.PKSState(geom, N, lo, hi, K, 1, 1.0, dt, rho0=TEST_A_RHO0, c0=TEST_A_C0, dt_mode="fixed")
    Np = o.sets["Np"]
    assert rel(r0[Np], o.rho[Np]) < (1e-14 if prec == abi.DPM_PREC_FP64 else 1e-7)
    # run the oracle from the GPU's (rounded) initial state
    o.rho, o.c = r0, c0
    st = abi.dpm_pks_step(pks, 1)
    o.step()
    r1, c1 = state(pks, N, prec)
    er, ec = rel(r1[Np], o.rho[Np]), rel(c1[Np], o.c[Np])
    print(f"PKS prec={prec}: rel err rho {er:.3e} c {ec:.3e}")
    assert er < tol and ec < tol, (er, ec)
    d = O.diagnostics(o.rho, o.c, o.sets, o.h, N, lo, hi)
    assert st.mass == pytest.approx(d["mass"], rel=tol)
    assert st.free_energy == pytest.approx(d["free_energy"], rel=tol)
    assert st.max_rho == pytest.approx(d["max_rho"], rel=tol)
    assert st.rebuilt == 1 and st.step == 1
    abi.dpm_pks_destroy(pks)


def test_cfl_mode_positivity_energy_mass(ctx):
    geom, N, lo, hi, K = Geometry.sphere(1.0), 48, -1.25, 1.25, 4
    pks = gpu_pks(ctx, geom, N, lo, hi, K, 1e-3, abi.DPM_PREC_FP32, dt_mode=1,
                  rho0=OFFC_RHO0, c0=OFFC_C0)
    hist = [abi.dpm_pks_step(pks, 1) for _ in range(6)]
    m0 = hist[0].mass
    for a, b in zip(hist, hist[1:]):
        assert b.free_energy <= a.free_energy * (1 + 1e-6)
        assert b.dt <= a.dt
    for s in hist:
        # Theorem 2.4 gives u >= 0; in FP32 a node whose exact value is 0 carries
        # rounding noise of the AP solve, ~1e-7 of the largest value
        assert s.min_rho >= -1e-6 * s.max_rho and s.min_c >= -1e-6 * s.max_rho
        assert abs(s.mass - m0) / m0 < 0.05
    abi.dpm_pks_destroy(pks)
