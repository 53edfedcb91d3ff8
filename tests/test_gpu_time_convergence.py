"""Convergence in time of Test (A) on the GPU (FP64), the protocol of Section 4
at small meshes: dt = dT/tau, final time T, errors over M^+ against the
dt = dT/tau_ref run.  The single-domain errors equal the oracle's, and single
domain and domain decomposition are first order in dt."""
import numpy as np
import pytest

from oracle import dpm_oracle as O
from paper_1811_03557_gb300.experiments import paper_geometry_a, run_time_convergence
from paper_1811_03557_gb300.workloads import TEST_A_C0, TEST_A_RHO0, Geometry

pytestmark = pytest.mark.gpu

TAUS, TAU_REF, DT, T = (1, 2, 4), 32, 1e-7, 1e-6
WANT = [np.log2((1 - 1 / 32) / (1 / 2 - 1 / 32)), np.log2((1 / 2 - 1 / 32) / (1 / 4 - 1 / 32))]


def oracle_errors(N):
    lo, hi, _ = paper_geometry_a(N)

    def final(tau):
        st = O.PKSState(Geometry.sphere(0.5), N, lo, hi, 0, 1, 1.0, DT / tau, rho0=TEST_A_RHO0,
                        c0=TEST_A_C0, dt_mode="fixed", clamp=True)
        for _ in range(int(round(T * tau / DT))):
            st.step()
        return st

    ref = final(TAU_REF)
    m = ref.sets["Mp"]
    return np.array([(np.max(np.abs(np.where(m, s.rho - ref.rho, 0))), np.max(np.abs(np.where(m, s.c - ref.c, 0))))
                     for s in (final(t) for t in TAUS)])


def test_time_convergence_sd_and_dd(ctx):
    N = 24
    res = run_time_convergence(ctx, N, dd_grids=((24, 20),), taus=TAUS, tau_ref=TAU_REF, dT=DT, T=T)
    sd = res["sd"]["rows"]
    E = np.array([(r["E_rho_0"], r["E_c_0"]) for r in sd])
    # E is a difference of two fields, each within 1e-11 (relative L-inf, FP64) of
    # the oracle's: |E - E_oracle| <= 2e-11 max|field| (rho <= 1000, c <= 500)
    Eo = oracle_errors(N)
    assert np.all(np.abs(E[:, 0] - Eo[:, 0]) <= 2e-11 * TEST_A_RHO0.amp)
    assert np.all(np.abs(E[:, 1] - Eo[:, 1]) <= 2e-11 * TEST_A_C0.amp)
    for r, w in zip(sd[1:], WANT):
        assert abs(r["rate_rho_0"] - w) < 0.03 and abs(r["rate_c_0"] - w) < 0.03
        assert abs(r["t"] - T) < 1e-12
    dd = res["dd"][0]["rows"]
    for r, w in zip(dd[1:], WANT):
        assert abs(r["rate_rho_0"] - w) < 0.05 and abs(r["rate_c_0"] - w) < 0.05, r
        # the shell's errors are ~1e-11 of the ball's: looser, rounding shows
        assert abs(r["rate_rho_1"] - w) < 0.2, r
