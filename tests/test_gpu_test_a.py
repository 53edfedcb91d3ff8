"""Test (A) of Section 4 with Step 3's CFL-limited dt and Step 4b's rebuild on
every decrease of dt: the GPU time series (dt, rebuild flags, max density,
mass, second moment, free energy) against the oracle's time loop on a coarse
mesh of the paper's geometry (sphere r = 0.5 in [-r-2h, r+2h]^3)."""
import numpy as np
import pytest

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.experiments import run_test_a, paper_geometry_a
from paper_1811_03557_gb300.workloads import TEST_A_C0, TEST_A_RHO0, Geometry

pytestmark = pytest.mark.gpu

N, K, STEPS = 24, 0, 6


def _oracle_series():
    lo, hi, h = paper_geometry_a(N)
    st = O.PKSState(Geometry.sphere(0.5), N, lo, hi, K, 1, 1.0, 0.5 * h * h, rho0=TEST_A_RHO0,
                    c0=TEST_A_C0, dt_mode="cfl", clamp=True)
    out = []
    prev = None
    for _ in range(STEPS):
        dt = st.step()
        d = O.diagnostics(st.rho, st.c, st.sets, st.h, N, lo, hi)
        out.append((st.t, dt, 1 if prev is None or dt != prev else 0, d["max_rho"], d["mass"]))
        prev = dt
    return np.array(out)


@pytest.mark.parametrize("prec,tol", [(abi.DPM_PREC_FP64, 1e-11), (abi.DPM_PREC_FP32, 1e-5)])
def test_test_a_series_matches_oracle(ctx, prec, tol):
    ref = _oracle_series()
    res = run_test_a(ctx, N, K, T=1.0, precision=prec, max_steps=STEPS)
    s = res["series"]
    got = np.array([(x["t"], x["dt"], x["rebuilt"], x["max_rho"], x["mass"]) for x in s])
    assert len(s) == STEPS
    # dt is the CFL bound of the current c: the max face gradient is taken in
    # the state precision, so in FP32 dt carries the FP32 state's rounding
    np.testing.assert_allclose(got[:, 0], ref[:, 0], rtol=tol)
    np.testing.assert_allclose(got[:, 1], ref[:, 1], rtol=tol)
    np.testing.assert_array_equal(got[:, 2], ref[:, 2])          # Step 4b rebuilds
    np.testing.assert_allclose(got[:, 3], ref[:, 3], rtol=tol)    # max density
    np.testing.assert_allclose(got[:, 4], ref[:, 4], rtol=tol)    # mass
    assert all(x["min_rho"] >= -1e-6 * x["max_rho"] for x in s)   # positivity


def test_test_a_blows_up_at_the_centre(ctx):
    # a short GPU-only run: the CFL step shrinks and the max density grows
    res = run_test_a(ctx, 64, 0, T=2e-5)
    s = res["series"]
    assert res["stopped"] == "T reached"
    dts = [x["dt"] for x in s]
    assert all(b <= a for a, b in zip(dts, dts[1:]))             # dt never increases
    assert s[-1]["max_rho"] > s[0]["max_rho"]
    assert res["rebuilds"] >= 1
    fe = [x["free_energy"] for x in s]
    assert fe[-1] < fe[0]                                         # free energy decreases
