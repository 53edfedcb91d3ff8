"""The CPU context figure of bench.py (an AP solve through scipy.fft's DST-I)
computes the same solve as the oracle, so the number it reports is the rate of
a correct solve (Definition of the auxiliary problem, solved by the
diagonalising DST-I as the paper's fast Poisson solver does)."""
import numpy as np

import bench
from oracle import dpm_oracle as O


def test_fft_ap_solve_matches_oracle():
    rng = np.random.default_rng(3)
    for N, h, sigma in ((9, 0.2, 3.0), (14, 2.5 / 15, 1e4 + 1.0)):
        q = rng.uniform(-1.0, 1.0, (N, N, N))
        u = bench.fft_ap_solve(q, h, sigma)
        ref = O.aux_solve(q, h, sigma)
        assert np.max(np.abs(u - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_cpu_fft_sample_reports_a_rate():
    w = bench.WORKLOADS["pks_sphere_N128_K8"]
    small = type("W", (), {"N": 16, "lo": w.lo, "hi": w.hi, "dt": w.dt})
    r = bench.cpu_fft_sample(small, 0.05, 1)
    assert r["value"] > 0 and r["cores"] == 1 and "N=16" in r["sample"]
