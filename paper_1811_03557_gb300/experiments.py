"""Test (A) of Section 4 run to blow-up on the GPU: the time loop with Step 3's
CFL-limited dt and Step 4b's BEP rebuild whenever dt decreases, recording the
max density, mass, second moment and free energy at every step (the
quantities of the paper's evolution figures for Test (A)).

Geometry and mesh as Section 4 states them: a sphere of radius r = 0.5 at the
origin in the box [-r - 2h, r + 2h]^3 with h = 2r/(N - 3) for N interior nodes
per axis (the paper counts N + 1 cells: h = 2r/(cells - 4)); dt = 0.5 h^2 before
blow-up and the CFL bound near it; chi = 1.  One zonal harmonic per term of the
extension (K = 0) suffices for this radially symmetric test, as the paper notes.

    python -m paper_1811_03557_gb300.experiments --N 128 --T 6e-5 --out series.json
"""
from __future__ import annotations

import json
import time


def paper_geometry_a(N: int, r: float = 0.5):
    h = 2.0 * r / (N - 3)
    return -r - 2.0 * h, r + 2.0 * h, h


def run_test_a(ctx, N: int = 128, K: int = 0, T: float = 6e-5, precision=None,
               max_steps: int = 100000, stop_jump: float = 0.0, stream=None):
    """Advance Test (A) to time T; with stop_jump > 0 also stop once ||rho||_inf
    changes by more than stop_jump over two consecutive steps (the termination
    rule the paper applies to its Test (B) runs).  Returns the per-step series
    and the wall time."""
    import torch

    from . import abi
    from .workloads import TEST_A_C0, TEST_A_RHO0, Geometry

    if precision is None:
        precision = abi.DPM_PREC_TC32 if N == 128 else abi.DPM_PREC_FP32
    lo, hi, h = paper_geometry_a(N)
    prm = abi.pks_params(Geometry.sphere(0.5), N, lo, hi, 1.0, 0.5 * h * h, K, 1, precision,
                         dt_mode=1, rebuild=0, clamp=1)
    pk = abi.dpm_pks_create(ctx, prm, TEST_A_RHO0, TEST_A_C0, stream=stream)
    series = []
    t0 = time.perf_counter()
    stopped = "T reached"
    try:
        while True:
            st = abi.dpm_pks_step(pk, 1, True, stream=stream)
            series.append({"step": int(st.step), "t": st.t, "dt": st.dt, "rebuilt": int(st.rebuilt),
                           "max_rho": st.max_rho, "min_rho": st.min_rho, "mass": st.mass,
                           "m2": st.m2, "free_energy": st.free_energy})
            if st.t >= T:
                break
            if (stop_jump > 0 and len(series) >= 2
                    and abs(series[-1]["max_rho"] - series[-2]["max_rho"]) > stop_jump):
                stopped = "max density jump"
                break
            if len(series) >= max_steps:
                stopped = "step limit"
                break
    finally:
        torch.cuda.synchronize()
        abi.dpm_pks_destroy(pk)
    wall = time.perf_counter() - t0
    return {"N": N, "K": K, "h": h, "T": T, "precision": precision, "steps": len(series),
            "rebuilds": sum(s["rebuilt"] for s in series), "stopped": stopped,
            "wall_s": wall, "series": series}


def main(argv=None):
    import argparse

    from . import abi

    ap = argparse.ArgumentParser(description="Test (A) to blow-up")
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--K", type=int, default=0)
    ap.add_argument("--T", type=float, default=6e-5)
    ap.add_argument("--stop-jump", type=float, default=0.0)
    ap.add_argument("--out", default="")
    a = ap.parse_args(argv)
    ctx = abi.dpm_ctx_create(0)
    res = run_test_a(ctx, a.N, a.K, a.T, stop_jump=a.stop_jump)
    abi.dpm_ctx_destroy(ctx)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f)
    s = res["series"]
    pick = [s[i] for i in sorted({0, len(s) // 4, len(s) // 2, 3 * len(s) // 4, len(s) - 1})]
    summary_keys = ("step", "t", "dt", "rebuilt", "max_rho", "mass", "m2", "free_energy")
    pick = [{k: x[k] for k in summary_keys} for x in pick]
    summary = {k: v for k, v in res.items() if k != "series"}
    summary["samples"] = pick
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
