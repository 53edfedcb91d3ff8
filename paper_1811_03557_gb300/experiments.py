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
        precision = abi.DPM_PREC_TC32 if N in (128, 256) else abi.DPM_PREC_FP32
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


def run_test_a_dd(ctx, N1: int = 128, N2: int = 64, K: int = 0, T: float = 6e-5, precision=None,
                  r1: float = 0.25, r2: float = 0.5, record: bool = True, stream=None):
    """Test (A) with the domain decomposition of Section 3 (Case 1): the ball
    r < r1 on an N1 grid and the shell r1 < r < r2 on an N2 grid, each box
    [-r - 2h, r + 2h]^3 with h = 2r/(N - 3); dt = min(dt_prev, CFL bounds of both
    grids, 0.5 min(h1, h2)^2), rebuild of the coupled BEP when dt decreases."""
    import torch

    from . import abi
    from .workloads import TEST_A_C0, TEST_A_RHO0

    if precision is None:
        precision = abi.DPM_PREC_TC32
    lo1, hi1, h1 = paper_geometry_a(N1, r1)
    lo2, hi2, h2 = paper_geometry_a(N2, r2)
    P = abi.dd_params((0.0, 0.0, 0.0), r1, r2, N1, lo1, hi1, N2, lo2, hi2, K, K, precision)
    h = min(h1, h2)
    pk = abi.dpm_dd_pks_create(ctx, P, 1.0, 0.5 * h * h, 1, 0, 1, TEST_A_RHO0, TEST_A_C0, stream=stream)
    series = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = 0
    try:
        while True:
            st = abi.dpm_dd_pks_step(pk, 1, record, stream=stream)
            steps += 1
            if record:
                series.append({"step": int(st.step), "t": st.t, "dt": st.dt, "rebuilt": int(st.rebuilt),
                               "max_rho": st.max_rho, "mass": st.mass, "m2": st.m2,
                               "free_energy": st.free_energy})
                if st.t >= T:
                    break
            elif abi.dpm_dd_pks_step(pk, 0, True, stream=stream).t >= T:
                break
        st = abi.dpm_dd_pks_step(pk, 0, True, stream=stream)
        torch.cuda.synchronize()
    finally:
        abi.dpm_dd_pks_destroy(pk)
    wall = time.perf_counter() - t0
    last = {"t": st.t, "dt": st.dt, "step": int(st.step), "max_rho": st.max_rho, "mass": st.mass,
            "m2": st.m2, "free_energy": st.free_energy}
    return {"N1": N1, "N2": N2, "h1": h1, "h2": h2, "K": K, "T": T, "wall_s": wall, "last": last,
            "series": series}


def sd_dd_speedup(ctx, N_sd: int = 256, dd_grids=((128, 128), (128, 64)), T: float = 6e-5):
    """Wall time of Test (A) to T on the single domain (N_sd) against the domain
    decomposition (N1, N2) for each pair: R_S = T_SD / T_DD (the paper's ratio).
    Both loops are host-driven (the CFL step is read back every step) and read
    the time after every step, so both stop at the first step with t >= T."""
    from . import abi

    def sd_run():
        lo, hi, h = paper_geometry_a(N_sd)
        from .workloads import TEST_A_C0, TEST_A_RHO0, Geometry
        import torch
        prec = abi.DPM_PREC_TC32 if N_sd in (128, 256) else abi.DPM_PREC_FP32
        prm = abi.pks_params(Geometry.sphere(0.5), N_sd, lo, hi, 1.0, 0.5 * h * h, 0, 1, prec,
                             dt_mode=1, rebuild=0, clamp=1)
        pk = abi.dpm_pks_create(ctx, prm, TEST_A_RHO0, TEST_A_C0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps = 0
        while True:
            abi.dpm_pks_step(pk, 1, False)
            steps += 1
            if abi.dpm_pks_step(pk, 0, True).t >= T:
                break
        st = abi.dpm_pks_step(pk, 0, True)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        abi.dpm_pks_destroy(pk)
        return wall, {"t": st.t, "step": int(st.step), "max_rho": st.max_rho, "mass": st.mass}

    sd_run()  # warm-up (tables, workspaces)
    wall_sd, last_sd = sd_run()
    out = {"T": T, "sd": {"N": N_sd, "wall_s": wall_sd, "last": last_sd}, "dd": []}
    for N1, N2 in dd_grids:
        run_test_a_dd(ctx, N1, N2, T=T, record=False)  # warm-up
        r = run_test_a_dd(ctx, N1, N2, T=T, record=False)
        out["dd"].append({"N1": N1, "N2": N2, "h1_over_h2": r["h1"] / r["h2"], "wall_s": r["wall_s"],
                          "R_S": wall_sd / r["wall_s"], "last": r["last"]})
    return out


def boxes_test_b(N1: int, N2: int, R: float = 0.5, r1: float = 0.25):
    """Boxes of Case 2 for Test (B): the lens box centred on the north pole
    (0, 0, R) with half-width r1 + 2 h1, h1 = 2 r1/(N1 - 3); the outer box
    [-R - 2 h2, R + 2 h2]^3, h2 = 2 R/(N2 - 3)."""
    h1, h2 = 2.0 * r1 / (N1 - 3), 2.0 * R / (N2 - 3)
    return (-r1 - 2 * h1, r1 + 2 * h1, (0.0, 0.0, R), h1), (-R - 2 * h2, R + 2 * h2, (0.0, 0.0, 0.0), h2)


def run_test_b_dd(ctx, N1: int = 128, N2: int = 128, MZ: int = 20, MG: int = 150, precision=None,
                  stop_jump: float = 1000.0, T: float = 0.1, max_steps: int = 200000, record_every: int = 50,
                  stream=None, gamma_series: int = 1):
    """Test (B) of Section 4 with the domain decomposition of Case 2: the sphere
    r < 0.5 split by the sphere Z of radius 0.25 about the north pole into the
    lens Omega_1 (N1 grid) and the rest (N2 grid); rho0 = 2000 exp(-100 |x -
    (0, 0, 0.25)|^2), c0 = 0, chi = 1; MZ zonal terms per series on Z, MG on
    Gamma (2-term extension there); dt = 0.5 min(h1, h2)^2 capped by the CFL
    bound of both grids, the coupled BEP rebuilt whenever dt decreases; stop
    once ||rho||_inf changes by more than stop_jump between two steps (the
    paper's termination rule) or at time T.  gamma_series = 1: the 2-term
    extension u + d g_N on Gamma, as the paper runs Test (B); 2: the 3-term one."""
    import torch

    from . import abi
    from .workloads import TEST_B_C0, TEST_B_RHO0

    if precision is None:
        precision = abi.DPM_PREC_TC32
    (lo1, hi1, o1, h1), (lo2, hi2, o2, h2) = boxes_test_b(N1, N2)
    P = abi.dd2_params((0.0, 0.0, 0.0), 0.5, 0.25, 0.5, N1, lo1, hi1, o1, N2, lo2, hi2, o2, MZ, MG, precision,
                       gamma_series=gamma_series)
    h = min(h1, h2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pk = abi.dpm_dd2_pks_create(ctx, P, 1.0, 0.5 * h * h, 1, 0, 1, TEST_B_RHO0, TEST_B_C0, stream=stream)
    t_setup = time.perf_counter() - t0
    series, prev, stopped, rebuilds = [], None, "T reached", 0
    t0 = time.perf_counter()
    try:
        while True:
            st = abi.dpm_dd2_pks_step(pk, 1, True, stream=stream)
            rebuilds += int(st.rebuilt)
            row = {"step": int(st.step), "t": st.t, "dt": st.dt, "rebuilt": int(st.rebuilt), "max_rho": st.max_rho,
                   "min_rho": st.min_rho, "mass": st.mass, "m2": st.m2, "free_energy": st.free_energy}
            jump = abs(st.max_rho - prev) if prev is not None else 0.0
            if row["step"] % record_every == 0 or jump > stop_jump or st.t >= T:
                series.append(row)
            prev = st.max_rho
            if stop_jump > 0 and jump > stop_jump:
                stopped = "max density jump"
                break
            if st.t >= T:
                break
            if row["step"] >= max_steps:
                stopped = "step limit"
                break
    finally:
        torch.cuda.synchronize()
        abi.dpm_dd2_pks_destroy(pk)
    wall = time.perf_counter() - t0
    return {"N1": N1, "N2": N2, "h1": h1, "h2": h2, "MZ": MZ, "MG": MG, "gamma_series": gamma_series,
            "precision": precision,
            "steps": series[-1]["step"] if series else 0, "rebuilds": rebuilds, "stopped": stopped,
            "setup_s": t_setup, "wall_s": wall, "last": series[-1] if series else None, "series": series}


def layered_uneven_config(seed: int = 0, n_shells: int = 7, r_ball: float = 0.4, R: float = 1.0):
    """The uneven-box layered workload: a fine inner ball r < 0.4 on a 192^3 grid
    and n_shells concentric shells of equal thickness out to R = 1, shell grids
    N ~ U{48..128}, interface degrees K ~ U{6..10} (seeded), Gamma degree 8; each
    box [-r - 2.5h, r + 2.5h]^3 around its outer sphere, h = 2r/(N - 4) (half a
    cell more than two layers of margin, so that no node rounds onto the sphere
    within two layers of a face)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    radii = [r_ball] + [r_ball + (R - r_ball) * l / n_shells for l in range(1, n_shells + 1)]
    Ns = [192] + [int(v) for v in rng.integers(48, 129, size=n_shells)]
    Ks = [int(v) for v in rng.integers(6, 11, size=n_shells)]
    grids = []
    for r, N in zip(radii, Ns):
        h = 2.0 * r / (N - 4)
        grids.append((N, -r - 2.5 * h, r + 2.5 * h))
    return radii, grids, Ks, 8


def run_layers_uneven(ctx, steps: int = 200, seed: int = 0, precision=None, group: bool = True,
                      graph: bool = True, stream=None):
    """PKS steps of Test (A)'s data on the uneven-box layered decomposition
    (ball + 7 shells of different N, all sub-domain solves of the SIMT grids in
    one grouped set of launches per batch; with `graph`, every step one CUDA
    graph replay of the device-resident step).  dt: 0.9 x the CFL bound of the
    initial c on the finest grid (max |grad c0| = 5000 e^{-1/2}), fixed, so the
    stacked BEP is built once.  Returns the sizes, the build time, the time per
    step and the device time per step by kernel family (host-driven steps)."""
    import os

    import torch

    from . import abi
    from .workloads import TEST_A_C0, TEST_A_RHO0

    if precision is None:
        precision = abi.DPM_PREC_FP32
    radii, grids, Ks, KG = layered_uneven_config(seed)
    hmin = min((hi - lo) / (N + 1) for N, lo, hi in grids)
    gmax = 5000.0 * 2.718281828459045 ** -0.5
    dt = 0.9 * hmin / (6.0 * gmax)
    old = os.environ.get("DPM_DD_GROUP")
    os.environ["DPM_DD_GROUP"] = "1" if group else "0"
    try:
        P = abi.ml_params((0.0, 0.0, 0.0), radii, grids, Ks, KG, precision)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pk = abi.dpm_ml_pks_create(ctx, P, 1.0, dt, 0, 0, 1, TEST_A_RHO0, TEST_A_C0, stream=stream)
        abi.dpm_ml_pks_step(pk, 1, False, stream=stream)  # Steps 1-2 (the stacked BEP) + the first step
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        if graph:
            abi.dpm_ml_pks_set_graph(pk, True, stream=stream)
            abi.dpm_ml_pks_step(pk, 2, False, stream=stream)  # the uncaptured step, the capture
            torch.cuda.synchronize()
        t0 = time.perf_counter()
        abi.dpm_ml_pks_step(pk, steps, False, stream=stream)
        torch.cuda.synchronize()
        t_steps = time.perf_counter() - t0
        st = abi.dpm_ml_pks_step(pk, 0, True, stream=stream)
        if graph:
            abi.dpm_ml_pks_set_graph(pk, False, stream=stream)
        # device time per step by kernel family (the library's CUDA events)
        nprof = 5
        abi.dpm_profile_reset()
        abi.dpm_profile_enable(True)
        abi.dpm_ml_pks_step(pk, nprof, False, stream=stream)
        torch.cuda.synchronize()
        abi.dpm_profile_enable(False)
        fam = {"ap_simt32": "ap_simt32", "ap_simt64": "ap_simt64", "tc": "tc_", "lsq": "lsq_",
               "flux": "pks_flux", "diag": "pks_diag", "extend": "extend"}
        device = {k: abi.dpm_profile_read(v)[0] / nprof for k, v in fam.items()}
        device = {k: v for k, v in device.items() if v > 0}
        device["all"] = abi.dpm_profile_read(None)[0] / nprof
        abi.dpm_profile_reset()
        abi.dpm_ml_pks_destroy(pk)
    finally:
        if old is None:
            del os.environ["DPM_DD_GROUP"]
        else:
            os.environ["DPM_DD_GROUP"] = old
    grid_pts = sum(N ** 3 for N, _, _ in grids)
    return {"radii": radii, "N": [g[0] for g in grids], "K": Ks, "KG": KG, "dt": dt, "steps": steps,
            "grouped": group, "graph": graph, "first_step_with_build_s": t_build, "ms_per_step": 1e3 * t_steps / steps,
            "aps_per_step": 4 * len(grids), "grid_pts_per_step": 4 * grid_pts, "device_ms_per_step": device,
            "last": {"t": st.t, "max_rho": st.max_rho, "mass": st.mass, "free_energy": st.free_energy}}


def _mplus_mask(ctx, geom, N, lo, hi):
    import types

    import torch

    from . import abi
    lab = torch.empty(N ** 3, dtype=torch.uint8, device="cuda")
    g = geom if not isinstance(geom, tuple) else types.SimpleNamespace(kind=geom[0], center=geom[1],
                                                                       axes=geom[2])
    abi.dpm_classify(ctx, g, N, lo, hi, labels=lab)
    return (lab & abi.DPM_LBL_MPLUS) != 0


def run_time_convergence(ctx, N: int = 128, dd_grids=((128, 128), (128, 64)), taus=(16, 32, 64, 128, 256),
                         tau_ref: int = 512, dT: float = 1e-7, T: float = 1e-6, precision=None):
    """Convergence in time for Test (A) (Section 4): fixed meshes, dt = dT/tau,
    rho and c at the final time T against the run with dt = dT/tau_ref, the
    error E_t = max over M^+ (of each sub-domain) of the difference, and the
    rate log2(E_t(tau)/E_t(2 tau)).  The single domain runs on an N grid, the
    domain decomposition (ball r < 0.25, shell 0.25 < r < 0.5) on each (N1, N2)
    pair.  FP64 throughout: the differences reach 1e-12 of the values."""
    import math

    import torch

    from . import abi
    from .workloads import TEST_A_C0, TEST_A_RHO0, Geometry

    if precision is None:
        precision = abi.DPM_PREC_FP64
    tdt = torch.float64 if precision == abi.DPM_PREC_FP64 else torch.float32
    all_taus = sorted(set(taus) | {tau_ref})

    def nsteps(tau):
        return int(round(T * tau / dT))

    def sd_final(tau):
        lo, hi, h = paper_geometry_a(N)
        prm = abi.pks_params(Geometry.sphere(0.5), N, lo, hi, 1.0, dT / tau, 0, 1, precision,
                             dt_mode=0, rebuild=0, clamp=1)
        pk = abi.dpm_pks_create(ctx, prm, TEST_A_RHO0, TEST_A_C0)
        try:
            abi.dpm_pks_step(pk, nsteps(tau), False)
            st = abi.dpm_pks_step(pk, 0, True)
            rho = torch.empty(N ** 3, dtype=tdt, device="cuda")
            c = torch.empty_like(rho)
            abi.dpm_pks_get_state(pk, rho, c)
            torch.cuda.synchronize()
        finally:
            abi.dpm_pks_destroy(pk)
        return st.t, [(rho.double(), c.double())]

    def dd_final(N1, N2):
        def run(tau):
            r1, r2 = 0.25, 0.5
            lo1, hi1, _ = paper_geometry_a(N1, r1)
            lo2, hi2, _ = paper_geometry_a(N2, r2)
            P = abi.dd_params((0.0, 0.0, 0.0), r1, r2, N1, lo1, hi1, N2, lo2, hi2, 0, 0, precision)
            pk = abi.dpm_dd_pks_create(ctx, P, 1.0, dT / tau, 0, 0, 1, TEST_A_RHO0, TEST_A_C0)
            out = []
            try:
                abi.dpm_dd_pks_step(pk, nsteps(tau), False)
                st = abi.dpm_dd_pks_step(pk, 0, True)
                for l, Nl in enumerate((N1, N2)):
                    rho = torch.empty(Nl ** 3, dtype=tdt, device="cuda")
                    c = torch.empty_like(rho)
                    abi.dpm_dd_pks_get_state(pk, l, rho, c)
                    out.append((rho.double(), c.double()))
                torch.cuda.synchronize()
            finally:
                abi.dpm_dd_pks_destroy(pk)
            return st.t, out
        return run

    def study(run, masks):
        finals = {tau: run(tau) for tau in all_taus}
        ref = finals[tau_ref][1]
        rows = []
        for tau in sorted(taus):
            t, fields = finals[tau]
            row = {"tau": tau, "dt": dT / tau, "steps": nsteps(tau), "t": t}
            for l, ((rho, c), (rr, cr), m) in enumerate(zip(fields, ref, masks)):
                row[f"E_rho_{l}"] = float(torch.max(torch.where(m, (rho - rr).abs(), 0.0)))
                row[f"E_c_{l}"] = float(torch.max(torch.where(m, (c - cr).abs(), 0.0)))
            rows.append(row)
        for a, b in zip(rows, rows[1:]):
            for k in [k for k in a if k.startswith("E_")]:
                if a[k] > 0 and b[k] > 0:
                    b["rate_" + k[2:]] = math.log2(a[k] / b[k])
        return rows

    lo, hi, _ = paper_geometry_a(N)
    out = {"dT": dT, "T": T, "tau_ref": tau_ref, "precision": precision,
           "sd": {"N": N, "rows": study(sd_final, [_mplus_mask(ctx, Geometry.sphere(0.5), N, lo, hi)])},
           "dd": []}
    for N1, N2 in dd_grids:
        lo1, hi1, h1 = paper_geometry_a(N1, 0.25)
        lo2, hi2, h2 = paper_geometry_a(N2, 0.5)
        masks = [_mplus_mask(ctx, Geometry.sphere(0.25), N1, lo1, hi1),
                 _mplus_mask(ctx, (2, (0.0, 0.0, 0.0), (0.5, 0.25, 0.0)), N2, lo2, hi2)]
        out["dd"].append({"N1": N1, "N2": N2, "h1_over_h2": h1 / h2,
                          "rows": study(dd_final(N1, N2), masks)})
    return out


def main(argv=None):
    import argparse

    from . import abi

    ap = argparse.ArgumentParser(description="Test (A) to blow-up")
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--K", type=int, default=0)
    ap.add_argument("--T", type=float, default=6e-5)
    ap.add_argument("--stop-jump", type=float, default=0.0)
    ap.add_argument("--out", default="")
    ap.add_argument("--speedup", action="store_true",
                    help="single domain (N) against the domain decomposition, R_S = T_SD/T_DD")
    ap.add_argument("--time-convergence", action="store_true",
                    help="convergence in time at fixed meshes (N, DD 128/128 and 128/64), FP64")
    ap.add_argument("--layers", action="store_true",
                    help="the uneven-box layered decomposition (ball N=192 + 7 shells), grouped vs separate")
    ap.add_argument("--test-b", default="",
                    help="Test (B) with the Case 2 decomposition: N1/N2/MZ/MG, e.g. 128/128/20/150")
    ap.add_argument("--gamma-series", type=int, default=1,
                    help="Test (B): unknown series on Gamma, 1 (the paper's 2-term extension) or 2")
    ap.add_argument("--precision", choices=["tc32", "fft32", "fp32", "fp64"], default="tc32",
                    help="Test (B): AP solver (fft32: FFT-style at N = 256, tensor cores at N = 128)")
    a = ap.parse_args(argv)
    ctx = abi.dpm_ctx_create(0)
    if a.layers:
        out = [run_layers_uneven(ctx, group=True, graph=True), run_layers_uneven(ctx, group=True, graph=False),
               run_layers_uneven(ctx, group=False, graph=False)]
        abi.dpm_ctx_destroy(ctx)
        print(json.dumps(out))
        return
    if a.test_b:
        N1, N2, MZ, MG = (int(v) for v in a.test_b.split("/"))
        prec = {"tc32": abi.DPM_PREC_TC32, "fft32": abi.DPM_PREC_FFT32, "fp32": abi.DPM_PREC_FP32,
                "fp64": abi.DPM_PREC_FP64}[a.precision]
        res = run_test_b_dd(ctx, N1, N2, MZ, MG, precision=prec, T=a.T, gamma_series=a.gamma_series)
        abi.dpm_ctx_destroy(ctx)
        if a.out:
            with open(a.out, "w") as f:
                json.dump(res, f)
        print(json.dumps({k: v for k, v in res.items() if k != "series"}))
        return
    if a.time_convergence:
        print(json.dumps(run_time_convergence(ctx, a.N)))
        abi.dpm_ctx_destroy(ctx)
        return
    if a.speedup:
        print(json.dumps(sd_dd_speedup(ctx, a.N, T=a.T)))
        abi.dpm_ctx_destroy(ctx)
        return
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
