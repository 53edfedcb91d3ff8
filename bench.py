#!/usr/bin/env python
"""Benchmark of the DPM hot path on GB300.

Workload (default): the N=128 PKS workload -- unit sphere in [-1.25, 1.25]^3,
N = 128 interior nodes per axis, spherical harmonics to K = 8 (beta = 1, 162
BEP columns), dt = h^2/4, off-centre Gaussian data (1200 e^{-120|x-x0|^2},
600 e^{-60|x-x0|^2}, x0 = (0.3, 0, 0)).  One bench step is one PKS time step
of the main algorithm with the BEP rebuilt (Steps 3, 4a, 4b, 5, 6, 7): the
flux, 162 BEP-column APs + 2 particular APs in one batch, the FP64 QR, the
least squares, the extensions, 2 Green's-formula APs and the diagnostics.

metric: aux-solve grid-points/s = (APs per step) * N^3 / (seconds per step).

--impl reference times the CPU oracle (the only implementation the paper
gives is a description; the oracle restates it) on a bounded sample of the
same step's AP solves.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1811_03557_gb300.workloads import WORKLOADS  # noqa: E402

METRIC = "aux-solve grid-pts/s"
UNIT = "grid-pts/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="pks_sphere_N128_K8")
    ap.add_argument("--precision", choices=["fp32", "tc32", "fp64"], default="tc32")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="bound on the oracle's CPU-baseline sample")
    ap.add_argument("--cpu-fft-seconds", type=float, default=2.0,
                    help="bound on the scipy DST-I context sample (0 skips it)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=10000,
                    help="requests in the serving leg (0 skips it)")
    ap.add_argument("--serving-rate", type=float, default=1000.0, help="mean arrivals per second")
    ap.add_argument("--serving-models", type=int, default=64)
    ap.add_argument("--serving-saturated-rate", type=float, default=8000.0,
                    help="offered rate of the second, saturated serving leg (0 skips it)")
    ap.add_argument("--serving-saturated-requests", type=int, default=3000)
    ap.add_argument("--serving-slots", type=int, default=4,
                    help="serving worker slots (threads, each with its own stream and buffers)")
    ap.add_argument("--serving-batch", type=int, default=8, help="right-hand sides per serving batch at most")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving legs and print their JSON (tuning runs)")
    ap.add_argument("--no-aux", action="store_true", help="skip the batched aux-solve leg")
    ap.add_argument("--no-graph", action="store_true", help="host-driven steps instead of graph replay")
    ap.add_argument("--aux-case", default=None,
                    help="N:B:precision (fp32|tc32|fft32|fp64): time only this batched AP solve, "
                         "--warmup then --steps calls, and print its own JSON line (profiling cases)")
    ap.add_argument("--bep-case", default=None,
                    help="N:K:precision (fp32|tc32|fft32|fp64): time only the BEP build of the unit "
                         "sphere in [-1.25, 1.25]^3 with 2 (K+1)^2 columns (sparse shell right-hand "
                         "sides in, traces on gamma_in out), --warmup then --steps builds, and print "
                         "its own JSON line with the AP passes' times (profiling cases)")
    return ap.parse_args()


def whole_job_rate(ms_local, units_per_rank, dist=None, device="cpu"):
    """Replicas: every rank times the same K steps between barriers; the job's
    step time is the slowest rank's, and the whole-job rate counts the units of
    all ranks.  Returns (max ms per step over ranks, units per second)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    ms_max = float(t.item())
    return ms_max, world * units_per_rank / (ms_max / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
def oracle_sample(w, seconds, log=None):
    """Time the oracle's BEP-column AP solves (difference potential of a basis
    density, traced on gamma_in) of the workload for about `seconds`."""
    from oracle import dpm_oracle as O
    s = O.DPMSetup(w.geom, w.N, w.lo, w.hi, w.K, w.beta, 1.0 / w.dt, build_bep=False)
    Psi = s.basis_densities()
    n = 0
    t0 = time.perf_counter()
    while True:
        s.i_minus_p_gin(Psi[:, n % Psi.shape[1]])
        n += 1
        el = time.perf_counter() - t0
        if (el >= seconds and n >= 2) or n >= Psi.shape[1]:
            break
    return n, el


def fft_ap_solve(q, h, sigma, workers=1):
    """(sigma - Lap_h) u = q with zero Dirichlet data through scipy.fft's DST-I
    (the fast-Poisson route of the paper's FFTW-based solver): the CPU context
    figure reported beside the oracle.  Not used by the library."""
    import scipy.fft as sf
    N = q.shape[0]
    wt = (4.0 / (h * h)) * np.sin(np.pi * np.arange(1, N + 1) / (2.0 * (N + 1))) ** 2
    lam = sigma + wt[:, None, None] + wt[None, :, None] + wt[None, None, :]
    return sf.idstn(sf.dstn(q, type=1, workers=workers) / lam, type=1, workers=workers)


def cpu_fft_sample(w, seconds, cores):
    """Dense AP solves of the workload's grid by fft_ap_solve on `cores` host
    threads for about `seconds` (FP64, uniform q in [-1, 1], seed 0)."""
    N = w.N
    h, sigma = (w.hi - w.lo) / (N + 1), 1.0 / w.dt
    q = np.random.default_rng(0).uniform(-1.0, 1.0, (N, N, N))
    n = 0
    t0 = time.perf_counter()
    while True:
        fft_ap_solve(q, h, sigma, cores)
        n += 1
        el = time.perf_counter() - t0
        if (el >= seconds and n >= 2) or n >= 500:
            break
    return {"value": n * N ** 3 / el, "unit": UNIT, "cores": cores,
            "kind": "scipy.fft DST-I (FP64), context beside the oracle",
            "sample": f"{n} dense AP solves at N={N}, {el:.1f} s"}


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return int(max(i.get("num_threads", 1) for i in info))
    except Exception:
        pass
    return os.cpu_count() or 1


def solves_per_step(w):
    return w.ncol + 4


# ---------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    per = []
    sample_s = max(1.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        n, el = oracle_sample(w, sample_s)
        if i >= args.warmup:
            per.append((n, el))
    tot_n = sum(n for n, _ in per)
    tot_t = sum(t for _, t in per)
    value = tot_n * w.N ** 3 / tot_t
    ms_per_step = tot_t / len(per) * 1e3
    cores = blas_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "N": w.N, "K": w.K, "ncol": w.ncol,
                   "step": f"bounded sample of the step's AP solves (up to {sample_s:.0f} s of oracle work "
                           f"or the step's {w.ncol} BEP columns, whichever ends first)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{tot_n} BEP-column AP solves at N={w.N} over {len(per)} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    from paper_1811_03557_gb300 import abi

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    w = WORKLOADS[args.workload]
    if args.precision == "tc32" and w.N != 128:
        args.precision = "fp32"          # the tensor-core solver covers N = 128
    prec = {"fp32": abi.DPM_PREC_FP32, "tc32": abi.DPM_PREC_TC32, "fp64": abi.DPM_PREC_FP64}[args.precision]
    tdt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
    ctx = abi.dpm_ctx_create(local)
    # replicas: every rank advances its own independent copy of the workload.
    # dt = min(dt_prev, CFL bound, h^2/4) (Step 3; h^2/4 alone violates the CFL
    # bound of this data), and the BEP is rebuilt on every step (Step 4b).
    params = abi.pks_params(w.geom, w.N, w.lo, w.hi, 1.0, w.dt, w.K, w.beta, prec,
                            dt_mode=1, rebuild=1, clamp=1)
    stream = torch.cuda.Stream()
    pks = abi.dpm_pks_create(ctx, params, w.rho0, w.c0, stream=stream)
    N = w.N
    # each step replays one CUDA graph of the device-resident step (the
    # warm-up steps include the uncaptured sizing step and the capture)
    if not args.no_graph:
        abi.dpm_pks_set_graph(pks, True, stream=stream)
    for _ in range(args.warmup):
        abi.dpm_pks_step(pks, 1, want_stats=False, stream=stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    l0 = abi.dpm_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        abi.dpm_pks_step(pks, 1, want_stats=False, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    launches = abi.dpm_launch_count() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # per-kernel device times: the same step run without the graph, with the
    # library's CUDA events around every launch (not part of the timed region)
    abi.dpm_pks_set_graph(pks, False, stream=stream)
    abi.dpm_profile_reset()
    abi.dpm_profile_enable(True)
    nprof = max(3, min(args.steps, 10))
    for _ in range(nprof):
        abi.dpm_pks_step(pks, 1, want_stats=False, stream=stream)
    torch.cuda.synchronize()
    abi.dpm_profile_enable(False)
    spp = solves_per_step(w)
    ms_max, value = whole_job_rate(ms, spp * N ** 3, dist, device="cuda")

    # per-kernel device time recorded by the library on the launching stream
    kinds = ["pass_k_fwd", "pass_j", "pass_i", "pass_k_inv", "lsq_householder_qr",
             "lsq_gram_syrk", "lsq_cholesky", "tc_plane_fwd", "tc_pencil", "tc_plane_inv"]
    prof = {}
    for k in kinds:
        tot, n = abi.dpm_profile_read(k)
        if n:
            prof[k] = {"ms_total": tot, "launches": n, "ms_per_launch": tot / n}
    abi.dpm_profile_reset()

    st = abi.dpm_pks_step(pks, 1, want_stats=True, stream=stream)   # sanity after timing
    finite = bool(np.isfinite(st.mass) and st.min_rho >= -1e-6 * st.max_rho)

    roof = roofline(w, prec, prof, spp)
    # every AP pass of the step against its own algorithmic bytes (the dominant
    # one is `roofline`)
    roof_all = {k: {f: v for f, v in (roofline(w, prec, prof, spp, k) or {}).items()
                    if f in ("achieved", "frac", "bytes_per_launch", "traffic")}
                for k in prof if k.startswith("pass") or k.startswith("tc_")}

    e2e = None
    if not args.no_e2e:
        if not args.no_graph:
            abi.dpm_pks_set_graph(pks, True, stream=stream)
        e2e = run_e2e(abi, torch, pks, w, tdt, spp, args, stream)

    # the serving legs run right after the main leg, in the state a serving
    # process would be in: after the aux, decomposition and layered legs (tens of
    # GB allocated and freed) its host<->device copies ran 2x slower and its
    # latency tails 8x longer
    serving = None
    if rank == 0 and args.serving_requests > 0:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        serving = run_serving(abi, torch, ctx, args)

    aux = None
    if rank == 0 and not args.no_aux:
        aux = run_aux(abi, torch, ctx, stream)

    sd_dd = None
    if rank == 0 and not args.no_aux:
        # the paper's only performance figure: Test (A) to t = 6e-5, single domain
        # against the domain decomposition, R_S = T_SD / T_DD
        from paper_1811_03557_gb300.experiments import sd_dd_speedup
        sd_dd = sd_dd_speedup(ctx, 256, ((128, 128), (128, 64)), 6e-5)
        sd_dd["paper_R_S"] = {"255 vs 127/127": 6.46, "255 vs 127/63": 9.26,
                              "hardware": "32-core CPU node, FFTW3 + OpenMP"}
    layers = None
    if rank == 0 and not args.no_aux:
        # the uneven-box layered decomposition: ball N = 192 + 7 shells of seeded
        # N in [48, 128], every SIMT grid's solves in one grouped set of launches
        from paper_1811_03557_gb300.experiments import run_layers_uneven
        layers = run_layers_uneven(ctx, steps=200)
        layers["grid_pts_per_s"] = layers["grid_pts_per_step"] / (layers["ms_per_step"] / 1e3)

    cpu = None
    if rank == 0:
        n, el = oracle_sample(w, args.cpu_seconds)
        cpu = {"value": n * N ** 3 / el, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
               "sample": f"{n} BEP-column AP solves at N={N} (numpy FP64 dense DST-I), {el:.1f} s"}
    cpu_fft = None
    if rank == 0 and args.cpu_fft_seconds > 0:
        cpu_fft = cpu_fft_sample(w, args.cpu_fft_seconds, os.cpu_count() or 1)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "tc32": "f32 (3-term f16 split on tcgen05)", "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": w.name, "N": N, "K": w.K, "ncol": w.ncol, "solves_per_step": spp,
                       "step": "PKS step with BEP rebuild (Steps 3-7 incl. 4b), CFL dt <= h^2/4",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": f"inputs larger than L2 ({spp * N ** 3 * 4 / 1e9:.2f} GB batch per step)"},
            "clocks": clk, "gpu_launches": int(launches), "roofline": roof, "roofline_passes": roof_all,
            "kernels": prof,
            "e2e": e2e, "cpu_baseline": cpu, "cpu_fft_context": cpu_fft, "aux_solve": aux, "sd_dd_test_a": sd_dd, "layers_uneven": layers, "serving": serving,
            "graph": not args.no_graph, "kernel_profile_steps": nprof,
            "sanity": {"finite": bool(finite), "mass": st.mass},
        }
        print(json.dumps(line), flush=True)
    abi.dpm_pks_destroy(pks)
    abi.dpm_ctx_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()


# library profile key -> kernel name in the ncu summaries
KERNEL_OF_PROF = {"tc_plane_fwd": "k_tc_plane<0>", "tc_pencil": "k_tc_pencil", "tc_plane_inv": "k_tc_plane<1>",
                  "fft256_plane_fwd": "k_fft_plane_fwd", "fft256_pencil": "k_fft_pencil",
                  "fft256_plane_inv": "k_fft_plane_inv"}


def source_sha(path, root=None):
    import hashlib
    with open(os.path.join(root or ROOT, path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def profile_traffic(kernel, root=None):
    """DRAM bytes per right-hand side of `kernel` from the tables of profiles/*.md
    ('| kernel | DRAM bytes per right-hand side | source | source sha256 |'),
    or None when no table has it or the kernel's source file has changed since
    the capture (its sha256 prefix differs)."""
    import glob
    root = root or ROOT
    for md in sorted(glob.glob(os.path.join(root, "profiles", "*.md"))):
        header = False
        for line in open(md):
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) == 4 and cells[1].startswith("DRAM bytes per right-hand side"):
                header = True
                continue
            if header and len(cells) == 4 and cells[0].replace("\\", "") == kernel:
                try:
                    return float(cells[1]) if source_sha(cells[2], root) == cells[3] else None
                except (OSError, ValueError):
                    return None
            if header and not line.startswith("|"):
                header = False
    return None


def roofline(w, prec, prof, spp, name=None):
    """Roofline of the dominant AP-pass kernel (largest device time), or of the
    pass `name`."""
    peaks, src = measured_peaks()
    passes = {k: v for k, v in prof.items() if k.startswith("pass") or k.startswith("tc_")}
    tc = prec == 2
    if not passes:
        return None
    if name is None:
        name, rec = max(passes.items(), key=lambda kv: kv[1]["ms_total"])
    else:
        rec = passes[name]
    N = w.N
    # right-hand sides per launch: every step runs one batch of (ncol + 2) and one of 2
    batches = [(w.ncol + 2), 2]
    rhs_per_launch = sum(batches) / len(batches)
    points = rhs_per_launch * N ** 3
    if prec in (0, 1):  # SIMT: fused-multiply-add bound
        H = N // 2
        passes_per_kind = {"pass_i": 2, "pass_j": 1, "pass_k_fwd": 1, "pass_k_inv": 1}
        nt = passes_per_kind.get(name, 1)
        flops = points * nt * (2.0 * H + 1.0)          # folded transform: N/2 FMAs + 1 add per point
        ach = flops / (rec["ms_per_launch"] / 1e3) / 1e12
        sm_max = peaks.get("sm_max_mhz", 2070.0)
        lanes = 128 if prec == 0 else 2                  # FP32 lanes / FP64 units per SM
        peak = 152 * lanes * 2 * sm_max * 1e6 / 1e12
        return {"bound": "alu", "kernel": name, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None,
                "peak_source": f"152 SMs x {lanes} lanes x 2 flop x {sm_max:.0f} MHz (derived)"}
    # tensor-core passes: algorithmic HBM bytes per launch, averaged over the
    # step's two batches (ncol sparse-RHS BEP columns + 2 dense-f particular
    # solves traced on gamma_in; then 2 Green's solves with dense output).
    n3 = float(N) ** 3
    c = w.ncol
    per_kernel = {
        # reads: f (4 B) + labels (1 B) for dense-f RHS; writes the 4 B cube
        "tc_plane_fwd": ((c * 4 + 2 * 9) * n3 + 2 * 9 * n3) / 2,
        # reads and writes the 4 B cube
        "tc_pencil": ((c + 2) * 8 * n3 + 2 * 8 * n3) / 2,
        # reads the cube; dense outputs also write it and read the labels
        "tc_plane_inv": ((c + 2) * 4 * n3 + 2 * 9 * n3) / 2,
    }
    bytes_per = per_kernel.get(name, points * 8.0)
    ach = bytes_per / (rec["ms_per_launch"] / 1e3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    # measured DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per
    # right-hand side from the committed ncu summary of these kernels, scaled to
    # the step's average launch; None when the kernel's source changed since
    per_rhs = profile_traffic(KERNEL_OF_PROF.get(name, name))
    traffic = per_rhs * rhs_per_launch if per_rhs is not None else None
    return {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "traffic": traffic, "bytes_per_launch": bytes_per,
            "peak_source": f"hbm_gbs ({src})"}


def run_aux(abi, torch, ctx, stream):
    """Batched auxiliary solves alone (Definition 2.4), dense uniform-random q
    in [-1, 1] (seed 0), inputs resident and larger than L2: the tensor-core
    solver at N = 128 with the 162-column batch, the FP32 SIMT solver and the
    plain FP64 solver (one right-hand side per call) at N = 256, and the N = 256
    tensor-core and FFT-style solvers.  Roofline: 24 bytes per grid point per FP32
    solve is the algorithmic minimum (three passes over a cube that does not fit
    on chip); the three-pass (tensor-core N = 128, FFT-style N = 256), five-pass
    (SIMT) and assemble + six-pass (tensor-core, N = 256, the last pass writing u)
    schedules move 24, 24, 40 and 56.  The N = 256, K = 12 BEP batch is built with
    both N = 256 solvers."""
    from paper_1811_03557_gb300.workloads import random_rhs
    peaks, src = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)

    def timed(N, B, prec, reps, calls=1):
        h = 2.5 / (N + 1)
        tdt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
        q = torch.from_numpy(random_rhs(0, B, N)).to("cuda", tdt)
        u = torch.empty_like(q)
        sigma = 1.0 / 1e-4 + 1.0
        for _ in range(2):
            abi.dpm_aux_solve_batched(ctx, N, h, sigma, B, q, u, prec, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            for c in range(calls):
                abi.dpm_aux_solve_batched(ctx, N, h, sigma, B // calls, q[c * (B // calls):],
                                          u[c * (B // calls):], prec, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        del q, u
        return ms, B * N ** 3 / (ms / 1e3)

    def leg(ms, v, N, B, sched, alg_bpp=24):
        # frac: against the algorithmic minimum of a dense solve whose cube does not
        # fit on chip, 24 bytes per grid point (read + write of one cube in each of
        # three passes; 8 when the cube fits in shared memory); frac_schedule:
        # against the bytes the kernels' schedule moves
        alg = alg_bpp * B * N ** 3 / (ms / 1e3) / 1e9
        sch = sched * B * N ** 3 / (ms / 1e3) / 1e9
        return {"ms": ms, "grid_pts_per_s": v, "hbm_gbs": alg, "frac": alg / hbm, "alg_bytes_per_pt": alg_bpp,
                "schedule_bytes_per_pt": sched, "schedule_gbs": sch, "frac_schedule": sch / hbm}

    out = {}
    ms, v = timed(128, 162, abi.DPM_PREC_TC32, 5)
    out["tc32_N128_B162"] = leg(ms, v, 128, 162, 24)   # plane, pencil, plane
    # N = 32 (the elliptic workload's grid): the cube in shared memory, one pass;
    # 1,024 right-hand sides so that the 134 MB in and out exceed L2
    ms, v = timed(32, 1024, abi.DPM_PREC_FP32, 10)
    out["fp32_N32_B1024"] = leg(ms, v, 32, 1024, 8, alg_bpp=8)
    ms, v = timed(256, 16, abi.DPM_PREC_TC32, 3)
    # assemble (read f, write q), five out-of-place passes, the last one writing u
    out["tc32_N256_B16"] = leg(ms, v, 256, 16, 56)
    ms, v = timed(256, 16, abi.DPM_PREC_FFT32, 3)
    out["fft32_N256_B16"] = leg(ms, v, 256, 16, 24)     # plane, pencil, plane (in place)
    ms, v = timed(256, 16, abi.DPM_PREC_FP32, 3)
    out["fp32_N256_B16"] = leg(ms, v, 256, 16, 40)      # five in-place passes
    out["fp32_N256_B16"]["simt_tile"] = abi.dpm_simt_tile(256, abi.DPM_PREC_FP32, 16)
    ms, v = timed(256, 2, abi.DPM_PREC_FP64, 1, calls=2)   # two calls of one right-hand side
    out["fp64_N256_per_solve"] = {"ms": ms / 2, "grid_pts_per_s": v,
                                  "simt_tile": abi.dpm_simt_tile(256, abi.DPM_PREC_FP64, 1)}
    # the BEP batch workload: ellipsoid (1, 0.8, 0.6) in [-1.2, 1.2]^3, N = 256,
    # K = 12 (338 columns in one batched solve), sigma = 1/dt + 1, dt = 1e-4
    from paper_1811_03557_gb300.workloads import WORKLOADS
    wb = WORKLOADS["bep_ellipsoid_N256_K12"]
    # the AP phase of the build against the algorithmic bytes of a BEP column:
    # 16 N^3 (one cube written and read in the middle of the transform; the sparse
    # input and the trace output are not cubes) + 8 (|gamma| + |gamma_in|)
    ap_keys = {abi.DPM_PREC_TC32: ("tc256_rhs", "tc256_k", "tc256_j", "tc256_i", "tc256_k_out"),
               abi.DPM_PREC_FFT32: ("fft256_rhs", "fft256_plane_fwd", "fft256_pencil", "fft256_plane_inv")}
    for prec, key in ((abi.DPM_PREC_TC32, "bep_build_N256_K12_tc32"),
                      (abi.DPM_PREC_FFT32, "bep_build_N256_K12_fft32")):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bep = abi.dpm_bep_build(ctx, wb.geom, wb.N, wb.lo, wb.hi, wb.sigma, wb.K, wb.beta, prec, stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        abi.dpm_profile_reset()
        abi.dpm_profile_enable(True)
        bep2 = abi.dpm_bep_build(ctx, wb.geom, wb.N, wb.lo, wb.hi, wb.sigma, wb.K, wb.beta, prec, stream)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        abi.dpm_profile_enable(False)
        per = {k: abi.dpm_profile_read(k)[0] for k in ap_keys[prec]}
        ap_ms = sum(per.values())
        fac_ms = sum(abi.dpm_profile_read(k)[0] for k in ("lsq_gram_syrk", "lsq_cholesky"))
        abi.dpm_profile_reset()
        info = abi.dpm_bep_get_info(bep2)
        abi.dpm_bep_destroy(bep)
        abi.dpm_bep_destroy(bep2)
        ncol = wb.ncol
        alg = ncol * (16.0 * wb.N ** 3 + 8.0 * (info.n_gamma + info.n_gin))
        gbs = alg / (ap_ms / 1e3) / 1e9 if ap_ms > 0 else None
        out[key] = {"build_ms": (t2 - t1) * 1e3, "first_build_ms": (t1 - t0) * 1e3, "ap_ms": ap_ms,
                    "ap_kernels_ms": per, "factor_ms": fac_ms, "ncol": ncol,
                    "ap_grid_pts_per_s": ncol * wb.N ** 3 / (ap_ms / 1e3) if ap_ms > 0 else None,
                    "ap_alg_bytes": alg, "ap_hbm_gbs": gbs, "ap_frac": gbs / hbm if gbs else None}
    out["peak"] = {"hbm_gbs": hbm, "source": src}
    out["data"] = "uniform [-1, 1] q, seed 0; dense in, dense out; inputs larger than L2"
    return out


def run_e2e(abi, torch, pks, w, tdt, spp, args, stream):
    """Same metric through the public API with host buffers: each step copies
    the state (rho, c) host->device, steps, and copies it device->host."""
    N = w.N
    # warm-up outside the timed region (with graph stepping: the sizing step and the capture)
    abi.dpm_pks_step(pks, 2, want_stats=False, stream=stream)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        rho_h = torch.empty((N, N, N), dtype=tdt).pin_memory()
        c_h = torch.empty_like(rho_h).pin_memory()
        rho_d = torch.empty((N, N, N), dtype=tdt, device="cuda")
        c_d = torch.empty_like(rho_d)
        abi.dpm_pks_get_state(pks, rho_d, c_d, stream=stream)
        rho_h.copy_(rho_d)
        c_h.copy_(c_d)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        K = max(1, min(args.steps, 5))
        e0.record(stream)
        for _ in range(K):
            rho_d.copy_(rho_h, non_blocking=True)
            c_d.copy_(c_h, non_blocking=True)
            abi.dpm_pks_set_state(pks, rho_d, c_d, stream=stream)
            abi.dpm_pks_step(pks, 1, want_stats=False, stream=stream)
            abi.dpm_pks_get_state(pks, rho_d, c_d, stream=stream)
            rho_h.copy_(rho_d, non_blocking=True)
            c_h.copy_(c_d, non_blocking=True)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    nb = 2 * N ** 3 * rho_h.element_size()
    return {"value": spp * N ** 3 / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": nb,
            "d2h_bytes_per_step": nb, "ms_per_step": ms}


def run_serving(abi, torch, ctx, args):
    """Serving legs: seeded Poisson streams of elliptic solves (and a few short
    PKS runs) over one catalog of resident factorisations drawn from the
    serving mix (N in {32, 64, 128, 256}, K in 4..12, sigma log-uniform in
    [1e2, 1e5], spheres and ellipsoids with radius in [0.5, 1]): the stream of
    --serving-requests at --serving-rate, then a saturated one (arrivals faster
    than the service rate, so batches form).  Latency is arrival -> solution
    back in host memory (copies included), split into build wait, slot wait and
    service (host->device copy, solve, device->host copy on the device)."""
    from paper_1811_03557_gb300.serving import LibraryBackend, ServingEngine
    from paper_1811_03557_gb300.workloads import (pks_run_catalog, poly_gauss_rhs,
                                                  serving_catalog, serving_stream)
    cat = serving_catalog(0, args.serving_models)
    pcat = pks_run_catalog(1, 4)
    legs = [("stream", 0, args.serving_requests, args.serving_rate)]
    if args.serving_saturated_rate > 0 and args.serving_saturated_requests > 0:
        legs.append(("saturated", 7, args.serving_saturated_requests, args.serving_saturated_rate))
    streams = {name: serving_stream(seed, n, rate, len(cat), len(pcat), 0.005) for name, seed, n, rate in legs}
    pool = {}
    for reqs in streams.values():
        for q in reqs:
            if q.kind == "solve" and q.rhs_seed not in pool:
                pool[q.rhs_seed] = torch.from_numpy(poly_gauss_rhs(q.rhs_seed, cat[q.model])).pin_memory()
    slots, batch = args.serving_slots, args.serving_batch
    be = LibraryBackend(ctx, slots, batch, max(m.N for m in cat))
    eng = ServingEngine(be, cat, pcat, n_slots=slots, max_batch=batch, rhs=lambda s, m: pool[s])
    t = time.perf_counter()
    warm = eng.warm()
    t_warm = time.perf_counter() - t
    out = {"catalog": len(cat), "resident_after_warm": warm, "warm_s": t_warm, "slots": slots,
           "max_batch": batch,
           "latency": "arrival -> solution in pinned host memory (H2D and D2H included)",
           "precision": "f32 storage (tcgen05 3-term f16 split at N=128, FFT-style FP32 at N=256, "
                        "SIMT FP32 otherwise), FP64 least squares"}
    for name, seed, n, rate in legs:
        l0 = abi.dpm_launch_count()
        rep = eng.run(streams[name])
        launches = abi.dpm_launch_count() - l0
        torch.cuda.synchronize()
        d = {k: v for k, v in rep.as_dict().items() if k != "errors"}
        d.update(requests=n, rate_hz=rate, gpu_launches=int(launches), errors=rep.errors)
        out[name] = d
    eng.shutdown()
    torch.cuda.synchronize()
    return out


def run_aux_case(args):
    """One batched AP solve configuration alone (a small case for kernel captures)."""
    import torch
    from paper_1811_03557_gb300 import abi
    from paper_1811_03557_gb300.workloads import random_rhs
    N, B, pname = args.aux_case.split(":")
    N, B = int(N), int(B)
    prec = {"fp32": abi.DPM_PREC_FP32, "tc32": abi.DPM_PREC_TC32, "fft32": abi.DPM_PREC_FFT32,
            "fp64": abi.DPM_PREC_FP64}[pname]
    torch.cuda.set_device(0)
    ctx = abi.dpm_ctx_create(0)
    tdt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
    q = torch.from_numpy(random_rhs(0, B, N)).to("cuda", tdt)
    u = torch.empty_like(q)
    h, sigma = 2.5 / (N + 1), 1e4 + 1.0
    stream = torch.cuda.Stream()
    for _ in range(args.warmup):
        abi.dpm_aux_solve_batched(ctx, N, h, sigma, B, q, u, prec, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        abi.dpm_aux_solve_batched(ctx, N, h, sigma, B, q, u, prec, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    peaks, _ = measured_peaks()
    gbs = 24.0 * B * N ** 3 / (ms / 1e3) / 1e9
    print(json.dumps({"aux_case": args.aux_case, "ms": ms, "grid_pts_per_s": B * N ** 3 / (ms / 1e3),
                      "alg_gbs": gbs, "frac": gbs / peaks.get("hbm_gbs", 6800.0)}), flush=True)
    abi.dpm_ctx_destroy(ctx)


def run_bep_case(args):
    """One BEP build alone: the AP passes on sparse shell right-hand sides with
    trace output, as in every PKS step (a small case for kernel captures)."""
    import torch
    from paper_1811_03557_gb300 import abi
    from paper_1811_03557_gb300.workloads import Geometry
    N, K, pname = args.bep_case.split(":")
    N, K = int(N), int(K)
    prec = {"fp32": abi.DPM_PREC_FP32, "tc32": abi.DPM_PREC_TC32, "fft32": abi.DPM_PREC_FFT32,
            "fp64": abi.DPM_PREC_FP64}[pname]
    torch.cuda.set_device(0)
    ctx = abi.dpm_ctx_create(0)
    lo, hi = -1.25, 1.25
    h = (hi - lo) / (N + 1)
    sigma = 4.0 / (h * h) + 1.0      # 1/dt + 1 at the PKS step's dt = h^2/4
    stream = torch.cuda.Stream()
    build = lambda: abi.dpm_bep_build(ctx, Geometry.sphere(1.0), N, lo, hi, sigma, K, 1, prec, stream)
    for _ in range(args.warmup):
        abi.dpm_bep_destroy(build())
    torch.cuda.synchronize()
    abi.dpm_profile_reset()
    abi.dpm_profile_enable(True)
    ms = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        bep = build()
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t0) * 1e3)
        info = abi.dpm_bep_get_info(bep)
        abi.dpm_bep_destroy(bep)
    abi.dpm_profile_enable(False)
    keys = ("tc_shell_rhs", "tc_plane_fwd", "tc_pencil", "tc_plane_inv", "lsq_gram_syrk", "lsq_cholesky")
    per = {k: abi.dpm_profile_read(k)[0] / max(1, args.steps) for k in keys}
    abi.dpm_profile_reset()
    print(json.dumps({"bep_case": args.bep_case, "ncol": info.ncol, "n_gamma": info.n_gamma,
                      "n_gin": info.n_gin, "build_ms": float(np.median(ms)) if ms else None,
                      "kernels_ms": per}), flush=True)
    abi.dpm_ctx_destroy(ctx)


def main():
    args = parse()
    if args.aux_case and args.impl != "reference":
        run_aux_case(args)
        return
    if args.bep_case and args.impl != "reference":
        run_bep_case(args)
        return
    if args.serving_only and args.impl != "reference":
        import torch
        from paper_1811_03557_gb300 import abi
        torch.cuda.set_device(0)
        ctx = abi.dpm_ctx_create(0)
        print(json.dumps({"serving": run_serving(abi, torch, ctx, args)}), flush=True)
        abi.dpm_ctx_destroy(ctx)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
