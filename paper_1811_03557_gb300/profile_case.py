"""Profiling cases: the BEP assembly of the N = 128, K = 8 sphere workload
(default), batched dense solves at N = 256 (--case aux256), or two PKS time
steps of the N = 128 sphere workload with the BEP rebuilt (--case pks128).

Builds the BEP twice (the first build creates the per-device tables) through
the C ABI; each build runs classification, the gamma geometry, one batched
auxiliary solve of the 162 basis columns and the least-squares factorisation.
Meant to be run under ncu with a kernel filter, e.g.

    python -m paper_1811_03557_gb300.profile_case --precision tc32
"""
from __future__ import annotations

import argparse


def main():
    import torch

    from . import abi
    from .workloads import WORKLOADS

    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", choices=["fp32", "tc32", "fp64"], default="tc32")
    ap.add_argument("--builds", type=int, default=2)
    ap.add_argument("--case", choices=["bep128", "aux256", "pks128"], default="bep128",
                    help="bep128: the BEP build above; aux256: two batched solves of 4 dense "
                         "right-hand sides at N = 256 on the tensor-core solver; pks128: two "
                         "host-driven PKS steps (Test (A) data, CFL time step, BEP rebuilt)")
    args = ap.parse_args()
    if args.case == "aux256":
        from .workloads import random_rhs
        ctx = abi.dpm_ctx_create(0)
        q = torch.from_numpy(random_rhs(0, 4, 256)).cuda()
        u = torch.empty_like(q)
        for _ in range(2):
            abi.dpm_aux_solve_batched(ctx, 256, 2.4 / 257, 1e4 + 1.0, 4, q, u, abi.DPM_PREC_TC32)
        torch.cuda.synchronize()
        abi.dpm_ctx_destroy(ctx)
        print("profile case done")
        return
    prec = {"fp32": abi.DPM_PREC_FP32, "tc32": abi.DPM_PREC_TC32, "fp64": abi.DPM_PREC_FP64}[args.precision]
    w = WORKLOADS["pks_sphere_N128_K8"]
    if args.case == "pks128":
        ctx = abi.dpm_ctx_create(0)
        prm = abi.pks_params(w.geom, w.N, w.lo, w.hi, 1.0, w.dt, w.K, w.beta, prec, dt_mode=1, rebuild=1,
                             clamp=1)
        pk = abi.dpm_pks_create(ctx, prm, w.rho0, w.c0)
        for _ in range(2):
            abi.dpm_pks_step(pk, 1, False)
        torch.cuda.synchronize()
        abi.dpm_pks_destroy(pk)
        abi.dpm_ctx_destroy(ctx)
        print("profile case done")
        return
    ctx = abi.dpm_ctx_create(0)
    for _ in range(args.builds):
        b = abi.dpm_bep_build(ctx, w.geom, w.N, w.lo, w.hi, 1.0 / w.dt, w.K, w.beta, prec)
        abi.dpm_bep_destroy(b)
    torch.cuda.synchronize()
    abi.dpm_ctx_destroy(ctx)
    print("profile case done")


if __name__ == "__main__":
    main()
