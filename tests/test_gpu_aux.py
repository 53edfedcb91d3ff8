"""GPU parity of the batched auxiliary-problem solve (Definition 2.4) against
the oracle's dense DST-I, through dpm_aux_solve_batched.

Tolerances (relative L-inf over the output, max|u - u_ref| / max|u_ref|):
FP32 storage/arithmetic 1e-5, FP64 1e-11."""
import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import random_rhs

pytestmark = pytest.mark.gpu

TOL = {abi.DPM_PREC_FP32: 1e-5, abi.DPM_PREC_FP64: 1e-11}


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def gpu_solve(ctx, q, h, sigma, prec):
    B, N = q.shape[0], q.shape[1]
    dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
    qd = torch.from_numpy(q).to("cuda", dt).contiguous()
    ud = torch.empty_like(qd)
    abi.dpm_aux_solve_batched(ctx, N, h, sigma, B, qd, ud, prec)
    torch.cuda.synchronize()
    return ud.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec", [abi.DPM_PREC_FP32, abi.DPM_PREC_FP64])
@pytest.mark.parametrize("N,B,h,sigma", [(2, 1, 0.3, 1.0), (7, 3, 0.2, 10.0), (16, 2, 0.05, 1001.0),
                                         (33, 2, 2.5 / 34, 1001.0), (50, 1, 0.02, 1e4),
                                         (64, 3, 0.04, 0.0)])
def test_matches_oracle(ctx, prec, N, B, h, sigma):
    q = random_rhs(N * 7 + B, B, N, np.float64)
    if prec == abi.DPM_PREC_FP32:
        q = q.astype(np.float32).astype(np.float64)
    u = gpu_solve(ctx, q, h, sigma, prec)
    for b in range(B):
        ref = O.aux_solve(q[b], h, sigma)
        assert rel_linf(u[b], ref) < TOL[prec], (b, rel_linf(u[b], ref))


@pytest.mark.parametrize("prec", [abi.DPM_PREC_FP32, abi.DPM_PREC_FP64])
def test_in_place_and_batch_independence(ctx, prec):
    N, h, sigma = 24, 0.1, 50.0
    q = random_rhs(5, 4, N, np.float64).astype(np.float32).astype(np.float64)
    dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
    qd = torch.from_numpy(q).to("cuda", dt).contiguous()
    alone = gpu_solve(ctx, q[2:3], h, sigma, prec)
    abi.dpm_aux_solve_batched(ctx, N, h, sigma, 4, qd, qd, prec)   # in place
    torch.cuda.synchronize()
    assert np.array_equal(qd.cpu().numpy()[2].astype(np.float64), alone[0])


def test_full_size_N256_residual_property(ctx):
    """N = 256, 2 right-hand sides, in the FP32 path: the 7-point residual
    (sigma - Lap_h) u - q, evaluated in FP64 with torch, stays within FP32
    rounding amplified by the operator norm."""
    N, B = 256, 2
    h, sigma = 2.4 / 257, 1e4 + 1.0
    q = torch.from_numpy(random_rhs(11, B, N, np.float32)).cuda()
    u = torch.empty_like(q)
    abi.dpm_aux_solve_batched(ctx, N, h, sigma, B, q, u, abi.DPM_PREC_FP32)
    torch.cuda.synchronize()
    for b in range(B):
        ud = torch.nn.functional.pad(u[b].double(), (1, 1, 1, 1, 1, 1))
        c = ud[1:-1, 1:-1, 1:-1]
        lap = (ud[2:, 1:-1, 1:-1] + ud[:-2, 1:-1, 1:-1] + ud[1:-1, 2:, 1:-1] + ud[1:-1, :-2, 1:-1]
               + ud[1:-1, 1:-1, 2:] + ud[1:-1, 1:-1, :-2] - 6 * c) / h ** 2
        r = (sigma * c - lap - q[b].double()).abs().max().item()
        # FP32 solution error ~1e-7 relative, amplified by the operator norm sigma + 12/h^2
        bound = 1e-5 * (sigma + 12 / h ** 2) * u[b].abs().max().item()
        assert r < bound, (r, bound)


@pytest.mark.parametrize("prec", [abi.DPM_PREC_FP32, abi.DPM_PREC_FP64])
def test_full_size_N256_matches_oracle(ctx, prec):
    """The SIMT solver at N = 256 (the autotuner's widest-row tiles) against the
    oracle's dense DST-I, one right-hand side, at the path's tolerance."""
    N = 256
    h, sigma = 2.4 / 257, 1e4 + 1.0
    q = random_rhs(13, 1, N, np.float32).astype(np.float64)
    u = gpu_solve(ctx, q, h, sigma, prec)
    e = rel_linf(u[0], O.aux_solve(q[0], h, sigma))
    print(f"SIMT N=256 prec={prec}: rel err {e:.3e}")
    assert e < TOL[prec], e


def test_solve_on_a_second_device(ctx):
    """Kernel attributes (the dynamic shared memory limits above 48 KB) belong to
    each device's context: after solves on device 0, the same solves on device 1
    in the same process must still run and agree."""
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible devices")
    N, B, h, sigma = 128, 2, 2.5 / 129, 1e4 + 1.0
    q = random_rhs(77, B, N, np.float32)
    outs = []
    for dev in (0, 1):
        with torch.cuda.device(dev):
            c = ctx if dev == 0 else abi.dpm_ctx_create(1)
            for prec in (abi.DPM_PREC_FP32, abi.DPM_PREC_TC32):
                qd = torch.from_numpy(q).to(f"cuda:{dev}")
                ud = torch.empty_like(qd)
                abi.dpm_aux_solve_batched(c, N, h, sigma, B, qd, ud, prec)
                torch.cuda.synchronize(dev)
                outs.append(ud.cpu().numpy())
            if dev == 1:
                abi.dpm_ctx_destroy(c)
    np.testing.assert_array_equal(outs[0], outs[2])
    np.testing.assert_array_equal(outs[1], outs[3])
