"""GPU test of dpm_aux_solve_batched_noalloc, the allocation-free FP32 AP
solve meant for callers that cannot let a library allocate device memory.

Through the C ABI it must agree with dpm_aux_solve_batched (FP32) and with the
oracle's FP64 solve within the 1e-5 relative L-inf tolerance of the AP parity
tests, on two calls in a row with different inputs (the shared static scratch
keeps the previous call's contents), must not change the free device memory on
either call, and must reject a batch beyond its fixed workspace (by total size
and by count).  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import random_rhs

pytestmark = pytest.mark.gpu


def rel_linf(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("N,B,h,sigma", [(33, 3, 2.5 / 34, 1001.0), (128, 2, 2.5 / 129, 3.0e4)])
def test_noalloc_matches_batched_entry_point(ctx, N, B, h, sigma):
    outs = []
    for call, seed in enumerate((101 + N, 202 + N)):
        q = torch.from_numpy(random_rhs(seed, B, N, np.float32)).cuda()
        ref = torch.empty_like(q)
        abi.dpm_aux_solve_batched(ctx, N, h, sigma, B, q, ref, abi.DPM_PREC_FP32)
        u = torch.full_like(q, float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        abi.dpm_aux_solve_batched_noalloc(N, h, sigma, B, q, u)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        # nothing allocated by either call (the library's module, and with it the
        # static array, is resident since the dpm_aux_solve_batched call above)
        assert free_after >= free_before, (call, free_before - free_after)
        assert torch.isfinite(u).all()
        e = rel_linf(u.double(), ref.double())
        assert e < 1e-5, (call, e)
        qh = q.cpu().numpy().astype(np.float64)
        uh = u.cpu().numpy().astype(np.float64)
        for b in range(B):
            uo = O.aux_solve(qh[b], h, sigma)
            eo = float(np.max(np.abs(uh[b] - uo)) / np.max(np.abs(uo)))
            assert eo < 1e-5, (call, b, eo)
        outs.append(u)
    assert not torch.equal(outs[0], outs[1])


def test_noalloc_in_place(ctx):
    N, B, h, sigma = 40, 2, 0.05, 100.0
    q = torch.from_numpy(random_rhs(7, B, N, np.float32)).cuda()
    ref = torch.empty_like(q)
    abi.dpm_aux_solve_batched(ctx, N, h, sigma, B, q, ref, abi.DPM_PREC_FP32)
    abi.dpm_aux_solve_batched_noalloc(N, h, sigma, B, q, q)
    torch.cuda.synchronize()
    assert rel_linf(q.double(), ref.double()) < 1e-5


def test_noalloc_rejects_batches_beyond_the_static_workspace(ctx):
    N = 256
    q = torch.zeros(2, N, N, N, device="cuda")
    with pytest.raises(abi.DPMError) as e:
        abi.dpm_aux_solve_batched_noalloc(N, 0.01, 1.0, 2, q, q)
    assert e.value.code == abi.DPM_EINVAL
    assert "static workspace" in str(e.value)


def test_noalloc_rejects_more_than_1024_right_hand_sides(ctx):
    N = 8                                  # 1025 * 8^3 floats fit the workspace; the count does not
    q = torch.zeros(1025, N, N, N, device="cuda")
    with pytest.raises(abi.DPMError) as e:
        abi.dpm_aux_solve_batched_noalloc(N, 0.1, 1.0, 1025, q, q)
    assert e.value.code == abi.DPM_EINVAL
    u = torch.empty(1024, N, N, N, device="cuda")
    abi.dpm_aux_solve_batched_noalloc(N, 0.1, 1.0, 1024, q[:1024].contiguous(), u)
    torch.cuda.synchronize()
    assert torch.count_nonzero(u) == 0
