"""Several host threads driving the library at once, as the serving loop does:
each thread solves batches against its own factorisation (different column
counts, so different launch sizes of the least-squares kernels) on its own
stream.  Every call must succeed and give the same result as the same solve
run alone."""
import threading

import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import Geometry

pytestmark = pytest.mark.gpu


def test_concurrent_batched_solves_from_threads(ctx):
    N, lo, hi, sigma = 32, -1.25, 1.25, 2.0e3
    Ks = (4, 7, 9, 11)               # 50 .. 288 columns: small and large trisolve launches
    nreq = 8
    beps = [abi.dpm_bep_build(ctx, Geometry.sphere(1.0), N, lo, hi, sigma, K, 1, abi.DPM_PREC_FP32) for K in Ks]
    for b in beps:
        abi.dpm_bep_reserve(b, nreq)
    X, Y, Z = O.mesh(N, lo, hi)
    f = np.stack([np.exp(-(X - 0.1 * r) ** 2 - Y ** 2 - Z ** 2) for r in range(nreq)]).astype(np.float32)
    fd = torch.from_numpy(f).cuda()
    ref = []
    for b in beps:
        u = torch.empty_like(fd)
        abi.dpm_solve_batched(b, [fd[r] for r in range(nreq)], [u[r] for r in range(nreq)])
        torch.cuda.synchronize()
        ref.append(u.cpu())
    errors, outs = [], {}

    def work(i):
        try:
            s = torch.cuda.Stream()
            u = torch.empty_like(fd)
            for _ in range(25):
                abi.dpm_solve_batched(beps[i], [fd[r] for r in range(nreq)], [u[r] for r in range(nreq)], stream=s)
            s.synchronize()
            outs[i] = u.cpu()
        except Exception as e:  # reported below
            errors.append(f"thread {i}: {e}")

    th = [threading.Thread(target=work, args=(i,)) for i in range(len(Ks))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for b in beps:
        abi.dpm_bep_destroy(b)
    assert not errors, errors
    for i in range(len(Ks)):
        assert torch.equal(outs[i], ref[i]), i
