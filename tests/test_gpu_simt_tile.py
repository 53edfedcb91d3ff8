"""The SIMT solver's tile width (16, 32 or 64 grid lines per CTA) changes its
run time only: every width gives bit-identical auxiliary solves (ragged N, so
the last tile is partial for each width; at N = 150 the 64-wide tiles have more
4 x 4 tasks than a CTA has threads, two rounds over the staged sine table) and
bit-identical BEP matrices (the
shell density sums and the gamma_in traces read per-tile row ranges), and the
autotuner picks one of the widths whose shared memory fits."""
import os

import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import Geometry, random_rhs

pytestmark = pytest.mark.gpu


class forced_tile:
    def __init__(self, c):
        self.c = c

    def __enter__(self):
        self.old = os.environ.get("DPM_SIMT_TILE")
        os.environ["DPM_SIMT_TILE"] = str(self.c)

    def __exit__(self, *exc):
        if self.old is None:
            del os.environ["DPM_SIMT_TILE"]
        else:
            os.environ["DPM_SIMT_TILE"] = self.old


def solve(ctx, q, h, sigma, prec):
    B, N = q.shape[0], q.shape[1]
    dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
    qd = torch.from_numpy(q).to("cuda", dt).contiguous()
    ud = torch.empty_like(qd)
    abi.dpm_aux_solve_batched(ctx, N, h, sigma, B, qd, ud, prec)
    torch.cuda.synchronize()
    return ud.cpu().numpy()


@pytest.mark.parametrize("prec", [abi.DPM_PREC_FP32, abi.DPM_PREC_FP64])
@pytest.mark.parametrize("N", [37, 70, 150])
def test_every_tile_width_gives_the_same_bits(ctx, prec, N):
    B, h, sigma = 3, 1.0 / (N + 1), 1001.0
    q = random_rhs(1000 + N, B, N, np.float64)
    outs = {}
    for c in (16, 32, 64):
        with forced_tile(c):
            outs[c] = solve(ctx, q, h, sigma, prec)
    assert np.array_equal(outs[16], outs[32]) and np.array_equal(outs[64], outs[32])
    ref = O.aux_solve(q[1].astype(np.float32 if prec == abi.DPM_PREC_FP32 else np.float64)
                      .astype(np.float64), h, sigma)
    tol = 1e-11 if prec == abi.DPM_PREC_FP64 else 1e-5
    assert np.max(np.abs(outs[32][1] - ref)) / np.max(np.abs(ref)) < tol


@pytest.mark.parametrize("prec", [abi.DPM_PREC_FP32, abi.DPM_PREC_FP64])
def test_bep_matrix_is_tile_independent(ctx, prec):
    geom, N, lo, hi, K = Geometry.ellipsoid(0.9, 0.7, 0.6), 41, -1.1, 1.1, 3
    mats = []
    for c in (16, 32, 64):
        with forced_tile(c):
            b = abi.dpm_bep_build(ctx, geom, N, lo, hi, 1001.0, K, 1, prec)
            i = abi.dpm_bep_get_info(b)
            A = torch.empty(i.n_gin * i.ncol, dtype=torch.float64, device="cuda")
            abi.dpm_bep_matrix(b, A)
            torch.cuda.synchronize()
            mats.append(A.cpu().numpy())
            abi.dpm_bep_destroy(b)
    assert np.array_equal(mats[0], mats[1]) and np.array_equal(mats[2], mats[1])


def test_autotuner_records_a_fitting_width(ctx):
    old = os.environ.pop("DPM_SIMT_TILE", None)
    try:
        for prec, N in ((abi.DPM_PREC_FP32, 52), (abi.DPM_PREC_FP64, 256)):
            q = random_rhs(7, 1, N, np.float64)
            solve(ctx, q, 1.0 / (N + 1), 10.0, prec)
            c = abi.dpm_simt_tile(N, prec, 1)
            # FP64 tiles of 64 lines need 2*64*257*8 bytes of shared memory at N = 256
            allowed = (16, 32) if (prec == abi.DPM_PREC_FP64 and N == 256) else (16, 32, 64)
            if os.environ.get("DPM_AUTOTUNE", "1") == "0":
                assert c == 0
            else:
                assert c in allowed
    finally:
        if old is not None:
            os.environ["DPM_SIMT_TILE"] = old
