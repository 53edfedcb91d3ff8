"""GPU parity of the N = 256 tensor-core AP solver (six per-axis tcgen05 passes,
3-term FP16 split) against the oracle: the batched solve directly, and the
BEP matrix and elliptic solve built on it.  Tolerance 1e-5 relative L-inf,
as for every FP32 result."""
import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import Geometry, random_rhs

pytestmark = pytest.mark.gpu
TC = abi.DPM_PREC_TC32
N = 256


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("B,h,sigma", [(2, 2.4 / 257, 1e4 + 1.0), (1, 0.004, 0.0)])
def test_tc256_aux_solve_matches_oracle(ctx, B, h, sigma):
    q = random_rhs(700 + B, B, N, np.float32)
    qd = torch.from_numpy(q).cuda()
    ud = torch.empty_like(qd)
    abi.dpm_aux_solve_batched(ctx, N, h, sigma, B, qd, ud, TC)
    torch.cuda.synchronize()
    u = ud.cpu().numpy().astype(np.float64)
    for b in range(B):
        e = rel(u[b], O.aux_solve(q[b].astype(np.float64), h, sigma))
        print(f"TC aux N=256 b={b} sigma={sigma}: rel err {e:.3e}")
        assert e < 1e-5


def test_tc256_single_mode_input(ctx):
    h, sigma = 2.4 / 257, 0.0
    idx = np.arange(1, N + 1)
    q = (np.sin(np.pi * 3 * idx / (N + 1))[:, None, None] * np.sin(np.pi * 200 * idx / (N + 1))[None, :, None]
         * np.sin(np.pi * 77 * idx / (N + 1))[None, None, :])[None].astype(np.float32)
    qd = torch.from_numpy(q).cuda()
    ud = torch.empty_like(qd)
    abi.dpm_aux_solve_batched(ctx, N, h, sigma, 1, qd, ud, TC)
    torch.cuda.synchronize()
    assert rel(ud.cpu().numpy()[0].astype(np.float64), O.aux_solve(q[0].astype(np.float64), h, sigma)) < 1e-5


def test_tc256_bep_matrix_and_elliptic_solve(ctx):
    geom, K, sigma = Geometry.ellipsoid(1.0, 0.8, 0.6), 1, 1e4 + 1.0
    lo, hi = -1.2, 1.2
    bep = abi.dpm_bep_build(ctx, geom, N, lo, hi, sigma, K, 1, TC)
    info = abi.dpm_bep_get_info(bep)
    A = torch.empty(info.n_gin * info.ncol, dtype=torch.float64, device="cuda")
    abi.dpm_bep_matrix(bep, A)
    s = O.DPMSetup(geom, N, lo, hi, K, 1, sigma)
    Ag = A.cpu().numpy().reshape(info.ncol, info.n_gin).T
    err = np.max(np.abs(Ag - s.A), axis=0) / np.max(np.abs(s.A), axis=0)
    print(f"TC N=256 BEP max column rel err {err.max():.3e}")
    assert err.max() < 1e-5, err.max()
    X, Y, Z = O.mesh(N, lo, hi)
    f = (np.exp(-4 * (X ** 2 + Y ** 2 + Z ** 2)) * (1 + X * Y)).astype(np.float32)
    fd = torch.from_numpy(f).cuda()
    u = torch.empty_like(fd)
    abi.dpm_solve(bep, fd, u)
    torch.cuda.synchronize()
    uo, _, _ = O.dpm_elliptic_solve(s, f.astype(np.float64))
    Np = s.sets["Np"]
    e = rel(u.cpu().numpy().astype(np.float64)[Np], uo[Np])
    print(f"TC N=256 elliptic rel err {e:.3e}")
    assert e < 1e-5, e
    abi.dpm_bep_destroy(bep)
