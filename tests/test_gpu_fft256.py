"""GPU parity of the FFT-style N = 256 AP solver (even/odd fold + Rader
convolutions by length-128 FFTs, plane / pencil / plane on 2-CTA clusters)
against the oracle: the batched solve on dense random, single-mode and smooth
inputs, in place, the BEP matrix and elliptic solve built on it, and the mean
error of a solve on positive data.  Tolerance 1e-5 relative L-inf, as for every
FP32 result."""
import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import Geometry, random_rhs

pytestmark = pytest.mark.gpu
FFT = abi.DPM_PREC_FFT32
N = 256


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def solve(ctx, q, h, sigma, inplace=False):
    qd = torch.from_numpy(np.ascontiguousarray(q, dtype=np.float32)).cuda()
    ud = qd if inplace else torch.empty_like(qd)
    abi.dpm_aux_solve_batched(ctx, N, h, sigma, q.shape[0], qd, ud, FFT)
    torch.cuda.synchronize()
    return ud.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("B,h,sigma", [(3, 2.4 / 257, 1e4 + 1.0), (1, 0.004, 0.0)])
def test_fft256_aux_solve_matches_oracle(ctx, B, h, sigma):
    q = random_rhs(1700 + B, B, N, np.float32)
    u = solve(ctx, q, h, sigma)
    for b in range(B):
        e = rel(u[b], O.aux_solve(q[b].astype(np.float64), h, sigma))
        print(f"FFT aux N=256 b={b} sigma={sigma}: rel err {e:.3e}")
        assert e < 1e-5, e


def test_fft256_single_mode_and_smooth_inputs(ctx):
    h, sigma = 2.4 / 257, 0.0
    idx = np.arange(1, N + 1)
    q = np.zeros((2, N, N, N))
    q[0] = (np.sin(np.pi * 3 * idx / (N + 1))[:, None, None] * np.sin(np.pi * 200 * idx / (N + 1))[None, :, None]
            * np.sin(np.pi * 77 * idx / (N + 1))[None, None, :])
    X, Y, Z = O.mesh(N, -1.2, 1.2)
    q[1] = np.exp(-6 * ((X - 0.2) ** 2 + Y ** 2 + (Z + 0.1) ** 2))
    q = q.astype(np.float32)
    u = solve(ctx, q, h, sigma)
    for b in range(2):
        e = rel(u[b], O.aux_solve(q[b].astype(np.float64), h, sigma))
        print(f"FFT aux N=256 input {b}: rel err {e:.3e}")
        assert e < 1e-5, e


def test_fft256_in_place(ctx):
    q = random_rhs(1801, 1, N, np.float32)
    h, sigma = 2.4 / 257, 3e3
    u = solve(ctx, q, h, sigma, inplace=True)
    assert rel(u[0], O.aux_solve(q[0].astype(np.float64), h, sigma)) < 1e-5


@pytest.mark.parametrize("kind", ["uniform", "gaussian"])
def test_fft256_has_no_systematic_bias(ctx, kind):
    """The mean relative error of a solve against the oracle, on positive data of
    two spectra (white and a smooth blob).  FP32 arithmetic rounds to nearest,
    but the error of the dominant low mode of smooth data is deterministic
    (~3 ulps per 128-point FFT round trip, the same sign on every line of the
    same shape), so the mean error can reach the per-transform error times the
    six transforms of a solve: |sum(u - u_ref)| / sum(u_ref) < 1e-6.  (A
    truncating accumulation, which loses ~0.5 ulp of the running sum at every
    step, exceeds that within a few dozen steps.)"""
    h, sigma = 1.0 / 253, 1.25e5
    if kind == "uniform":
        q = np.random.default_rng(5).uniform(0.0, 1.0, (1, N, N, N))
    else:
        X, Y, Z = O.mesh(N, -0.51, 0.51)
        q = 1000.0 * np.exp(-100 * (X ** 2 + Y ** 2 + Z ** 2))[None]
    q = q.astype(np.float32)
    u = solve(ctx, q, h, sigma)[0]
    ref = O.aux_solve(q[0].astype(np.float64), h, sigma)
    bias = float(np.sum(u - ref) / np.sum(ref))
    worst = rel(u, ref)
    print(f"FFT N=256 {kind}: mean rel bias {bias:.2e}, max rel err {worst:.2e}")
    assert abs(bias) < 1e-6 and worst < 1e-5, (bias, worst)


def test_fft256_rejects_other_sizes(ctx):
    q = torch.zeros(1, 128, 128, 128, device="cuda")
    with pytest.raises(abi.DPMError) as e:
        abi.dpm_aux_solve_batched(ctx, 128, 0.01, 1.0, 1, q, q, FFT)
    assert e.value.code == abi.DPM_EUNSUPPORTED


def test_fft256_bep_matrix_and_elliptic_solve(ctx):
    geom, K, sigma = Geometry.ellipsoid(1.0, 0.8, 0.6), 1, 1e4 + 1.0
    lo, hi = -1.2, 1.2
    bep = abi.dpm_bep_build(ctx, geom, N, lo, hi, sigma, K, 1, FFT)
    info = abi.dpm_bep_get_info(bep)
    A = torch.empty(info.n_gin * info.ncol, dtype=torch.float64, device="cuda")
    abi.dpm_bep_matrix(bep, A)
    s = O.DPMSetup(geom, N, lo, hi, K, 1, sigma)
    Ag = A.cpu().numpy().reshape(info.ncol, info.n_gin).T
    err = np.max(np.abs(Ag - s.A), axis=0) / np.max(np.abs(s.A), axis=0)
    print(f"FFT N=256 BEP max column rel err {err.max():.3e}")
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
    print(f"FFT N=256 elliptic rel err {e:.3e}")
    assert e < 1e-5, e
    abi.dpm_bep_destroy(bep)
