"""GPU parity of the tensor-core (tcgen05, 3-term FP16 split) AP solver at
N = 128 against the oracle, directly and inside the BEP assembly, the
elliptic solve and a PKS step.  Tolerance 1e-5 relative L-inf, as for
every FP32 result."""
import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import (OFFC_C0, OFFC_RHO0, Geometry, manufactured_grad,
                                              manufactured_u, random_rhs)

pytestmark = pytest.mark.gpu
TC = abi.DPM_PREC_TC32
N = 128
LO, HI = -1.25, 1.25


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("B,h,sigma", [(2, 2.5 / 129, 1e4 + 1.0), (3, 0.01, 0.0), (1, 0.05, 300.0)])
def test_tc_aux_solve_matches_oracle(ctx, B, h, sigma):
    q = random_rhs(900 + B, B, N, np.float32)
    qd = torch.from_numpy(q).cuda()
    ud = torch.empty_like(qd)
    abi.dpm_aux_solve_batched(ctx, N, h, sigma, B, qd, ud, TC)
    torch.cuda.synchronize()
    u = ud.cpu().numpy().astype(np.float64)
    for b in range(B):
        e = rel(u[b], O.aux_solve(q[b].astype(np.float64), h, sigma))
        print(f"TC aux N=128 b={b} sigma={sigma}: rel err {e:.3e}")
        assert e < 1e-5


def test_tc_smooth_and_single_mode_inputs(ctx):
    """Low-mode input (large dynamic range after the division by lambda)."""
    h, sigma = 2.5 / 129, 0.0
    idx = np.arange(1, N + 1)
    q = np.zeros((2, N, N, N))
    q[0] = (np.sin(np.pi * idx / (N + 1))[:, None, None] * np.sin(np.pi * 2 * idx / (N + 1))[None, :, None]
            * np.sin(np.pi * 3 * idx / (N + 1))[None, None, :])
    q[1] = q[0] + 1e-3 * random_rhs(5, 1, N, np.float64)[0]
    q = q.astype(np.float32)
    qd = torch.from_numpy(q).cuda()
    ud = torch.empty_like(qd)
    abi.dpm_aux_solve_batched(ctx, N, h, sigma, 2, qd, ud, TC)
    torch.cuda.synchronize()
    u = ud.cpu().numpy().astype(np.float64)
    for b in range(2):
        assert rel(u[b], O.aux_solve(q[b].astype(np.float64), h, sigma)) < 1e-5


def test_tc_rejects_other_sizes(ctx):  # N = 64 has no tensor-core solver
    q = torch.zeros(1, 64, 64, 64, device="cuda")
    with pytest.raises(abi.DPMError) as e:
        abi.dpm_aux_solve_batched(ctx, 64, 0.1, 1.0, 1, q, q, TC)
    assert e.value.code == abi.DPM_EUNSUPPORTED


def test_tc_bep_matrix_and_elliptic_solve(ctx):
    geom, K, sigma = Geometry.sphere(1.0), 2, 1001.0
    bep = abi.dpm_bep_build(ctx, geom, N, LO, HI, sigma, K, 1, TC)
    info = abi.dpm_bep_get_info(bep)
    A = torch.empty(info.n_gin * info.ncol, dtype=torch.float64, device="cuda")
    abi.dpm_bep_matrix(bep, A)
    s = O.DPMSetup(geom, N, LO, HI, K, 1, sigma)
    Ag = A.cpu().numpy().reshape(info.ncol, info.n_gin).T
    err = np.max(np.abs(Ag - s.A), axis=0) / np.max(np.abs(s.A), axis=0)
    print(f"TC BEP N=128 K=2: max column rel err {err.max():.3e}")
    assert err.max() < 1e-5, err.max()
    X, Y, Z = O.mesh(N, LO, HI)
    f = ((sigma + 1.0) * manufactured_u(X, Y, Z)).astype(np.float32).astype(np.float64)
    gn = np.sum(manufactured_grad(s.xf[:, 0], s.xf[:, 1], s.xf[:, 2]) * s.normal, axis=1)
    fd = torch.from_numpy(f).float().cuda()
    u = torch.empty_like(fd)
    abi.dpm_solve(bep, fd, u, neumann=torch.from_numpy(gn).cuda())
    torch.cuda.synchronize()
    uo, _, _ = O.dpm_elliptic_solve(s, f, gn)
    Np = s.sets["Np"]
    e = rel(u.cpu().numpy().astype(np.float64)[Np], uo[Np])
    print(f"TC elliptic N=128 K=2: rel err {e:.3e}")
    assert e < 1e-5, e
    abi.dpm_bep_destroy(bep)


def test_tc_pks_step_matches_oracle(ctx):
    geom, K = Geometry.sphere(1.0), 2
    h = (HI - LO) / (N + 1)
    dt = 2e-7
    p = abi.pks_params(geom, N, LO, HI, 1.0, dt, K, 1, TC, dt_mode=0, rebuild=0, clamp=1)
    pks = abi.dpm_pks_create(ctx, p, OFFC_RHO0, OFFC_C0)
    r = torch.empty(N, N, N, device="cuda")
    c = torch.empty_like(r)
    abi.dpm_pks_get_state(pks, r, c)
    torch.cuda.synchronize()
    o = O.PKSState(geom, N, LO, HI, K, 1, 1.0, dt, rho=r.cpu().double().numpy(), c=c.cpu().double().numpy())
    abi.dpm_pks_step(pks, 1)
    o.step()
    abi.dpm_pks_get_state(pks, r, c)
    torch.cuda.synchronize()
    Np = o.sets["Np"]
    er = rel(r.cpu().double().numpy()[Np], o.rho[Np])
    ec = rel(c.cpu().double().numpy()[Np], o.c[Np])
    print(f"TC PKS N=128 K=2: rel err rho {er:.3e} c {ec:.3e} (h={h:.4f})")
    assert er < 1e-5 and ec < 1e-5, (er, ec)
    abi.dpm_pks_destroy(pks)


def _unseen_spectra(n):
    """Positive right-hand sides of two spectra that differ from the dense random
    and Gaussian data the solvers' rounding compensation was measured on: a
    linear ramp (energy in the lowest modes, decaying as 1/a) and a handful of
    point sources (a flat spectrum)."""
    X, Y, Z = O.mesh(n, -1.0, 1.0)
    ramp = (X + Y + Z + 3.5).astype(np.float32)
    spikes = np.zeros((n, n, n), np.float32)
    rng = np.random.default_rng(n + 7)
    for _ in range(12):
        i, j, k = rng.integers(n // 8, n - n // 8, 3)
        spikes[i, j, k] = rng.uniform(1.0, 3.0)
    return {"ramp": ramp, "spikes": spikes}


@pytest.mark.parametrize("n,prec", [(128, TC), (256, TC), (256, abi.DPM_PREC_FFT32)])
@pytest.mark.parametrize("kind", ["ramp", "spikes"])
def test_solve_mean_error_against_oracle(ctx, n, prec, kind):
    """The mean relative error of a solve against the oracle, |sum(u - u_ref)| /
    sum(u_ref), on positive data of two spectra the tensor-core solvers' rounding
    compensation never saw (a bias of 2e-6 per solve drifts a 10,000-step time
    loop by 2 %).  The tensor cores round their FP32 accumulator toward zero; the
    tensor-core solvers issue the small cross terms first and scale the
    spectrum by the expected loss of that rounding, derived from the number of
    accumulation steps per transform (half an ulp per step, six transforms), not
    fitted to data.  The FFT-style solver rounds to nearest.  Bound: 1e-6, the per-transform FP32
    error of the dominant mode times the six transforms of a solve."""
    h, sigma = 1.0 / (n - 3), 1.25e5
    q = _unseen_spectra(n)[kind]
    qd = torch.from_numpy(q[None]).cuda()
    ud = torch.empty_like(qd)
    abi.dpm_aux_solve_batched(ctx, n, h, sigma, 1, qd, ud, prec)
    torch.cuda.synchronize()
    u = ud.cpu().numpy()[0].astype(np.float64)
    ref = O.aux_solve(q.astype(np.float64), h, sigma)
    bias = float(np.sum(u - ref) / np.sum(ref))
    worst = rel(u, ref)
    print(f"mean error N={n} prec={prec} {kind}: bias {bias:.2e}, max {worst:.2e}")
    assert abs(bias) < 1e-6 and worst < 1e-5, (bias, worst)
