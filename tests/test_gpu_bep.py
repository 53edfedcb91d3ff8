"""GPU parity of Steps 1-2 and the elliptic DPM solve against the oracle:
gamma geometry (Definition 2.6), the BEP matrix (eq. BEP_recast), and
dpm_solve (particular solution, least squares, extension, Green's formula)."""
import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import (WORKLOADS, Geometry, manufactured_grad,
                                              manufactured_u)

pytestmark = pytest.mark.gpu

W1 = WORKLOADS["elliptic_sphere_N32_K4"]


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


class GpuBep:
    def __init__(self, ctx, geom, N, lo, hi, sigma, K, beta, prec):
        self.ctx, self.prec = ctx, prec
        self.h = abi.dpm_bep_build(ctx, geom, N, lo, hi, sigma, K, beta, prec)
        self.info = abi.dpm_bep_get_info(self.h)
        self.dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32

    def matrix(self):
        i = self.info
        A = torch.empty(i.n_gin * i.ncol, dtype=torch.float64, device="cuda")
        abi.dpm_bep_matrix(self.h, A)
        torch.cuda.synchronize()
        return A.cpu().numpy().reshape(i.ncol, i.n_gin).T

    def geometry(self):
        n = self.info.n_gamma
        gi = torch.empty(n, dtype=torch.int32, device="cuda")
        ft = torch.empty(n, 3, dtype=torch.float64, device="cuda")
        nr = torch.empty(n, 3, dtype=torch.float64, device="cuda")
        d = torch.empty(n, dtype=torch.float64, device="cuda")
        abi.dpm_bep_gamma_geometry(self.h, gi, ft, nr, d)
        torch.cuda.synchronize()
        return gi.cpu().numpy(), ft.cpu().numpy(), nr.cpu().numpy(), d.cpu().numpy()

    def solve(self, f, neumann=None):
        N = self.info.N
        fd = torch.from_numpy(np.ascontiguousarray(f)).to("cuda", self.dt)
        u = torch.empty_like(fd)
        C = torch.empty(self.info.ncol, dtype=torch.float64, device="cuda")
        nd = None if neumann is None else torch.from_numpy(neumann).to("cuda", torch.float64)
        abi.dpm_solve(self.h, fd, u, neumann=nd, coeffs=C)
        torch.cuda.synchronize()
        return u.cpu().numpy().astype(np.float64).reshape(N, N, N), C.cpu().numpy()

    def close(self):
        abi.dpm_bep_destroy(self.h)


@pytest.mark.parametrize("geom,N,lo,hi", [(Geometry.sphere(1.0), 32, -1.25, 1.25),
                                          (Geometry.ellipsoid(1.0, 0.8, 0.6), 40, -1.2, 1.2)])
def test_gamma_geometry_matches_oracle(ctx, geom, N, lo, hi):
    b = GpuBep(ctx, geom, N, lo, hi, 100.0, 2, 1, abi.DPM_PREC_FP64)
    gi, ft, nr, d = b.geometry()
    s = O.DPMSetup(geom, N, lo, hi, 2, 1, 100.0, build_bep=False)
    assert np.array_equal(gi, s.gamma_idx)
    assert np.max(np.abs(ft - s.xf)) < 1e-12
    assert np.max(np.abs(nr - s.normal)) < 1e-11
    assert np.max(np.abs(d - s.d)) < 1e-12
    info = b.info
    assert (info.n_gin, info.n_gex, info.n_gamma) == (len(s.gin_idx), len(s.gex_idx), len(s.gamma_idx))
    b.close()


@pytest.mark.parametrize("prec,tol", [(abi.DPM_PREC_FP64, 1e-11), (abi.DPM_PREC_FP32, 1e-5)])
@pytest.mark.parametrize("geom,N,lo,hi,K", [(Geometry.sphere(1.0), 32, -1.25, 1.25, 4),
                                            (Geometry.ellipsoid(1.0, 0.8, 0.6), 36, -1.2, 1.2, 3)])
def test_bep_matrix_matches_oracle(ctx, prec, tol, geom, N, lo, hi, K):
    sigma = 1001.0
    b = GpuBep(ctx, geom, N, lo, hi, sigma, K, 1, prec)
    A = b.matrix()
    s = O.DPMSetup(geom, N, lo, hi, K, 1, sigma)
    err = np.max(np.abs(A - s.A), axis=0) / np.max(np.abs(s.A), axis=0)
    print(f"BEP prec={prec} max column rel err {err.max():.3e}")
    assert err.max() < tol
    b.close()


def manufactured_case(setup_like, geom, N, lo, hi, sigma, xf, normal):
    x = O.node_coords(N, lo, hi)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    f = (sigma + 1.0) * manufactured_u(X, Y, Z)
    gn = np.sum(manufactured_grad(xf[:, 0], xf[:, 1], xf[:, 2]) * normal, axis=1)
    return f, gn


@pytest.mark.parametrize("prec,tol", [(abi.DPM_PREC_FP64, 1e-11), (abi.DPM_PREC_FP32, 1e-5)])
def test_elliptic_solve_matches_oracle(ctx, prec, tol):
    """The N=32, K=4 sphere workload: (1/dt+1) u - Lap u = f, Neumann data of
    u = exp(x) sin(y) cos(z)."""
    w = W1
    b = GpuBep(ctx, w.geom, w.N, w.lo, w.hi, w.sigma, w.K, w.beta, prec)
    s = O.DPMSetup(w.geom, w.N, w.lo, w.hi, w.K, w.beta, w.sigma)
    f, gn = manufactured_case(s, w.geom, w.N, w.lo, w.hi, w.sigma, s.xf, s.normal)
    if prec == abi.DPM_PREC_FP32:
        f = f.astype(np.float32).astype(np.float64)
    u, C = b.solve(f, gn)
    uo, Co, ugo = O.dpm_elliptic_solve(s, f, gn)
    Np = s.sets["Np"]
    e = rel(u[Np], uo[Np])
    print(f"elliptic prec={prec} rel err on N+ {e:.3e}")
    assert e < tol
    assert np.all(u[~Np] == 0.0)
    # and both are close to the exact solution (spectral + O(h^2) error)
    X, Y, Z = O.mesh(w.N, w.lo, w.hi)
    assert np.max(np.abs(np.where(s.sets["Mp"], u - manufactured_u(X, Y, Z), 0))) < 1e-2
    b.close()


@pytest.mark.parametrize("prec,tol", [(abi.DPM_PREC_FP64, 1e-11), (abi.DPM_PREC_FP32, 1e-5)])
@pytest.mark.parametrize("K", [9, 12])
def test_elliptic_solve_many_harmonics(ctx, prec, tol, K):
    """K = 9 and 12 (200 and 338 columns, past the in-shared-memory Cholesky):
    the serving mix's upper range of harmonic degrees on an N=32 ellipsoid."""
    geom, N, lo, hi, sigma = Geometry.ellipsoid(0.9, 0.75, 0.6), 32, -1.125, 1.125, 3.0e3
    b = GpuBep(ctx, geom, N, lo, hi, sigma, K, 1, prec)
    s = O.DPMSetup(geom, N, lo, hi, K, 1, sigma)
    f, gn = manufactured_case(s, geom, N, lo, hi, sigma, s.xf, s.normal)
    if prec == abi.DPM_PREC_FP32:
        f = f.astype(np.float32).astype(np.float64)
    u, C = b.solve(f, gn)
    uo, Co, _ = O.dpm_elliptic_solve(s, f, gn)
    Np = s.sets["Np"]
    e = rel(u[Np], uo[Np])
    print(f"elliptic K={K} prec={prec} rel err on N+ {e:.3e}")
    assert e < tol
    b.close()


@pytest.mark.parametrize("K,beta", [(0, 0), (2, 1), (6, 0), (7, 1), (8, 1), (12, 0)])
def test_elliptic_solve_factor_sizes(ctx, K, beta):
    """The FP32 path's least squares at n = 1, 18, 49, 128, 162 columns (the
    one-CTA FP32 Cholesky: a single partial panel, partial last panels, full
    panels) and n = 169 (just past it: the FP64 Cholesky from global memory),
    on an N=32 ellipsoid against the oracle's Householder solve."""
    geom, N, lo, hi, sigma = Geometry.ellipsoid(0.9, 0.75, 0.6), 32, -1.125, 1.125, 3.0e3
    prec = abi.DPM_PREC_FP32
    b = GpuBep(ctx, geom, N, lo, hi, sigma, K, beta, prec)
    s = O.DPMSetup(geom, N, lo, hi, K, beta, sigma)
    assert s.ncol == (K + 1) ** 2 * (2 if beta else 1)
    f, gn = manufactured_case(s, geom, N, lo, hi, sigma, s.xf, s.normal)
    f = f.astype(np.float32).astype(np.float64)
    u, C = b.solve(f, gn)
    uo, Co, _ = O.dpm_elliptic_solve(s, f, gn)
    Np = s.sets["Np"]
    e = rel(u[Np], uo[Np])
    print(f"elliptic n={s.ncol} rel err on N+ {e:.3e}")
    assert e < 1e-5, e
    b.close()
