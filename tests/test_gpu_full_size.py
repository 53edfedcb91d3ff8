"""Parity at the full sizes of the benchmark workloads, in the launch
configuration the bench runs (tensor-core solver, every BEP column in one
batch), on sampled outputs the oracle computes one by one: BEP columns of the
N = 128, K = 8 sphere (162 columns; sigma = 4/h^2, the time step h^2/4) and of
the N = 256, K = 12 ellipsoid (338 columns; sigma = 1e4 + 1).  Each sampled
column is Tr_gamma_in (I - P) psi_k, one oracle AP at full size."""
import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import WORKLOADS

pytestmark = pytest.mark.gpu


def sampled_columns(ctx, w, sigma, cols):
    bep = abi.dpm_bep_build(ctx, w.geom, w.N, w.lo, w.hi, sigma, w.K, w.beta, abi.DPM_PREC_TC32)
    try:
        info = abi.dpm_bep_get_info(bep)
        A = torch.empty(info.n_gin * info.ncol, dtype=torch.float64, device="cuda")
        abi.dpm_bep_matrix(bep, A)
        torch.cuda.synchronize()
        Ag = A.cpu().numpy().reshape(info.ncol, info.n_gin).T
    finally:
        abi.dpm_bep_destroy(bep)
    s = O.DPMSetup(w.geom, w.N, w.lo, w.hi, w.K, w.beta, sigma, build_bep=False)
    assert Ag.shape == (len(s.gin_idx), s.ncol)
    Psi = s.basis_densities()
    errs = []
    for k in cols:
        ref = s.i_minus_p_gin(Psi[:, k])
        errs.append(float(np.max(np.abs(Ag[:, k] - ref)) / np.max(np.abs(ref))))
    return errs


def test_bep_columns_at_the_pks_step_size(ctx):
    w = WORKLOADS["pks_sphere_N128_K8"]
    h = (w.hi - w.lo) / (w.N + 1)
    errs = sampled_columns(ctx, w, 1.0 / (h * h / 4.0), [0, 17, 80, 81, 161])
    assert max(errs) < 1e-5, errs


def test_bep_columns_at_the_n256_batch_size(ctx):
    w = WORKLOADS["bep_ellipsoid_N256_K12"]
    errs = sampled_columns(ctx, w, w.sigma, [0, 168, 337])
    assert max(errs) < 1e-5, errs
