"""GPU parity of node classification (Definition 2.1): bit-exact labels and
gamma_in / gamma_ex index lists against the oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import Geometry

pytestmark = pytest.mark.gpu

CASES = [
    (Geometry.sphere(1.0), 32, -1.25, 1.25),
    (Geometry.sphere(1.0), 33, -1.25, 1.25),                   # odd N, ragged tiles
    (Geometry.sphere(0.8, (0.05, -0.1, 0.02)), 47, -1.1, 1.1),
    (Geometry.ellipsoid(1.0, 0.8, 0.6), 64, -1.2, 1.2),
    (Geometry.sphere(1.0), 128, -1.25, 1.25),                  # the N=128 PKS workload grid
    (Geometry.ellipsoid(1.0, 0.8, 0.6), 256, -1.2, 1.2),       # the N=256 BEP workload grid
]


def gpu_classify(ctx, geom, N, lo, hi):
    n3 = N ** 3
    lab = torch.empty(n3, dtype=torch.uint8, device="cuda")
    ngin, ngex = abi.dpm_classify(ctx, geom, N, lo, hi, labels=lab)
    gin = torch.empty(ngin, dtype=torch.int32, device="cuda")
    gex = torch.empty(ngex, dtype=torch.int32, device="cuda")
    abi.dpm_classify(ctx, geom, N, lo, hi, labels=lab, gin_idx=gin, gex_idx=gex)
    torch.cuda.synchronize()
    return lab.cpu().numpy().reshape(N, N, N), gin.cpu().numpy(), gex.cpu().numpy()


@pytest.mark.parametrize("geom,N,lo,hi", CASES)
def test_labels_and_lists_bit_exact(ctx, geom, N, lo, hi):
    lab, gin, gex = gpu_classify(ctx, geom, N, lo, hi)
    olab, ogin, ogex = O.classify(geom, N, lo, hi)
    assert np.array_equal(lab & 7, olab)
    assert np.array_equal(gin, ogin)
    assert np.array_equal(gex, ogex)


def test_shell_bit_is_support_of_potential_rhs(ctx):
    geom, N, lo, hi = Geometry.ellipsoid(1.0, 0.8, 0.6), 40, -1.3, 1.3
    lab, _, _ = gpu_classify(ctx, geom, N, lo, hi)
    sets = O.point_sets(O.inside_mask(geom, N, lo, hi))
    # L[v_gamma] on M^- for v = 1 on gamma: nonzero exactly on the shell (generic sigma)
    v = np.where(sets["gamma"], 1.0, 0.0)
    q = np.where(sets["Mm"], O.apply_L(v, 0.1, 3.14159), 0.0)
    assert np.array_equal((lab & 8) > 0, q != 0.0)


def test_rejects_domain_touching_faces(ctx):
    with pytest.raises(abi.DPMError) as e:
        gpu_classify(ctx, Geometry.sphere(1.0), 16, -1.05, 1.05)
    assert e.value.code == abi.DPM_EINVAL
    with pytest.raises(abi.DPMError):
        gpu_classify(ctx, Geometry.sphere(0.01), 16, -1.0, 1.0)   # no node inside


def test_capacity_too_small_is_an_error(ctx):
    geom, N, lo, hi = Geometry.sphere(1.0), 32, -1.25, 1.25
    small = torch.empty(5, dtype=torch.int32, device="cuda")
    with pytest.raises(abi.DPMError):
        abi.dpm_classify(ctx, geom, N, lo, hi, gin_idx=small)
