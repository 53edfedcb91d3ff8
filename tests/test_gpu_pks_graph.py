"""Graph stepping of the PKS loop (device-resident Step 3, the whole step
replayed as a CUDA graph) against the default host-driven stepping: same
kernels and arithmetic, so the same states and statistics."""
import numpy as np
import pytest
import torch

from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import TEST_A_C0, TEST_A_RHO0, Geometry

pytestmark = pytest.mark.gpu


def _run(ctx, N, K, prec, dt_mode, rebuild, graph, steps, stream):
    lo, hi = -1.25, 1.25
    h = (hi - lo) / (N + 1)
    prm = abi.pks_params(Geometry.sphere(1.0), N, lo, hi, 1.0, h * h / 4.0, K, 1, prec,
                         dt_mode=dt_mode, rebuild=rebuild, clamp=1)
    pk = abi.dpm_pks_create(ctx, prm, TEST_A_RHO0, TEST_A_C0, stream=stream)
    if graph:
        abi.dpm_pks_set_graph(pk, True, stream=stream)
    stats = []
    for _ in range(steps):
        st = abi.dpm_pks_step(pk, 1, True, stream=stream)
        stats.append((st.t, st.dt, st.step, st.mass, st.max_rho, st.min_rho, st.free_energy))
    dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
    rho = torch.empty((N, N, N), dtype=dt, device="cuda")
    c = torch.empty_like(rho)
    abi.dpm_pks_get_state(pk, rho, c, stream=stream)
    torch.cuda.synchronize()
    abi.dpm_pks_destroy(pk)
    return np.array(stats), rho.cpu().numpy(), c.cpu().numpy()


@pytest.mark.parametrize("N,K,prec,dt_mode,rebuild", [
    (32, 4, abi.DPM_PREC_FP32, 1, 1),
    (32, 4, abi.DPM_PREC_FP64, 1, 1),
    (32, 4, abi.DPM_PREC_FP32, 0, 0),
    (128, 4, abi.DPM_PREC_TC32, 1, 1),
])
def test_graph_steps_match_default_steps(ctx, N, K, prec, dt_mode, rebuild):
    s = torch.cuda.Stream()
    a = _run(ctx, N, K, prec, dt_mode, rebuild, False, 4, s)
    b = _run(ctx, N, K, prec, dt_mode, rebuild, True, 4, s)
    np.testing.assert_array_equal(a[0][:, 2], b[0][:, 2])           # step counter
    np.testing.assert_allclose(b[0], a[0], rtol=1e-12, atol=0)      # t, dt, diagnostics
    for x, y in ((a[1], b[1]), (a[2], b[2])):
        assert np.max(np.abs(x - y)) <= 1e-6 * np.max(np.abs(x)), "state differs"
    print("bit-identical states:", np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]))


def test_graph_on_default_stream_and_switch_back(ctx):
    # replay on the legacy default stream; switching off hands t/dt back to the host path
    a = _run(ctx, 32, 4, abi.DPM_PREC_FP32, 1, 1, False, 5, None)
    lo, hi, N = -1.25, 1.25, 32
    h = (hi - lo) / (N + 1)
    prm = abi.pks_params(Geometry.sphere(1.0), N, lo, hi, 1.0, h * h / 4.0, 4, 1, abi.DPM_PREC_FP32,
                         dt_mode=1, rebuild=1, clamp=1)
    pk = abi.dpm_pks_create(ctx, prm, TEST_A_RHO0, TEST_A_C0)
    abi.dpm_pks_step(pk, 1, False)
    abi.dpm_pks_set_graph(pk, True)
    abi.dpm_pks_step(pk, 3, False)
    abi.dpm_pks_set_graph(pk, False)
    st = abi.dpm_pks_step(pk, 1, True)
    abi.dpm_pks_destroy(pk)
    assert st.step == 5
    assert abs(st.t - a[0][-1, 0]) <= 1e-12 * a[0][-1, 0]
    assert abs(st.mass - a[0][-1, 3]) <= 1e-6 * abs(a[0][-1, 3])


def _run_rebuilds(ctx, prec, graph):
    """Test (A) data at N = 32 in CFL mode without forced rebuilds: four steps
    (dt stays at the first step's bound), then c doubled through the public
    API (the bound halves: the next step must rebuild), then four more."""
    lo, hi, N = -1.25, 1.25, 32
    prm = abi.pks_params(Geometry.sphere(1.0), N, lo, hi, 1.0, 1.0, 4, 1, prec, dt_mode=1, rebuild=0, clamp=1)
    pk = abi.dpm_pks_create(ctx, prm, TEST_A_RHO0, TEST_A_C0)
    if graph:
        abi.dpm_pks_set_graph(pk, True)
    dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
    rho = torch.empty((N, N, N), dtype=dt, device="cuda")
    c = torch.empty_like(rho)
    rows = []
    for k in range(8):
        if k == 4:
            abi.dpm_pks_get_state(pk, rho, c)
            abi.dpm_pks_set_state(pk, rho, 2.0 * c)
        st = abi.dpm_pks_step(pk, 1, True)
        rows.append((st.rebuilt, st.dt, st.mass, st.max_rho, st.free_energy))
    abi.dpm_pks_get_state(pk, rho, c)
    torch.cuda.synchronize()
    abi.dpm_pks_destroy(pk)
    return np.array(rows), rho.cpu().numpy(), c.cpu().numpy()


@pytest.mark.parametrize("prec", [abi.DPM_PREC_FP32, abi.DPM_PREC_FP64])
def test_graph_step4b_rebuilds_only_when_dt_decreases(ctx, prec):
    """Step 4b inside the graph (dt_mode 1 without rebuild = 1): a conditional
    graph node, switched by a kernel from the step's dt, rebuilds the BEP only
    when dt decreases.  The replayed steps keep dt (no rebuild) until c is
    doubled between steps, which halves the CFL bound (one rebuild), and keep
    the new dt afterwards; the rebuild flags, dt, the statistics and the state
    equal the host-driven loop's."""
    a = _run_rebuilds(ctx, prec, False)
    b = _run_rebuilds(ctx, prec, True)
    flags = a[0][:, 0]
    print("rebuilt per step:", flags.astype(int).tolist(), "dt:", a[0][:, 1].tolist())
    assert flags[0] == 1 and flags[4] == 1 and 0 in flags[2:4] and 0 in flags[5:], flags
    np.testing.assert_array_equal(a[0][:, 0], b[0][:, 0])
    np.testing.assert_allclose(b[0], a[0], rtol=1e-12, atol=0)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]), "state differs"
