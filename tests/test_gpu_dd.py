"""GPU parity of the domain decomposition (Section 3, Case 1: ball + shell on
separate grids, coupled through the shared interface series) against the
oracle: the shell's point sets (bit-exact), the stacked BEP matrix, the
coupled elliptic solve and the coupled time loop."""
import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import (TEST_A_C0, TEST_A_RHO0, manufactured_grad,
                                              manufactured_u)

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def boxes(N1, N2, r1, r2):
    h1, h2 = 2 * r1 / (N1 - 3), 2 * r2 / (N2 - 3)
    return (-r1 - 2 * h1, r1 + 2 * h1), (-r2 - 2 * h2, r2 + 2 * h2)


def test_shell_classification_bit_exact(ctx):
    g = abi.dpm_geom()
    g.kind = 2
    g.axes[0], g.axes[1] = 1.0, 0.45
    N, lo, hi = 40, -1.2, 1.2
    lab = torch.empty(N ** 3, dtype=torch.uint8, device="cuda")
    gin = torch.empty(N ** 3, dtype=torch.int32, device="cuda")
    gex = torch.empty(N ** 3, dtype=torch.int32, device="cuda")
    ngin, ngex = abi.dpm_classify(ctx, g, N, lo, hi, lab, gin, gex)
    torch.cuda.synchronize()
    sets = O.point_sets(O.inside_mask(O.Shell(1.0, 0.45), N, lo, hi))
    ref = O.labels_from_sets(sets).reshape(-1)
    assert np.array_equal(lab.cpu().numpy() & 7, ref & 7)
    assert np.array_equal(gin.cpu().numpy()[:ngin], np.flatnonzero(sets["gin"].reshape(-1)))
    assert np.array_equal(gex.cpu().numpy()[:ngex], np.flatnonzero(sets["gex"].reshape(-1)))


@pytest.mark.parametrize("prec,tol_a,tol_u", [(abi.DPM_PREC_FP64, 1e-11, 1e-11),
                                              (abi.DPM_PREC_FP32, 1e-5, 1e-5)])
def test_dd_bep_and_elliptic_solve_match_oracle(ctx, prec, tol_a, tol_u):
    r1, r2, N1, N2, K, sigma = 0.5, 1.0, 24, 28, 4, 1001.0
    (lo1, hi1), (lo2, hi2) = boxes(N1, N2, r1, r2)
    P = abi.dd_params((0.0, 0.0, 0.0), r1, r2, N1, lo1, hi1, N2, lo2, hi2, K, K, prec)
    dd = abi.dpm_dd_build(ctx, P, sigma)
    info = abi.dpm_dd_get_info(dd)
    S = O.DDSetup((0, 0, 0), r1, r2, N1, lo1, hi1, N2, lo2, hi2, K, K, sigma)
    assert (info.n_gin[0], info.n_gin[1]) == (len(S.sub[0].gin_idx), len(S.sub[1].gin_idx))
    assert (info.n_gamma[0], info.n_gamma[1]) == (len(S.sub[0].gamma_idx), len(S.sub[1].gamma_idx))
    m = info.n_gin[0] + info.n_gin[1]
    A = torch.empty(m * info.ncol, dtype=torch.float64, device="cuda")
    abi.dpm_dd_matrix(dd, A)
    torch.cuda.synchronize()
    Ag = A.cpu().numpy().reshape(info.ncol, m).T
    err = np.max(np.abs(Ag - S.A), axis=0) / np.max(np.abs(S.A), axis=0)
    print(f"DD BEP prec={prec}: max column rel err {err.max():.3e}")
    assert err.max() < tol_a
    # manufactured solution with Neumann data on Gamma
    dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
    fs, us = [], []
    for sd in S.sub:
        X, Y, Z = O.mesh(sd.N, sd.lo, sd.hi)
        f = (sigma + 1) * manufactured_u(X, Y, Z)
        if prec != abi.DPM_PREC_FP64:
            f = f.astype(np.float32).astype(np.float64)
        fs.append(f)
        us.append(torch.empty(sd.N ** 3, dtype=dt, device="cuda"))
    S2 = S.sub[1]
    gn = np.sum(manufactured_grad(S2.xf[:, 0], S2.xf[:, 1], S2.xf[:, 2]) * S2.normal, axis=1)
    fd = [torch.from_numpy(f.reshape(-1)).to("cuda", dt) for f in fs]
    C = torch.empty(info.ncol, dtype=torch.float64, device="cuda")
    abi.dpm_dd_solve(dd, fd[0], fd[1], us[0], us[1], torch.from_numpy(gn).cuda(), C)
    torch.cuda.synchronize()
    u1o, u2o, Co = O.dd_elliptic_solve(S, fs[0], fs[1], gn)
    for sd, u, uo in zip(S.sub, us, (u1o, u2o)):
        Np = sd.sets["Np"]
        ug = u.cpu().numpy().astype(np.float64).reshape(sd.N, sd.N, sd.N)
        e = rel(ug[Np], uo[Np])
        print(f"DD elliptic prec={prec} N={sd.N}: rel err on N+ {e:.3e}")
        assert e < tol_u
        assert np.all(ug[~Np] == 0.0)
    abi.dpm_dd_destroy(dd)


# FP64 with the fixed dt: the CFL mode's dt comes from FP32-rounded gradient
# maxima on the GPU (a 1e-8 relative difference in dt), so the tight FP64
# comparison runs at dt_max; the FP32 case runs the CFL mode.
@pytest.mark.parametrize("prec,mode,tol", [(abi.DPM_PREC_FP64, 0, 1e-11), (abi.DPM_PREC_FP32, 1, 1e-5)])
def test_dd_pks_steps_match_oracle(ctx, prec, mode, tol):
    r1, r2, N1, N2 = 0.25, 0.5, 24, 20
    (lo1, hi1), (lo2, hi2) = boxes(N1, N2, r1, r2)
    h = min(2 * r1 / (N1 - 3), 2 * r2 / (N2 - 3))
    dtm = 0.5 * h * h if mode == 1 else 1e-6
    P = abi.dd_params((0.0, 0.0, 0.0), r1, r2, N1, lo1, hi1, N2, lo2, hi2, 0, 0, prec)
    pk = abi.dpm_dd_pks_create(ctx, P, 1.0, dtm, mode, 0, 1, TEST_A_RHO0, TEST_A_C0)
    st = O.DDPKSState((0, 0, 0), r1, r2, N1, lo1, hi1, N2, lo2, hi2, 0, 0, 1.0, dtm,
                      TEST_A_RHO0, TEST_A_C0, dt_mode="cfl" if mode == 1 else "fixed")
    for _ in range(3):
        g = abi.dpm_dd_pks_step(pk, 1, True)
        dto = st.step()
        d = st.diagnostics()
        assert abs(g.dt - dto) <= 1e-6 * dto
        for key in ("mass", "max_rho", "m2", "free_energy"):
            assert abs(getattr(g, key) - d[key]) <= tol * abs(d[key]), (key, getattr(g, key), d[key])
    dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
    for l, sd in enumerate(st.sub):
        rho = torch.empty(sd.N ** 3, dtype=dt, device="cuda")
        c = torch.empty_like(rho)
        abi.dpm_dd_pks_get_state(pk, l, rho, c)
        torch.cuda.synchronize()
        Np = sd.sets["Np"]
        r_g = rho.cpu().numpy().astype(np.float64).reshape(sd.N, sd.N, sd.N)
        assert rel(r_g[Np], st.rho[l][Np]) < tol, rel(r_g[Np], st.rho[l][Np])
    abi.dpm_dd_pks_destroy(pk)


@pytest.mark.parametrize("prec", [abi.DPM_PREC_FP64, abi.DPM_PREC_FP32])
def test_grouped_launch_matches_separate_launches(ctx, prec):
    """With both sub-domains on the SIMT solver (grids of different N), their
    solves run as one grouped set of launches; the results are bit-identical to
    one batched solve per sub-domain (DPM_DD_GROUP=0)."""
    import os
    N1, N2 = 24, 20
    r1, r2 = 0.25, 0.5
    h1, h2 = 2 * r1 / (N1 - 3), 2 * r2 / (N2 - 3)
    P = abi.dd_params((0.0, 0.0, 0.0), r1, r2, N1, -r1 - 2 * h1, r1 + 2 * h1, N2, -r2 - 2 * h2, r2 + 2 * h2,
                      1, 1, prec)
    dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
    states = []
    for group in ("1", "0"):
        os.environ["DPM_DD_GROUP"] = group
        try:
            pk = abi.dpm_dd_pks_create(ctx, P, 1.0, 0.5 * h1 * h1, 1, 0, 1, TEST_A_RHO0, TEST_A_C0)
            abi.dpm_dd_pks_step(pk, 3, False)
            out = []
            for l, Nl in enumerate((N1, N2)):
                rho = torch.empty(Nl ** 3, dtype=dt, device="cuda")
                c = torch.empty_like(rho)
                abi.dpm_dd_pks_get_state(pk, l, rho, c)
                out += [rho, c]
            torch.cuda.synchronize()
            abi.dpm_dd_pks_destroy(pk)
            states.append([t.cpu().numpy() for t in out])
        finally:
            del os.environ["DPM_DD_GROUP"]
    for a, b in zip(*states):
        assert np.array_equal(a, b)


def test_grouped_launch_at_larger_grids(ctx):
    """Grouped SIMT launches whose tiles need more than the default 48 KB of
    shared memory (FP64, N1 = 96): bit-identical to separate launches."""
    import os
    N1, N2 = 96, 40
    r1, r2 = 0.25, 0.5
    h1, h2 = 2 * r1 / (N1 - 3), 2 * r2 / (N2 - 3)
    P = abi.dd_params((0.0, 0.0, 0.0), r1, r2, N1, -r1 - 2 * h1, r1 + 2 * h1, N2, -r2 - 2 * h2, r2 + 2 * h2,
                      0, 0, abi.DPM_PREC_FP64)
    states = []
    for group in ("1", "0"):
        os.environ["DPM_DD_GROUP"] = group
        try:
            pk = abi.dpm_dd_pks_create(ctx, P, 1.0, 0.5 * h1 * h1, 1, 0, 1, TEST_A_RHO0, TEST_A_C0)
            abi.dpm_dd_pks_step(pk, 2, False)
            rho = torch.empty(N1 ** 3, dtype=torch.float64, device="cuda")
            abi.dpm_dd_pks_get_state(pk, 0, rho, None)
            torch.cuda.synchronize()
            abi.dpm_dd_pks_destroy(pk)
            states.append(rho.cpu().numpy())
        finally:
            del os.environ["DPM_DD_GROUP"]
    assert np.array_equal(states[0], states[1])


def _dd_run(ctx, P, Ns, dtm, mode, rebuild, graph, steps, prec):
    pk = abi.dpm_dd_pks_create(ctx, P, 1.0, dtm, mode, rebuild, 1, TEST_A_RHO0, TEST_A_C0)
    try:
        if graph:
            abi.dpm_dd_pks_set_graph(pk, True)
        flags = [abi.dpm_dd_pks_step(pk, 1, True).rebuilt for _ in range(steps)]
        st = abi.dpm_dd_pks_step(pk, 0, True)
        dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
        out = []
        for l, Nl in enumerate(Ns):
            rho = torch.empty(Nl ** 3, dtype=dt, device="cuda")
            c = torch.empty_like(rho)
            abi.dpm_dd_pks_get_state(pk, l, rho, c)
            out += [rho, c]
        torch.cuda.synchronize()
        if graph:
            abi.dpm_dd_pks_set_graph(pk, False)
            assert abi.dpm_dd_pks_step(pk, 1, True).step == steps + 1  # back on host stepping
        return flags, st, [t.cpu().numpy() for t in out]
    finally:
        abi.dpm_dd_pks_destroy(pk)


@pytest.mark.parametrize("prec,N1,N2,mode,rebuild", [
    (abi.DPM_PREC_FP64, 24, 20, 0, 0), (abi.DPM_PREC_FP64, 24, 20, 1, 0),
    (abi.DPM_PREC_FP32, 24, 20, 1, 1), (abi.DPM_PREC_FP32, 24, 20, 1, 0),
    (abi.DPM_PREC_TC32, 128, 128, 1, 0)])
def test_graph_steps_match_host_steps(ctx, prec, N1, N2, mode, rebuild):
    """Case 1's device-resident steps replayed as a CUDA graph (dt on the device,
    both grids' solves prepared once: one SIMT group, or the tensor-core solver
    per grid at N = 128) equal the host-driven steps bit for bit: rebuild flags
    (Step 4b by a conditional graph node in CFL mode), dt, statistics, state.
    With a fixed dt the graph path builds the BEP when graph stepping starts, so
    its first step reports no rebuild where the host path's first step builds."""
    r1, r2 = 0.25, 0.5
    (lo1, hi1), (lo2, hi2) = boxes(N1, N2, r1, r2)
    h = min(2 * r1 / (N1 - 3), 2 * r2 / (N2 - 3))
    P = abi.dd_params((0.0, 0.0, 0.0), r1, r2, N1, lo1, hi1, N2, lo2, hi2, 1, 1, prec)
    dtm = 0.5 * h * h if mode == 1 else 1e-6
    a = _dd_run(ctx, P, (N1, N2), dtm, mode, rebuild, False, 4, prec)
    b = _dd_run(ctx, P, (N1, N2), dtm, mode, rebuild, True, 4, prec)
    first = 1 if mode == 0 and not rebuild else 0
    assert a[0][first:] == b[0][first:], (a[0], b[0])
    for key in ("t", "dt", "step", "mass", "max_rho", "min_rho", "m2", "free_energy"):
        assert getattr(a[1], key) == getattr(b[1], key), key
    for x, y in zip(a[2], b[2]):
        assert np.array_equal(x, y)
