"""GPU parity of the domain decomposition, Case 2 (Section 3, interface Z
meeting Gamma), through dpm_dd2_*: the lens / outside point sets and the Gamma
/ Z split of each grid boundary bit for bit, the stacked BEP matrix, the
coupled elliptic solve with Neumann data, and the coupled time loop, each
against the oracle on the same grids (Omega = r < 0.5, Z = the sphere of
radius 0.25 about the north pole, the lens box centred on the pole)."""
import types

import numpy as np
import pytest
import torch

from oracle import dpm_oracle as O
from paper_1811_03557_gb300 import abi
from paper_1811_03557_gb300.workloads import Gaussian

pytestmark = pytest.mark.gpu

R, RZ, SIGMA = 0.5, 0.25, 1001.0
TOL = {abi.DPM_PREC_FP64: 1e-11, abi.DPM_PREC_FP32: 1e-5}


def boxes(N1, N2):
    h1, h2 = 2 * RZ / (N1 - 3), 2 * R / (N2 - 3)
    return (-RZ - 2 * h1, RZ + 2 * h1, (0.0, 0.0, R)), (-R - 2 * h2, R + 2 * h2, (0.0, 0.0, 0.0))


def params(N1, N2, MZ, MG, prec, gs=2):
    (lo1, hi1, o1), (lo2, hi2, o2) = boxes(N1, N2)
    return abi.dd2_params((0.0, 0.0, 0.0), R, RZ, R, N1, lo1, hi1, o1, N2, lo2, hi2, o2, MZ, MG, prec,
                          gamma_series=gs)


def oracle_setup(N1, N2, MZ, MG, build=True, gs=2):
    (lo1, hi1, o1), (lo2, hi2, o2) = boxes(N1, N2)
    return O.DD2Setup((0.0, 0.0, 0.0), R, RZ, R, N1, lo1, hi1, o1, N2, lo2, hi2, o2, MZ, MG, SIGMA,
                      build_bep=build, gamma_series=gs)


def u_exact(X, Y, Z):
    return np.exp(Z) * np.cos(X * X + Y * Y)


def lap_exact(X, Y, Z):
    q = X * X + Y * Y
    return np.exp(Z) * ((1 - 4 * q) * np.cos(q) - 4 * np.sin(q))


def grad_exact(X, Y, Z):
    q = X * X + Y * Y
    e = np.exp(Z)
    return np.stack([-2 * X * e * np.sin(q), -2 * Y * e * np.sin(q), e * np.cos(q)], axis=-1)


def global_mesh(sd):
    X, Y, Z = O.mesh(sd.N, sd.lo, sd.hi)
    return X + sd.origin[0], Y + sd.origin[1], Z + sd.origin[2]


@pytest.mark.parametrize("N1,N2", [(20, 20), (33, 26)])
def test_sets_and_split_bit_exact(ctx, N1, N2):
    S = oracle_setup(N1, N2, 3, 4, build=False)
    d = abi.dpm_dd2_build(ctx, params(N1, N2, 3, 4, abi.DPM_PREC_FP64), SIGMA)
    try:
        info = abi.dpm_dd2_get_info(d)
        for l, sd in enumerate(S.sub):
            # the sub-domain's own point sets, classified as dpm_geom kind 3 / 4
            g = types.SimpleNamespace(kind=sd.geom.kind, center=sd.geom.center, axes=sd.geom.axes)
            lab = torch.empty(sd.N ** 3, dtype=torch.uint8, device="cuda")
            abi.dpm_classify(ctx, g, sd.N, sd.lo, sd.hi, labels=lab)
            got = lab.cpu().numpy().reshape((sd.N,) * 3) & 7
            assert np.array_equal(got, sd.labels)
            n = info.n_gamma[l]
            assert n == len(sd.gamma_idx)
            gi = torch.empty(n, dtype=torch.int32, device="cuda")
            fl = torch.empty(n, dtype=torch.uint8, device="cuda")
            ft = torch.empty(n, 3, dtype=torch.float64, device="cuda")
            abi.dpm_dd2_gamma(d, l, gi, fl, ft)
            torch.cuda.synchronize()
            assert np.array_equal(gi.cpu().numpy(), sd.gamma_idx)
            assert np.array_equal(fl.cpu().numpy(), sd.on_g.astype(np.uint8) + 2 * sd.on_z.astype(np.uint8))
            np.testing.assert_allclose(ft.cpu().numpy(), sd.footG, rtol=0, atol=1e-15)
            assert info.n_rows[l] == len(sd.rows)
            assert info.n_wedge[l] == int(np.count_nonzero(sd.on_g & sd.on_z))
    finally:
        abi.dpm_dd2_destroy(d)


@pytest.mark.parametrize("gs", [2, 1])
@pytest.mark.parametrize("prec", [abi.DPM_PREC_FP64, abi.DPM_PREC_FP32])
def test_bep_matrix_matches_oracle(ctx, prec, gs):
    MZ, MG = 4, 6
    S = oracle_setup(20, 20, MZ, MG, gs=gs)
    d = abi.dpm_dd2_build(ctx, params(20, 20, MZ, MG, prec, gs), SIGMA)
    try:
        info = abi.dpm_dd2_get_info(d)
        m = info.n_rows[0] + info.n_rows[1]
        A = torch.empty(m * info.ncol, dtype=torch.float64, device="cuda")
        abi.dpm_dd2_matrix(d, A)
        torch.cuda.synchronize()
        A = A.cpu().numpy().reshape(info.ncol, m).T
    finally:
        abi.dpm_dd2_destroy(d)
    assert A.shape == S.A.shape
    err = np.max(np.abs(A - S.A), axis=0) / np.max(np.abs(S.A), axis=0)
    assert np.max(err) < (1e-12 if prec == abi.DPM_PREC_FP64 else 1e-5), np.max(err)


@pytest.mark.parametrize("gs", [2, 1])
@pytest.mark.parametrize("prec", [abi.DPM_PREC_FP64, abi.DPM_PREC_FP32])
def test_elliptic_solve_matches_oracle(ctx, prec, gs):
    MZ, MG = 6, 10
    S = oracle_setup(24, 22, MZ, MG, gs=gs)
    fs, gn = [], []
    for sd in S.sub:
        X, Y, Z = global_mesh(sd)
        fs.append(SIGMA * u_exact(X, Y, Z) - lap_exact(X, Y, Z))
        xf = sd.footG + sd.origin
        gn.append(np.sum(grad_exact(xf[:, 0], xf[:, 1], xf[:, 2]) * sd.normalG, axis=1))
    if prec == abi.DPM_PREC_FP32:
        fs = [f.astype(np.float32).astype(np.float64) for f in fs]
    u1, u2, C = O.dd2_elliptic_solve(S, fs[0], fs[1], gn)
    dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
    d = abi.dpm_dd2_build(ctx, params(24, 22, MZ, MG, prec, gs), SIGMA)
    try:
        fd = [torch.from_numpy(f).to("cuda", dt).contiguous() for f in fs]
        ud = [torch.empty_like(f) for f in fd]
        gd = [torch.from_numpy(g).to("cuda", torch.float64) for g in gn]
        Cd = torch.empty(S.ncol, dtype=torch.float64, device="cuda")
        abi.dpm_dd2_solve(d, fd[0], fd[1], ud[0], ud[1], gd[0], gd[1], Cd)
        torch.cuda.synchronize()
    finally:
        abi.dpm_dd2_destroy(d)
    for sd, ref, got in zip(S.sub, (u1, u2), ud):
        g = got.cpu().numpy().astype(np.float64)
        m = sd.sets["Np"]
        rel = np.max(np.abs(np.where(m, g - ref, 0))) / np.max(np.abs(np.where(m, ref, 0)))
        assert rel < TOL[prec], rel
        X, Y, Z = global_mesh(sd)
        # discretisation error (the 2-term Gamma extension drops an O(h^2) term there)
        assert np.max(np.abs(np.where(sd.sets["Mp"], g - u_exact(X, Y, Z), 0))) < (1e-4 if gs == 2 else 1e-3)


@pytest.mark.parametrize("gs", [2, 1])
@pytest.mark.parametrize("prec,tol", [(abi.DPM_PREC_FP64, 1e-11), (abi.DPM_PREC_FP32, 1e-5)])
def test_time_loop_matches_oracle(ctx, prec, tol, gs):
    MZ, MG, N1, N2 = 6, 6, 20, 20
    (lo1, hi1, o1), (lo2, hi2, o2) = boxes(N1, N2)
    h = min(2 * RZ / (N1 - 3), 2 * R / (N2 - 3))
    rho0, c0 = Gaussian(200.0, 20.0, (0.0, 0.0, 0.25)), Gaussian(0.0, 1.0)
    st = O.DD2PKSState((0.0, 0.0, 0.0), R, RZ, R, N1, lo1, hi1, o1, N2, lo2, hi2, o2, MZ, MG, 1.0,
                       0.5 * h * h, rho0, c0, dt_mode="fixed", gamma_series=gs)
    pk = abi.dpm_dd2_pks_create(ctx, params(N1, N2, MZ, MG, prec, gs), 1.0, 0.5 * h * h, 0, 0, 1, rho0, c0)
    try:
        for _ in range(3):
            st.step()
            s = abi.dpm_dd2_pks_step(pk, 1, True)
            d = st.diagnostics()
            for key in ("mass", "max_rho", "m2", "free_energy"):
                assert abs(getattr(s, key) - d[key]) <= tol * abs(d[key]), (key, getattr(s, key), d[key])
        dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
        for l, sd in enumerate(st.sub):
            rho = torch.empty(sd.N ** 3, dtype=dt, device="cuda")
            c = torch.empty_like(rho)
            abi.dpm_dd2_pks_get_state(pk, l, rho, c)
            torch.cuda.synchronize()
            m = sd.sets["Np"].reshape(-1)
            for got, ref in ((rho, st.rho[l]), (c, st.c[l])):
                g = got.cpu().numpy().astype(np.float64)
                r = ref.reshape(-1)
                assert np.max(np.abs(g[m] - r[m])) <= tol * np.max(np.abs(r[m])), np.max(np.abs(g[m] - r[m])) / np.max(np.abs(r[m]))
    finally:
        abi.dpm_dd2_pks_destroy(pk)


def _dd2_run(ctx, P, Ns, dtm, mode, rebuild, graph, steps, prec, rho0, c0):
    pk = abi.dpm_dd2_pks_create(ctx, P, 1.0, dtm, mode, rebuild, 1, rho0, c0)
    try:
        if graph:
            abi.dpm_dd2_pks_set_graph(pk, True)
        flags = [abi.dpm_dd2_pks_step(pk, 1, True).rebuilt for _ in range(steps)]
        st = abi.dpm_dd2_pks_step(pk, 0, True)
        dt = torch.float64 if prec == abi.DPM_PREC_FP64 else torch.float32
        out = []
        for l, Nl in enumerate(Ns):
            rho = torch.empty(Nl ** 3, dtype=dt, device="cuda")
            c = torch.empty_like(rho)
            abi.dpm_dd2_pks_get_state(pk, l, rho, c)
            out += [rho, c]
        torch.cuda.synchronize()
        if graph:
            abi.dpm_dd2_pks_set_graph(pk, False)
        return flags, st, [t.cpu().numpy() for t in out]
    finally:
        abi.dpm_dd2_pks_destroy(pk)


@pytest.mark.parametrize("prec,mode,rebuild", [(abi.DPM_PREC_FP64, 0, 0), (abi.DPM_PREC_FP32, 1, 0),
                                               (abi.DPM_PREC_FP32, 1, 1)])
def test_graph_steps_match_host_steps(ctx, prec, mode, rebuild):
    """Case 2's device-resident steps replayed as a CUDA graph equal the
    host-driven steps bit for bit (rebuild flags after the first step of the
    fixed-dt mode, whose BEP the graph path builds when graph stepping starts;
    dt, statistics, state)."""
    MZ, MG, N1, N2 = 6, 6, 20, 20
    h = min(2 * RZ / (N1 - 3), 2 * R / (N2 - 3))
    rho0, c0 = Gaussian(200.0, 20.0, (0.0, 0.0, 0.25)), Gaussian(100.0, 10.0, (0.0, 0.0, 0.25))
    P = params(N1, N2, MZ, MG, prec, 1)
    a = _dd2_run(ctx, P, (N1, N2), 0.5 * h * h, mode, rebuild, False, 4, prec, rho0, c0)
    b = _dd2_run(ctx, P, (N1, N2), 0.5 * h * h, mode, rebuild, True, 4, prec, rho0, c0)
    first = 1 if mode == 0 and not rebuild else 0
    assert a[0][first:] == b[0][first:], (a[0], b[0])
    for key in ("t", "dt", "step", "mass", "max_rho", "min_rho", "m2", "free_energy"):
        assert getattr(a[1], key) == getattr(b[1], key), key
    for x, y in zip(a[2], b[2]):
        assert np.array_equal(x, y)
