"""Pins of the oracle's domain decomposition (Section 3, Case 1: a ball and the
spherical shell around it, each on its own grid, coupled through the shared
series on the interface Z): the shell's point sets and foot points against
their closed forms, the coupled solve against the manufactured solution with
the single-domain solve's accuracy as the yardstick, the structure of the
stacked BEP matrix, a planted orientation error that the accuracy check
catches, and the invariants of the coupled time loop."""
import numpy as np
import pytest

from oracle import dpm_oracle as O
from paper_1811_03557_gb300.workloads import (TEST_A_C0, TEST_A_RHO0, Geometry, manufactured_grad,
                                              manufactured_u)


def boxes(N1, N2, r1, r2):
    h1, h2 = 2 * r1 / (N1 - 3), 2 * r2 / (N2 - 3)
    return (-r1 - 2 * h1, r1 + 2 * h1), (-r2 - 2 * h2, r2 + 2 * h2)


def test_shell_sets_and_foot_points():
    N, r2, r1 = 22, 1.0, 0.45
    lo, hi = -1.2, 1.2
    g = O.Shell(r2, r1)
    m = O.inside_mask(g, N, lo, hi)
    X, Y, Z = O.mesh(N, lo, hi)
    R = np.sqrt(X * X + Y * Y + Z * Z)
    # brute force away from round-off ties
    safe = (np.abs(R - r1) > 1e-9) & (np.abs(R - r2) > 1e-9)
    assert np.array_equal(m[safe], ((R > r1) & (R < r2))[safe])
    P = np.array([[0.3, 0.1, -0.2], [0.9, 0.3, 0.2], [0.0, 0.0, 0.5]])
    xf, d, n = O.foot_point(g, P)
    rho = np.linalg.norm(P, axis=1)
    r = np.where(np.abs(rho - r2) <= np.abs(rho - r1), r2, r1)
    np.testing.assert_allclose(np.linalg.norm(xf, axis=1), r, rtol=1e-15)
    np.testing.assert_allclose(d, rho - r, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(n, P / rho[:, None], rtol=1e-15)


def _dd_solve(N1, N2, K, r1=0.5, r2=1.0, sigma=1001.0):
    (lo1, hi1), (lo2, hi2) = boxes(N1, N2, r1, r2)
    S = O.DDSetup((0, 0, 0), r1, r2, N1, lo1, hi1, N2, lo2, hi2, K, K, sigma)
    fs = []
    for sd in S.sub:
        X, Y, Z = O.mesh(sd.N, sd.lo, sd.hi)
        fs.append((sigma + 1) * manufactured_u(X, Y, Z))
    S2 = S.sub[1]
    gn = np.sum(manufactured_grad(S2.xf[:, 0], S2.xf[:, 1], S2.xf[:, 2]) * S2.normal, axis=1)
    u1, u2, C = O.dd_elliptic_solve(S, fs[0], fs[1], gn)
    errs = []
    for sd, u in zip(S.sub, (u1, u2)):
        X, Y, Z = O.mesh(sd.N, sd.lo, sd.hi)
        errs.append(np.max(np.abs(np.where(sd.sets["Mp"], u - manufactured_u(X, Y, Z), 0))))
    return S, errs


def _sd_error(N, K, r=1.0, sigma=1001.0):
    (lo, hi) = boxes(N, N, r, r)[1]
    s = O.DPMSetup(Geometry.sphere(r), N, lo, hi, K, 1, sigma)
    X, Y, Z = O.mesh(N, lo, hi)
    gn = np.sum(manufactured_grad(s.xf[:, 0], s.xf[:, 1], s.xf[:, 2]) * s.normal, axis=1)
    u, _, _ = O.dpm_elliptic_solve(s, (sigma + 1) * manufactured_u(X, Y, Z), gn)
    return np.max(np.abs(np.where(s.sets["Mp"], u - manufactured_u(X, Y, Z), 0)))


def test_dd_elliptic_matches_single_domain_accuracy():
    """(sigma - Lap) u = f with u = e^x sin y cos z: the coupled solve is as
    accurate in the shell as the single-domain solve on the same grid, and more
    accurate in the finer ball."""
    S, (e1, e2) = _dd_solve(20, 20, 8)
    esd = _sd_error(20, 8)
    assert e2 <= 1.2 * esd and esd < 1e-4
    assert e1 <= e2
    # refining both grids does not lose accuracy
    _, (f1, f2) = _dd_solve(36, 36, 8)
    assert f1 < e1 and f2 < e2


def test_dd_bep_structure():
    S, _ = _dd_solve(20, 20, 4)
    m1 = len(S.sub[0].gin_idx)
    nz = S.nz
    # Gamma unknowns do not act on the ball's rows; every Z unknown does
    assert np.all(S.A[:m1, 3 * nz:] == 0.0)
    assert np.all(np.max(np.abs(S.A[:m1, :3 * nz]), axis=0) > 0)
    sv = np.linalg.svd(S.A / np.linalg.norm(S.A, axis=0), compute_uv=False)
    assert sv[-1] > 0 and sv[0] / sv[-1] < 100.0


def test_planted_orientation_error_is_caught(monkeypatch):
    """Flip the sign of s in the shell's Z series (a plausible mistake: the
    inner sphere's outward normal of the shell points to the centre): the
    coupled solve then loses its accuracy."""
    _, (e1, e2) = _dd_solve(20, 20, 6)
    orig = O.DDSetup.column_density

    def flipped(self, l, k):
        out = orig(self, l, k)
        if l == 1 and self.nz <= k < 2 * self.nz:
            out = -out
        return out

    monkeypatch.setattr(O.DDSetup, "column_density", flipped)
    _, (g1, g2) = _dd_solve(20, 20, 6)
    assert max(g1, g2) > 20 * max(e1, e2)


@pytest.mark.slow
def test_dd_pks_invariants():
    r1, r2, N1, N2 = 0.25, 0.5, 20, 20
    (lo1, hi1), (lo2, hi2) = boxes(N1, N2, r1, r2)
    h = min(2 * r1 / (N1 - 3), 2 * r2 / (N2 - 3))
    st = O.DDPKSState((0, 0, 0), r1, r2, N1, lo1, hi1, N2, lo2, hi2, 0, 0, 1.0, 0.5 * h * h,
                      TEST_A_RHO0, TEST_A_C0)
    d0 = None
    prev = None
    for _ in range(4):
        st.step()
        d = st.diagnostics()
        d0 = d0 or d
        assert d["min_rho"] >= -1e-9 * d["max_rho"]   # positivity up to rounding
        if prev:
            assert d["free_energy"] < prev["free_energy"]
            assert d["m2"] < prev["m2"]
            assert d["max_rho"] > prev["max_rho"]
        prev = d
    assert abs(prev["mass"] - d0["mass"]) < 1e-3 * d0["mass"]
