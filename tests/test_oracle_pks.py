"""Pins of the oracle's PKS discretisation (eqs. discrete_chemotaxis ..
slope_limiter, the flux split of the positivity proof, eq. cfl_condition)."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import dpm_oracle as O
from paper_1811_03557_gb300.workloads import (Geometry, Gaussian, TEST_A_C0, TEST_A_RHO0,
                                              random_field)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_minmod_golden_cases():
    rows = np.loadtxt(os.path.join(GOLD, "minmod_cases.txt"))
    got = O.minmod(rows[:, 0], rows[:, 1], rows[:, 2])
    assert np.array_equal(got, rows[:, 3])


def test_paper_parameters_match_workloads():
    p = json.load(open(os.path.join(GOLD, "paper_parameters.json")))
    assert TEST_A_RHO0.amp == p["test_A"]["rho0"]["amp"] and TEST_A_RHO0.alpha == p["test_A"]["rho0"]["alpha"]
    assert TEST_A_C0.amp == p["test_A"]["c0"]["amp"] and TEST_A_C0.alpha == p["test_A"]["c0"]["alpha"]


def _setup(N=20, lo=-1.3, hi=1.3):
    g = Geometry.sphere(1.0)
    return g, O.point_sets(O.inside_mask(g, N, lo, hi)), O.grid_spacing(N, lo, hi), O.mesh(N, lo, hi)


@pytest.mark.parametrize("ax", [0, 1, 2])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_linear_fields_give_closed_form_flux(ax, sign):
    """rho = a + b x_ax, c = s*k x_ax: exact slopes, g = chi * (s k) * b away from gamma."""
    g, sets, h, XYZ = _setup()
    x = XYZ[ax]
    a, b, k, chi = 5.0, 1.5, 2.0, 0.7
    rho = np.where(sets["Np"], a + b * x, 0.0)
    c = np.where(sets["Np"], sign * k * x, 0.0)
    gterm = O.convective_term(rho, c, sets, h, chi)
    # nodes whose x_ax-neighbours j-1, j, j+1 are all in M^+ have exact slopes on both faces
    deep = sets["Mp"].copy()
    for s in (1, -1, 2, -2):
        deep &= O._shift(sets["Mp"], ax, s, False)
    assert deep.sum() > 50
    assert np.allclose(gterm[deep], chi * sign * k * b, rtol=1e-12, atol=1e-9)


def _face_split(rho, c, sets, h, chi, dt):
    """f_rho = F^E+F^W+F^N+F^S+F^U+F^D node by node (positivity proof, flux split)."""
    N = rho.shape[0]
    Np = sets["Np"]

    def slope(p, ax):
        e = np.eye(3, dtype=int)[ax]
        pp, pm = tuple(np.add(p, e)), tuple(np.subtract(p, e))
        if not (Np[p] and Np[pp] and Np[pm]):
            return 0.0
        return float(O.minmod(np.array(2 * (rho[pp] - rho[p]) / h), np.array((rho[pp] - rho[pm]) / (2 * h)),
                              np.array(2 * (rho[p] - rho[pm]) / h)))

    f = np.zeros_like(rho)
    for p in itertools.product(range(2, N - 2), repeat=3):
        if not sets["Mp"][p]:
            continue
        tot = 0.0
        for ax in range(3):
            e = np.eye(3, dtype=int)[ax]
            pp, pm = tuple(np.add(p, e)), tuple(np.subtract(p, e))
            sE = slope(p, ax)
            rE, rW = rho[p] + h / 2 * sE, rho[p] - h / 2 * sE
            gcp, gcm = (c[pp] - c[p]) / h, (c[p] - c[pm]) / h
            face_p = rE if gcp > 0 else rho[pp] - h / 2 * slope(pp, ax)
            face_m = (rho[pm] + h / 2 * slope(pm, ax)) if gcm > 0 else rW
            FE = rE / 6 - dt * chi * gcp / h * face_p
            FW = rW / 6 + dt * chi * gcm / h * face_m
            tot += FE + FW
        f[p] = tot
    return f


def test_flux_split_identity():
    g, sets, h, _ = _setup(N=14, lo=-1.45, hi=1.45)
    rho = np.where(sets["Np"], random_field(20, sets["Np"].shape, 0.0, 3.0), 0.0)
    c = np.where(sets["Np"], random_field(21, sets["Np"].shape, 0.0, 2.0), 0.0)
    dt, chi = 0.003, 1.0
    f_rho, _ = O.pks_rhs(rho, c, sets, h, chi, dt)
    f_split = _face_split(rho, c, sets, h, chi, dt)
    assert np.allclose(f_rho, f_split, atol=1e-12)


def test_cfl_dt_gives_nonnegative_rhs():
    g, sets, h, _ = _setup(N=18)
    for seed in range(4):
        rho = np.where(sets["Np"], random_field(30 + seed, sets["Np"].shape, 0.0, 5.0), 0.0)
        c = np.where(sets["Np"], random_field(40 + seed, sets["Np"].shape, 0.0, 50.0), 0.0)
        dt = O.cfl_dt(c, sets, h, 1.0)
        f_rho, f_c = O.pks_rhs(rho, c, sets, h, 1.0, dt)
        assert f_rho[sets["Mp"]].min() >= -1e-12 * rho.max()
        assert f_c[sets["Mp"]].min() >= 0.0
        # 2x the CFL step is allowed to go negative for some seeds; 1x never
        assert dt > 0


def _cone(sets, h, G, p):
    """c = G h (|i - i_p| + |j - j_p| + |k - k_p|): |grad_h c| = G on every face."""
    N = sets["Np"].shape[0]
    i, j, k = np.meshgrid(*(np.arange(N),) * 3, indexing="ij")
    return G * h * (np.abs(i - p[0]) + np.abs(j - p[1]) + np.abs(k - p[2])).astype(np.float64)


def test_cfl_dt_denominator_is_the_papers_and_sharp():
    """eq. cfl_condition: dt = h / (6 chi max|grad_h c|), the 6 read from the
    golden file.  The bound is sharp: a single spike of density at the bottom of
    a cone of c (every face gradient equal to G, pointing away from the spike)
    sends the whole spike out through its six faces, so f_rho at the spike is
    exactly 0 at the CFL step and -rho at twice the step."""
    den = json.load(open(os.path.join(GOLD, "paper_parameters.json")))["cfl_denominator"]["value"]
    g, sets, h, _ = _setup(N=18)
    p = (9, 9, 9)
    assert sets["Mp"][p]
    for G, chi in ((3.0, 1.0), (40.0, 0.5)):
        c = _cone(sets, h, G, p)
        dt = O.cfl_dt(c, sets, h, chi)
        assert dt == pytest.approx(h / (den * chi * G), rel=1e-12)
        rho = np.zeros_like(c)
        rho[p] = 7.0
        f1, _ = O.pks_rhs(rho, c, sets, h, chi, dt)
        f2, _ = O.pks_rhs(rho, c, sets, h, chi, 2 * dt)
        assert abs(f1[p]) <= 1e-12 * 7.0
        assert f2[p] == pytest.approx(-7.0, rel=1e-12)
        assert f1[sets["Mp"]].min() >= -1e-12 * 7.0
    # per-axis maxima: the bound is set by the steepest axis
    X, Y, Z = O.mesh(18, -1.3, 1.3)
    c = np.where(sets["Np"], 1.0 * X - 4.0 * Y + 2.5 * Z, 0.0)
    assert O.cfl_dt(c, sets, h, 1.0) == pytest.approx(h / (den * 4.0), rel=1e-9)


def test_interior_fluxes_telescope():
    """Sum over M^+ of h^3 g = boundary fluxes; with c flat near gamma it is 0."""
    g, sets, h, (X, Y, Z) = _setup(N=22)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    c = np.where(sets["Np"], np.maximum(0.0, 0.5 - r) ** 2, 0.0)
    rho = np.where(sets["Np"], 1.0 + random_field(50, X.shape, 0, 1), 0.0)
    gterm = O.convective_term(rho, c, sets, h, 1.0)
    assert abs(gterm[sets["Mp"]].sum()) < 1e-10 * np.abs(gterm).sum()


def test_diagnostics_closed_forms():
    g, sets, h, (X, Y, Z) = _setup(N=16)
    N = 16
    rho = np.where(sets["Np"], 2.0, 0.0)
    c = np.where(sets["Np"], 0.0, 0.0)
    d = O.diagnostics(rho, c, sets, h, N, -1.3, 1.3)
    nMp = sets["Mp"].sum()
    assert d["mass"] == pytest.approx(2.0 * nMp * h ** 3)
    assert d["max_rho"] == 2.0
    # free energy of a constant density with c = 0: rho log rho per cell
    assert d["free_energy"] == pytest.approx(nMp * h ** 3 * 2.0 * np.log(2.0))


def test_second_moment_of_single_nodes():
    """eq. sd-norm:second-moment for a density that is one unit at a single node
    p of M^+ and zero elsewhere: M_h = h^3 |x_p|^2, with x_p = lo + (index + 1) h
    (the node grid); nodes of M^- contribute nothing."""
    N, lo, hi = 16, -1.3, 1.3
    g, sets, h, _ = _setup(N=N, lo=lo, hi=hi)
    for p in [(8, 8, 8), (3, 8, 10), (12, 5, 7), (0, 0, 0)]:
        rho = np.zeros((N, N, N))
        rho[p] = 1.0
        d = O.diagnostics(rho, np.zeros_like(rho), sets, h, N, lo, hi)
        x = [lo + (q + 1) * h for q in p]
        want = h ** 3 * (x[0] ** 2 + x[1] ** 2 + x[2] ** 2) if sets["Mp"][p] else 0.0
        assert d["m2"] == pytest.approx(want, rel=1e-12, abs=1e-300)
        assert d["mass"] == pytest.approx(h ** 3 if sets["Mp"][p] else 0.0, rel=1e-12, abs=1e-300)


def _free_energy_linear_c(sets, h, X, rho0, a, k, ax, grad_coef):
    """Closed form of eq. sd-norm:free-energy for rho = rho0 on M^+ and
    c = a + k x_ax on the whole grid: per node rho0 ln rho0 - rho0 c + c^2/2
    plus grad_coef * (2 h k)^2 (the central differences of a linear c are 2 h k
    along ax and 0 along the other axes)."""
    Mp = sets["Mp"]
    x = X[ax][Mp]
    n = Mp.sum()
    return h ** 3 * (n * rho0 * np.log(rho0) - rho0 * np.sum(a + k * x) + 0.5 * np.sum((a + k * x) ** 2)
                     + n * grad_coef * (2.0 * h * k) ** 2)


@pytest.mark.parametrize("ax", [0, 1, 2])
def test_free_energy_linear_c_closed_form(ax):
    """Every term of eq. sd-norm:free-energy: the gradient term of a linear c is
    (2 h k)^2 / (8 h^2) = k^2 / 2 per node whatever h is; -rho c and c^2 / 2
    against their sums.  A 1/(4 h^2) in place of 1/(8 h^2), a dropped -rho c or
    a + sign on it each move F by far more than the tolerance."""
    N, lo, hi = 16, -1.3, 1.3
    g, sets, h, XYZ = _setup(N=N, lo=lo, hi=hi)
    rho0, a, k = 1.5, 2.0, 3.0
    rho = np.where(sets["Np"], rho0, 0.0)
    c = a + k * XYZ[ax]
    F = O.diagnostics(rho, c, sets, h, N, lo, hi)["free_energy"]
    want = _free_energy_linear_c(sets, h, XYZ, rho0, a, k, ax, 1.0 / (8.0 * h * h))
    assert F == pytest.approx(want, rel=1e-12)
    # planted mistakes, each evaluated in the same closed form, are all rejected
    wrong_grad = _free_energy_linear_c(sets, h, XYZ, rho0, a, k, ax, 1.0 / (4.0 * h * h))
    wrong_rc = want + h ** 3 * rho0 * np.sum((a + k * XYZ[ax])[sets["Mp"]])
    wrong_sign = want + 2.0 * h ** 3 * rho0 * np.sum((a + k * XYZ[ax])[sets["Mp"]])
    for w in (wrong_grad, wrong_rc, wrong_sign):
        assert abs(F - w) > 1e-3 * abs(F)


@pytest.fixture(scope="module")
def pks_run():
    st = O.PKSState(Geometry.sphere(1.0), 24, -1.25, 1.25, K=4, beta=1, chi=1.0, dt_max=1e-3,
                    rho0=TEST_A_RHO0, c0=TEST_A_C0, dt_mode="cfl")
    hist = [O.diagnostics(st.rho, st.c, st.sets, st.h, st.N, st.lo, st.hi)]
    for _ in range(4):
        st.step()
        hist.append(O.diagnostics(st.rho, st.c, st.sets, st.h, st.N, st.lo, st.hi))
    return st, hist


def test_pks_positivity_under_cfl(pks_run):
    st, hist = pks_run
    assert all(hd["min_rho"] >= -1e-9 * hd["max_rho"] for hd in hist)
    assert all(hd["min_c"] >= -1e-9 for hd in hist)


def test_pks_free_energy_decreases(pks_run):
    st, hist = pks_run
    F = [hd["free_energy"] for hd in hist]
    assert all(b <= a + 1e-9 * abs(a) for a, b in zip(F, F[1:])), F


def test_pks_mass_approximately_conserved(pks_run):
    st, hist = pks_run
    m = [hd["mass"] for hd in hist]
    assert max(abs(x - m[0]) for x in m) / m[0] < 0.05


def test_pks_solution_keeps_cube_symmetry(pks_run):
    st, _ = pks_run
    for arr in (st.rho, st.c):
        scale = np.abs(arr).max()
        for perm in [(1, 0, 2), (2, 1, 0)]:
            assert np.allclose(arr, arr.transpose(perm), atol=1e-9 * scale)
        for ax in range(3):
            assert np.allclose(arr, np.flip(arr, axis=ax), atol=1e-9 * scale)


def _time_errors(taus, tau_ref, N=16, dT=1e-7, T=1e-6):
    """Test (A) on a fixed N = 16 mesh of the paper's geometry (sphere r = 0.5 in
    [-r - 2h, r + 2h]^3), dt = dT/tau: max over M^+ of rho and c at time T
    against the dt = dT/tau_ref run (the convergence-in-time protocol of
    Section 4)."""
    h = 1.0 / (N - 3)
    lo, hi = -0.5 - 2 * h, 0.5 + 2 * h

    def final(tau):
        st = O.PKSState(Geometry.sphere(0.5), N, lo, hi, 0, 1, 1.0, dT / tau, rho0=TEST_A_RHO0,
                        c0=TEST_A_C0, dt_mode="fixed", clamp=True)
        for _ in range(int(round(T * tau / dT))):
            st.step()
        assert abs(st.t - T) < 1e-12 * T * tau
        return st

    ref = final(tau_ref)
    m = ref.sets["Mp"]
    out = []
    for tau in taus:
        s = final(tau)
        out.append((np.max(np.abs(np.where(m, s.rho - ref.rho, 0.0))),
                    np.max(np.abs(np.where(m, s.c - ref.c, 0.0)))))
    return np.array(out)


def test_first_order_in_time():
    """The IMEX step is first order in dt: with E(tau) ~ C (1/tau - 1/tau_ref),
    the rate log2(E(tau)/E(2 tau)) is log2((1 - 1/32)/(1/2 - 1/32)) = 1.047 for
    tau = 1 -> 2 and log2((1/2 - 1/32)/(1/4 - 1/32)) = 1.100 for 2 -> 4 (the same
    rise of the apparent rate as the reference nears, seen in Section 4's
    tables), for rho and for c."""
    E = _time_errors((1, 2, 4), 32)
    rates = np.log2(E[:-1] / E[1:])
    want = np.array([np.log2((1 - 1 / 32) / (1 / 2 - 1 / 32)), np.log2((1 / 2 - 1 / 32) / (1 / 4 - 1 / 32))])
    np.testing.assert_allclose(rates[:, 0], want, atol=0.03)
    np.testing.assert_allclose(rates[:, 1], want, atol=0.03)
    assert 1e-7 < E[0, 0] / TEST_A_RHO0.amp < 1e-3     # the error is resolved, not rounding


def test_planted_dt_mistake_breaks_time_convergence(monkeypatch):
    """A flux that takes its dt from the base step dT instead of the current dt
    (a plausible mistake) is inconsistent: the errors stop falling with dt."""
    orig = O.pks_rhs

    def wrong(rho, c, sets, h, chi, dt):
        f_rho, _ = orig(rho, c, sets, h, chi, 1e-7)
        _, f_c = orig(rho, c, sets, h, chi, dt)
        return f_rho, f_c

    monkeypatch.setattr(O, "pks_rhs", wrong)
    E = _time_errors((1, 2), 8)
    assert E[1, 0] > 0.8 * E[0, 0]
