"""Pins of the oracle's DPM operators against the paper's theorems.

* Theorem 2.1 (BEP): the trace on gamma of any solution of the difference
  equation on M^+ satisfies u_gamma - P_gamma u_gamma = Tr_gamma G f; the
  solution is computed here by a sparse direct solve on N^+, without the DST.
* Proposition 2.2: rank(I - P_gamma) = |gamma_in|.
* Theorem 2.3: a density satisfying the reduced BEP on gamma_in also
  satisfies it on gamma_ex.
* Green's formula (Proposition 2.7 and the positivity proof): u = P u_gamma + G f
  solves the difference equation on M^+ for any density.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import dpm_oracle as O
from paper_1811_03557_gb300.workloads import Geometry, random_field

CASES = [(Geometry.sphere(1.0), 10, -1.45, 1.45, 40.0),
         (Geometry.ellipsoid(1.0, 0.8, 0.6), 12, -1.35, 1.35, 7.0)]


def solve_on_Nplus(sets, f, u_ex, h, sigma):
    """(sigma - Lap_h) u = f on M^+, u = u_ex on gamma_ex: sparse direct solve."""
    N = f.shape[0]
    Mp = np.flatnonzero(sets["Mp"].reshape(-1))
    pos = -np.ones(N ** 3, dtype=np.int64)
    pos[Mp] = np.arange(len(Mp))
    rows, cols, vals = [], [], []
    rhs = f.reshape(-1)[Mp].copy()
    known = u_ex.reshape(-1)
    for r, p in enumerate(Mp):
        i, j, k = np.unravel_index(p, (N, N, N))
        rows.append(r); cols.append(r); vals.append(sigma + 6.0 / h ** 2)
        for di, dj, dk in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
            q = np.ravel_multi_index((i + di, j + dj, k + dk), (N, N, N))
            if pos[q] >= 0:
                rows.append(r); cols.append(pos[q]); vals.append(-1.0 / h ** 2)
            else:
                rhs[r] += known[q] / h ** 2
    A = sp.csc_matrix((vals, (rows, cols)), shape=(len(Mp), len(Mp)))
    u = np.zeros(N ** 3)
    u[Mp] = spla.spsolve(A, rhs)
    gex = np.flatnonzero(sets["gex"].reshape(-1))
    u[gex] = known[gex]
    return u.reshape(N, N, N)


def i_minus_p_matrix(s):
    """(I - P_gamma) as a |gamma| x |gamma| matrix, one AP per unit density."""
    n = len(s.gamma_idx)
    M = np.zeros((n, n))
    for e in range(n):
        v = np.zeros(n)
        v[e] = 1.0
        Pv = O.difference_potential(s.gamma_grid(v), s.sets, s.h, s.sigma)
        M[:, e] = v - Pv.reshape(-1)[s.gamma_idx]
    return M


@pytest.mark.parametrize("geom,N,lo,hi,sigma", CASES)
def test_theorem_bep_holds_for_traces_of_solutions(geom, N, lo, hi, sigma):
    s = O.DPMSetup(geom, N, lo, hi, K=2, beta=1, sigma=sigma, build_bep=False)
    f = random_field(10, (N, N, N), -1, 1)
    u_ex = random_field(11, (N, N, N), -1, 1)
    u = solve_on_Nplus(s.sets, f, u_ex, s.h, sigma)
    ug = u.reshape(-1)[s.gamma_idx]
    Pu = O.difference_potential(s.gamma_grid(ug), s.sets, s.h, sigma).reshape(-1)[s.gamma_idx]
    Gf = O.particular_solution(f, s.sets, s.h, sigma).reshape(-1)[s.gamma_idx]
    assert np.max(np.abs(ug - Pu - Gf)) < 1e-11 * np.max(np.abs(ug))
    # ... and a density that is not such a trace does not satisfy it
    bad = ug.copy()
    bad[s.gin_pos[0]] += 1.0
    Pb = O.difference_potential(s.gamma_grid(bad), s.sets, s.h, sigma).reshape(-1)[s.gamma_idx]
    assert np.max(np.abs(bad - Pb - Gf)) > 1e-3


@pytest.mark.parametrize("geom,N,lo,hi,sigma", CASES)
def test_rank_of_bep_is_gamma_in(geom, N, lo, hi, sigma):
    s = O.DPMSetup(geom, N, lo, hi, K=1, beta=0, sigma=sigma, build_bep=False)
    M = i_minus_p_matrix(s)
    sv = np.linalg.svd(M, compute_uv=False)
    rank = int(np.sum(sv > 1e-9 * sv[0]))
    assert rank == len(s.gin_idx)
    # P_gamma is a projection: (I-P)^2 = (I-P)
    assert np.allclose(M @ M, M, atol=1e-9)


@pytest.mark.parametrize("geom,N,lo,hi,sigma", CASES[:1])
def test_reduced_bep_implies_full_bep(geom, N, lo, hi, sigma):
    s = O.DPMSetup(geom, N, lo, hi, K=1, beta=0, sigma=sigma, build_bep=False)
    M = i_minus_p_matrix(s)
    f = random_field(12, (N, N, N), -1, 1)
    Gf = O.particular_solution(f, s.sets, s.h, sigma).reshape(-1)[s.gamma_idx]
    ex_pos = np.setdiff1d(np.arange(len(s.gamma_idx)), s.gin_pos)
    u = np.zeros(len(s.gamma_idx))
    u[ex_pos] = random_field(13, len(ex_pos), -1, 1)
    rin = s.gin_pos
    u[rin] = np.linalg.solve(M[np.ix_(rin, rin)], Gf[rin] - M[np.ix_(rin, ex_pos)] @ u[ex_pos])
    assert np.max(np.abs(M[ex_pos] @ u - Gf[ex_pos])) < 1e-10


@pytest.mark.parametrize("geom,N,lo,hi,sigma", CASES)
def test_greens_formula_solves_difference_equation(geom, N, lo, hi, sigma):
    s = O.DPMSetup(geom, N, lo, hi, K=2, beta=1, sigma=sigma, build_bep=False)
    f = random_field(14, (N, N, N), -1, 1)
    ug = random_field(15, len(s.gamma_idx), -1, 1)
    u = O.particular_solution(f, s.sets, s.h, sigma) + O.difference_potential(
        s.gamma_grid(ug), s.sets, s.h, sigma)
    r = O.apply_L(u, s.h, sigma) - f
    assert np.max(np.abs(np.where(s.sets["Mp"], r, 0.0))) < 1e-10
    # on gamma_ex the potential reproduces the density up to the BEP residual only:
    # away from N^+ u is zero by the restriction
    assert np.all(u[~s.sets["Np"]] == 0.0)


def test_bep_matrix_column_is_i_minus_p_of_basis():
    g, N, lo, hi, sigma = Geometry.sphere(1.0), 10, -1.45, 1.45, 40.0
    s = O.DPMSetup(g, N, lo, hi, K=2, beta=1, sigma=sigma)
    M = i_minus_p_matrix(s)
    Psi = s.basis_densities()
    assert np.allclose(s.A, (M @ Psi)[s.gin_pos], atol=1e-11)
    assert s.A.shape == (len(s.gin_idx), 2 * 9)
