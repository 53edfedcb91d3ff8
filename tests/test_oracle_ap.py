"""Pins of the oracle's auxiliary-problem solve (Definition 2.4).

The AP is the linear system (sigma - Lap_h) v = q on M^0 with v = 0 on the
ghost layer.  The oracle solves it with the 3D DST-I; these tests pin that
against definitions that do not use the DST: the 7-point residual written as
plain loops, a sparse direct solve of the assembled matrix, the involution of
the sine transform, and single-mode inputs whose eigenvalue the stencil fixes.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import dpm_oracle as O
from paper_1811_03557_gb300.workloads import random_field


def stencil_residual_loops(u, q, h, sigma):
    """(sigma - Lap_h) u - q evaluated node by node with explicit neighbours."""
    N = u.shape[0]
    r = np.zeros_like(u)

    def val(i, j, k):
        if 0 <= i < N and 0 <= j < N and 0 <= k < N:
            return u[i, j, k]
        return 0.0  # ghost node: zero Dirichlet data

    for i, j, k in itertools.product(range(N), repeat=3):
        nb = (val(i + 1, j, k) + val(i - 1, j, k) + val(i, j + 1, k) + val(i, j - 1, k)
              + val(i, j, k + 1) + val(i, j, k - 1))
        lap = (nb - 6.0 * u[i, j, k]) / (h * h)
        r[i, j, k] = sigma * u[i, j, k] - lap - q[i, j, k]
    return r


def sparse_operator(N, h, sigma):
    T = sp.diags([-np.ones(N - 1), 2 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1]) / (h * h)
    I = sp.identity(N)
    return (sigma * sp.identity(N ** 3) + sp.kron(sp.kron(T, I), I) + sp.kron(sp.kron(I, T), I)
            + sp.kron(sp.kron(I, I), T)).tocsc()


@pytest.mark.parametrize("N", [1, 2, 5, 8])
def test_dst_is_an_involution_up_to_scale(N):
    S = O.dst1_matrix(N)
    assert np.allclose(S @ S, (N + 1) / 2 * np.eye(N), atol=1e-12)


@pytest.mark.parametrize("N,h,sigma", [(6, 0.3, 2.0), (7, 0.11, 1001.0), (9, 1.0, 0.0)])
def test_residual_of_the_7_point_operator(N, h, sigma):
    q = random_field(1, (N, N, N), -1, 1)
    u = O.aux_solve(q, h, sigma)
    r = stencil_residual_loops(u, q, h, sigma)
    assert np.max(np.abs(r)) < 1e-11 * max(1.0, np.max(np.abs(q)))


@pytest.mark.parametrize("N,h,sigma", [(10, 0.2, 5.0), (11, 0.05, 4e4)])
def test_matches_sparse_direct_solve(N, h, sigma):
    q = random_field(2, (N, N, N), -1, 1)
    ref = spla.spsolve(sparse_operator(N, h, sigma), q.reshape(-1)).reshape(N, N, N)
    u = O.aux_solve(q, h, sigma)
    assert np.max(np.abs(u - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("abc", [(1, 1, 1), (2, 5, 3), (7, 1, 4)])
def test_single_mode_eigenvalue(abc):
    N, h, sigma = 7, 0.25, 3.0
    idx = np.arange(1, N + 1)
    a, b, c = abc
    mode = (np.sin(np.pi * a * idx / (N + 1))[:, None, None]
            * np.sin(np.pi * b * idx / (N + 1))[None, :, None]
            * np.sin(np.pi * c * idx / (N + 1))[None, None, :])
    # eigenvalue fixed by the stencil: apply it once to the mode
    Lmode = O.apply_L(mode, h, sigma)
    lam = np.sum(Lmode * mode) / np.sum(mode * mode)
    assert np.allclose(Lmode, lam * mode, atol=1e-9 * abs(lam))
    lam_tab = O.ap_eigenvalues(N, h, sigma)[a - 1, b - 1, c - 1]
    assert lam_tab == pytest.approx(lam, rel=1e-13)
    assert np.allclose(O.aux_solve(mode, h, sigma), mode / lam, atol=1e-13)


def test_apply_L_matches_sparse_matrix():
    N, h, sigma = 6, 0.4, 1.5
    v = random_field(3, (N, N, N), -1, 1)
    ref = (sparse_operator(N, h, sigma) @ v.reshape(-1)).reshape(N, N, N)
    assert np.allclose(O.apply_L(v, h, sigma), ref, atol=1e-12)


def test_linearity_and_batch_independence():
    N, h, sigma = 8, 0.2, 7.0
    q1 = random_field(4, (N, N, N), -1, 1)
    q2 = random_field(5, (N, N, N), -1, 1)
    u = O.aux_solve(2.0 * q1 - 3.0 * q2, h, sigma)
    assert np.allclose(u, 2.0 * O.aux_solve(q1, h, sigma) - 3.0 * O.aux_solve(q2, h, sigma), atol=1e-12)
