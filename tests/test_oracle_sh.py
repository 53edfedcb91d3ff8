"""Pins of the oracle's real spherical harmonics (eq. spectral_approximation_sd).

Checked against scipy.special.sph_harm_y (an independent library routine,
complex convention with the Condon-Shortley phase), against closed forms of
low degree, and against orthonormality by Gauss-Legendre x trapezoid quadrature.
"""
import math

import numpy as np
import pytest

from oracle import dpm_oracle as O

K = 12


def test_closed_forms():
    ct = np.array([0.3, -0.7, 1.0, 0.0])
    ph = np.array([0.2, 2.5, 0.0, -1.1])
    Y = O.real_sph_harm(2, ct, ph)
    st = np.sqrt(1 - ct ** 2)
    assert np.allclose(Y[:, 0], 0.5 / math.sqrt(math.pi))
    assert np.allclose(Y[:, 2], math.sqrt(3 / (4 * math.pi)) * ct)            # l=1, m=0
    assert np.allclose(Y[:, 3], math.sqrt(3 / (4 * math.pi)) * st * np.cos(ph))  # l=1, m=1
    assert np.allclose(Y[:, 1], math.sqrt(3 / (4 * math.pi)) * st * np.sin(ph))  # l=1, m=-1
    assert np.allclose(Y[:, 6], math.sqrt(5 / (16 * math.pi)) * (3 * ct ** 2 - 1))  # l=2, m=0


def test_matches_scipy_complex_harmonics():
    sph = pytest.importorskip("scipy.special")
    if not hasattr(sph, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(0)
    theta = rng.uniform(0, np.pi, 50)
    phi = rng.uniform(-np.pi, np.pi, 50)
    Y = O.real_sph_harm(K, np.cos(theta), phi)
    for l in range(K + 1):
        for m in range(-l, l + 1):
            Yc = sph.sph_harm_y(l, abs(m), theta, phi)
            cs = (-1) ** abs(m)          # remove the Condon-Shortley phase
            if m == 0:
                ref = Yc.real
            elif m > 0:
                ref = math.sqrt(2) * cs * Yc.real
            else:
                ref = math.sqrt(2) * cs * Yc.imag
            assert np.allclose(Y[:, l * l + l + m], ref, atol=1e-12), (l, m)


def test_orthonormal_by_quadrature():
    nt, nph = 40, 60
    x, w = np.polynomial.legendre.leggauss(nt)
    ph = 2 * np.pi * np.arange(nph) / nph
    X, PH = np.meshgrid(x, ph, indexing="ij")
    W = np.repeat(w[:, None], nph, axis=1) * (2 * np.pi / nph)
    Y = O.real_sph_harm(K, X.reshape(-1), PH.reshape(-1))
    G = Y.T @ (W.reshape(-1)[:, None] * Y)
    assert np.allclose(G, np.eye((K + 1) ** 2), atol=1e-12)
