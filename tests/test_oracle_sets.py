"""Pins of the oracle's point sets (Definition 2.1).

A brute-force construction with Python sets of index triples, written
directly from the definition (unions of 7-point stencils, intersections),
must equal the oracle's array version node for node.
"""
import itertools

import numpy as np
import pytest

from oracle import dpm_oracle as O
from paper_1811_03557_gb300.workloads import Geometry


def brute_force_sets(inside):
    N = inside.shape[0]
    M0 = set(itertools.product(range(N), repeat=3))
    Mp = {p for p in M0 if inside[p]}
    Mm = M0 - Mp

    def stencil(p):
        i, j, k = p
        return {(i, j, k), (i + 1, j, k), (i - 1, j, k), (i, j + 1, k), (i, j - 1, k),
                (i, j, k + 1), (i, j, k - 1)}

    Np = set().union(*[stencil(p) for p in Mp]) if Mp else set()
    Nm = set().union(*[stencil(p) for p in Mm]) if Mm else set()
    gamma = Np & Nm
    return dict(Mp=Mp, Mm=Mm, Np=Np, Nm=Nm, gamma=gamma, gin=Mp & gamma, gex=Mm & gamma)


GEOMS = [
    (Geometry.sphere(1.0), 9, -1.6, 1.6),
    (Geometry.sphere(0.7, (0.1, -0.05, 0.2)), 11, -1.2, 1.2),
    (Geometry.ellipsoid(1.0, 0.8, 0.6), 12, -1.3, 1.3),
    (Geometry.sphere(1.0), 6, -1.05, 1.05),     # domain touching the ghost layer
]


@pytest.mark.parametrize("geom,N,lo,hi", GEOMS)
def test_sets_equal_brute_force(geom, N, lo, hi):
    inside = O.inside_mask(geom, N, lo, hi)
    bf = brute_force_sets(inside)
    arr = O.point_sets(inside)
    for name in ("Mp", "Mm", "gamma", "gin", "gex"):
        got = {tuple(int(v) for v in p) for p in np.argwhere(arr[name])}
        want = {p for p in bf[name] if all(0 <= c < N for c in p)}
        assert got == want, name
    for name in ("Np", "Nm"):
        got = {tuple(int(v) for v in p) for p in np.argwhere(arr[name])}
        want = {p for p in bf[name] if all(0 <= c < N for c in p)}
        assert got == want, name


def test_gamma_in_is_mplus_with_mminus_neighbour():
    geom, N, lo, hi = Geometry.ellipsoid(1.0, 0.8, 0.6), 20, -1.3, 1.3
    lab, gin, gex = O.classify(geom, N, lo, hi)
    Mp = (lab & O.LBL_MPLUS) > 0
    pad = np.pad(Mp, 1, constant_values=False)
    padm = np.pad(~Mp, 1, constant_values=False)
    nb_minus = np.zeros_like(Mp)
    nb_plus = np.zeros_like(Mp)
    for ax in range(3):
        for s in (1, -1):
            nb_minus |= np.roll(padm, s, axis=ax)[1:-1, 1:-1, 1:-1]
            nb_plus |= np.roll(pad, s, axis=ax)[1:-1, 1:-1, 1:-1]
    assert set(gin) == set(np.flatnonzero(Mp & nb_minus))
    assert set(gex) == set(np.flatnonzero(~Mp & nb_plus))
    assert np.all(np.diff(gin) > 0) and np.all(np.diff(gex) > 0)


def test_sphere_counts_have_cube_symmetry():
    N, lo, hi = 24, -1.25, 1.25
    lab, _, _ = O.classify(Geometry.sphere(1.0), N, lo, hi)
    for perm in [(1, 0, 2), (2, 1, 0), (0, 2, 1)]:
        assert np.array_equal(lab, lab.transpose(perm))
    for ax in range(3):
        assert np.array_equal(lab, np.flip(lab, axis=ax))


def test_margin_detection():
    lab, _, _ = O.classify(Geometry.sphere(1.0), 6, -1.05, 1.05)
    assert not O.margin_ok(lab)
    lab, _, _ = O.classify(Geometry.sphere(1.0), 32, -1.25, 1.25)
    assert O.margin_ok(lab)
