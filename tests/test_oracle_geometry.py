"""Pins of the oracle's orthogonal projection on Gamma (Definition 2.6).

Sphere: closed form.  Ellipsoid: the optimality conditions of the closest
point (on the surface, p - x' parallel to the normal), brute-force distance
minimisation over a dense surface sample, the sphere limit, and the closed
forms on the principal axes (outside: the vertex; inside on the shortest axis:
its vertex)."""
import numpy as np
import pytest

from oracle import dpm_oracle as O
from paper_1811_03557_gb300.workloads import Geometry


def test_sphere_closed_form():
    g = Geometry.sphere(0.8, (0.1, 0.2, -0.1))
    rng = np.random.default_rng(0)
    P = rng.uniform(-1.2, 1.2, (200, 3))
    xf, d, n = O.foot_point(g, P)
    c = np.array(g.center)
    r = np.linalg.norm(P - c, axis=1)
    assert np.allclose(d, r - 0.8)
    assert np.allclose(np.linalg.norm(xf - c, axis=1), 0.8)
    assert np.allclose(P, xf + d[:, None] * n)


def test_ellipsoid_as_sphere_limit():
    rng = np.random.default_rng(1)
    P = rng.uniform(-1.5, 1.5, (100, 3))
    a = O.foot_point(Geometry.sphere(1.0), P)
    b = O.foot_point(Geometry.ellipsoid(1.0, 1.0, 1.0), P)
    for u, v in zip(a, b):
        assert np.allclose(u, v, atol=1e-12)


def test_ellipsoid_optimality_and_brute_force():
    g = Geometry.ellipsoid(1.0, 0.8, 0.6)
    rng = np.random.default_rng(2)
    # points in a shell around Gamma, as the nodes of gamma are
    dirs = rng.normal(size=(60, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    base = dirs * np.array(g.axes) / np.linalg.norm(dirs / np.array(g.axes), axis=1)[:, None]
    P = base + rng.uniform(-0.05, 0.05, (60, 1)) * dirs
    xf, d, n = O.foot_point(g, P)
    F = O.ellipsoid_form(g, xf[:, 0], xf[:, 1], xf[:, 2])
    assert np.allclose(F, 1.0, atol=1e-13)
    assert np.allclose(P, xf + d[:, None] * n, atol=1e-12)
    inside = O.ellipsoid_form(g, P[:, 0], P[:, 1], P[:, 2]) < 1
    assert np.all((d < 0) == inside)
    # brute force: minimum distance over a fine parametric sample
    t = np.linspace(0, np.pi, 721)
    p = np.linspace(-np.pi, np.pi, 1441)
    T, PH = np.meshgrid(t, p, indexing="ij")
    S = np.stack([np.sin(T) * np.cos(PH), np.sin(T) * np.sin(PH), np.cos(T)], -1).reshape(-1, 3)
    S = S * np.array(g.axes)
    for k in range(0, 60, 6):
        dmin = np.min(np.linalg.norm(S - P[k], axis=1))
        assert abs(d[k]) <= dmin + 1e-12
        assert abs(d[k]) >= dmin - 5e-5


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_ellipsoid_axis_points_outside(axis):
    """A point on a principal axis beyond the vertex projects onto the vertex:
    x' = c +- a_i e_i, d = |t| - a_i, n = +-e_i (closed form)."""
    g = Geometry.ellipsoid(1.0, 0.8, 0.6, (0.1, -0.2, 0.05))
    c, a = np.array(g.center), np.array(g.axes)
    e = np.eye(3)[axis]
    t = np.array([a[axis] + 0.01, a[axis] + 0.3, -(a[axis] + 0.07), -(a[axis] + 1.0)])
    P = c + t[:, None] * e
    xf, d, n = O.foot_point(g, P)
    sgn = np.sign(t)
    assert np.allclose(xf, c + (sgn * a[axis])[:, None] * e, atol=1e-13)
    assert np.allclose(d, np.abs(t) - a[axis], atol=1e-13)
    assert np.allclose(n, sgn[:, None] * e, atol=1e-13)


def test_ellipsoid_shortest_axis_points_inside():
    """Inside, on the shortest axis, the nearest surface point is that axis's
    vertex (the other vertices and every off-axis point are farther):
    d = |t| - a_min < 0."""
    g = Geometry.ellipsoid(1.0, 0.8, 0.6)
    t = np.array([0.55, 0.3, 0.05, -0.2, -0.59])
    P = np.zeros((len(t), 3))
    P[:, 2] = t
    xf, d, n = O.foot_point(g, P)
    sgn = np.sign(t)
    assert np.allclose(xf, np.stack([0 * t, 0 * t, 0.6 * sgn], 1), atol=1e-12)
    assert np.allclose(d, np.abs(t) - 0.6, atol=1e-12)
    assert np.allclose(n[:, 2], sgn, atol=1e-12)
