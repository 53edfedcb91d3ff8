"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no step of the Difference Potentials Method: it only produces
input data (random right-hand sides, the analytic initial conditions and the
manufactured exact solution) and the named workload shapes.  Both the CUDA path
and the CPU oracle receive the same arrays from here and evaluate the method
themselves.

The paper's workloads are analytic initial data, not a dataset: Test (A) and
Test (B) of Section 4 are Gaussians of the form amp * exp(-alpha * (x^2 + y^2 +
b (z - z0)^2)) (Section 4, "Initial Conditions", and Remark 2.3 (i)).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Gaussian:
    """amp * exp(-alpha * ((x-x0)^2 + (y-y0)^2 + zscale*(z-z0)^2))."""

    amp: float
    alpha: float
    center: tuple = (0.0, 0.0, 0.0)
    zscale: float = 1.0

    def __call__(self, x, y, z):
        x0, y0, z0 = self.center
        r2 = (x - x0) ** 2 + (y - y0) ** 2 + self.zscale * (z - z0) ** 2
        return self.amp * np.exp(-self.alpha * r2)


# Section 4, Test (A): blow-up at the centre.
TEST_A_RHO0 = Gaussian(1000.0, 100.0)
TEST_A_C0 = Gaussian(500.0, 50.0)
# Section 4, Test (B): blow-up at the boundary (c0 = 0).
TEST_B_RHO0 = Gaussian(2000.0, 100.0, (0.0, 0.0, 0.25))
TEST_B_C0 = Gaussian(0.0, 1.0)
# Off-centre seed of the N=128 PKS workload.
OFFC_RHO0 = Gaussian(1200.0, 120.0, (0.3, 0.0, 0.0))
OFFC_C0 = Gaussian(600.0, 60.0, (0.3, 0.0, 0.0))


def manufactured_u(x, y, z):
    """Exact solution u = exp(x) sin(y) cos(z); Lap u = -u."""
    return np.exp(x) * np.sin(y) * np.cos(z)


def manufactured_grad(x, y, z):
    """Gradient of manufactured_u, stacked on the last axis."""
    ex = np.exp(x)
    return np.stack(
        [ex * np.sin(y) * np.cos(z), ex * np.cos(y) * np.cos(z), -ex * np.sin(y) * np.sin(z)],
        axis=-1,
    )


def random_rhs(seed: int, B: int, N: int, dtype=np.float32) -> np.ndarray:
    """B dense right-hand sides, uniform in [-1, 1], shape (B, N, N, N)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(B, N, N, N)).astype(dtype)


def random_field(seed: int, shape, lo=0.0, hi=1.0, dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape).astype(dtype)


@dataclass(frozen=True)
class Geometry:
    """kind 0 = sphere (axes all equal the radius), 1 = ellipsoid."""

    kind: int
    center: tuple
    axes: tuple

    @staticmethod
    def sphere(r, center=(0.0, 0.0, 0.0)):
        return Geometry(0, tuple(center), (r, r, r))

    @staticmethod
    def ellipsoid(a, b, c, center=(0.0, 0.0, 0.0)):
        return Geometry(1, tuple(center), (a, b, c))


@dataclass(frozen=True)
class Workload:
    name: str
    geom: Geometry
    N: int
    lo: float
    hi: float
    K: int
    beta: int = 1
    sigma: float | None = None       # elliptic / BEP batch shift
    dt: float | None = None          # PKS dt_max
    steps: int = 0
    rho0: Gaussian | None = None
    c0: Gaussian | None = None
    extra: dict = field(default_factory=dict)

    @property
    def h(self):
        return (self.hi - self.lo) / (self.N + 1)

    @property
    def ncol(self):
        return (self.beta + 1) * (self.K + 1) ** 2


def _cfg_pks128() -> Workload:
    N, lo, hi = 128, -1.25, 1.25
    h = (hi - lo) / (N + 1)
    return Workload("pks_sphere_N128_K8", Geometry.sphere(1.0), N, lo, hi, K=8,
                    dt=h * h / 4.0, steps=500, rho0=OFFC_RHO0, c0=OFFC_C0)


# Named workloads (sizes as the paper-shaped benchmark configurations state them).
WORKLOADS = {
    "elliptic_sphere_N32_K4": Workload(
        "elliptic_sphere_N32_K4", Geometry.sphere(1.0), 32, -1.25, 1.25, K=4,
        sigma=1.0 / 1e-3 + 1.0, dt=1e-3, steps=10, rho0=TEST_A_RHO0, c0=TEST_A_C0),
    "pks_sphere_N128_K8": _cfg_pks128(),
    "bep_ellipsoid_N256_K12": Workload(
        "bep_ellipsoid_N256_K12", Geometry.ellipsoid(1.0, 0.8, 0.6), 256, -1.2, 1.2, K=12,
        sigma=1.0 / 1e-4 + 1.0),
}


@dataclass(frozen=True)
class ServingModel:
    """One resident factorisation of the request stream: an elliptic problem
    (sigma - Lap) u = f in the body `geom`, on an N^3 grid of the box
    [lo, hi]^3, with degree-K harmonics on the boundary."""

    geom: Geometry
    N: int
    lo: float
    hi: float
    K: int
    sigma: float
    beta: int = 1

    @property
    def ncol(self):
        return (self.beta + 1) * (self.K + 1) ** 2


@dataclass(frozen=True)
class PksRunModel:
    """A short PKS run: Test (A) data on the unit sphere, `steps` steps with the
    CFL-limited step size (dt_max = h^2/4)."""

    N: int
    K: int
    steps: int
    lo: float = -1.25
    hi: float = 1.25

    @property
    def geom(self):
        return Geometry.sphere(1.0)

    @property
    def dt_max(self):
        h = (self.hi - self.lo) / (self.N + 1)
        return h * h / 4.0


def serving_catalog(seed: int, n_models: int, Ns=(32, 64, 128, 256), K_range=(4, 12),
                    sigma_range=(1e2, 1e5), radius_range=(0.5, 1.0)) -> list:
    """n_models elliptic problems drawn from the serving mix: N uniform over Ns,
    K uniform in K_range, sigma log-uniform in sigma_range, sphere or
    ellipsoid (equal odds) with largest semi-axis uniform in radius_range; the
    box is [-1.25 r, 1.25 r]^3."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_models):
        N = int(rng.choice(np.asarray(Ns)))
        K = int(rng.integers(K_range[0], K_range[1] + 1))
        sigma = float(10.0 ** rng.uniform(np.log10(sigma_range[0]), np.log10(sigma_range[1])))
        r = float(rng.uniform(*radius_range))
        if rng.integers(0, 2):
            g = Geometry.ellipsoid(r, r * float(rng.uniform(0.7, 1.0)), r * float(rng.uniform(0.6, 1.0)))
        else:
            g = Geometry.sphere(r)
        out.append(ServingModel(g, N, -1.25 * r, 1.25 * r, K, sigma))
    return out


def poly_gauss_coeffs(seed: int):
    """Coefficients of a random polynomial of degree <= 3 (c[a, b, c] for
    x^a y^b z^c, zero when a + b + c > 3) and a Gaussian width in [0.5, 3]."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1.0, 1.0, size=(4, 4, 4))
    a, b, d = np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij")
    c[a + b + d > 3] = 0.0
    return c, float(rng.uniform(0.5, 3.0))


def poly_gauss_rhs(seed: int, model, dtype=np.float32) -> np.ndarray:
    """f = p(x/r, y/r, z/r) * exp(-w |x/r|^2) on the model's N^3 grid (r the
    largest semi-axis), for the coefficients poly_gauss_coeffs(seed)."""
    c, w = poly_gauss_coeffs(seed)
    N = model.N
    r = max(model.geom.axes)
    h = (model.hi - model.lo) / (N + 1)
    x = (model.lo + h * np.arange(1, N + 1) - 0.0) / r
    cx, cy, cz = (np.asarray(model.geom.center, dtype=np.float64) / r)
    X = np.stack([(x - cx) ** a * np.exp(-w * (x - cx) ** 2) for a in range(4)], axis=1)
    Y = np.stack([(x - cy) ** a * np.exp(-w * (x - cy) ** 2) for a in range(4)], axis=1)
    Z = np.stack([(x - cz) ** a * np.exp(-w * (x - cz) ** 2) for a in range(4)], axis=1)
    # separable sum over (a, b, c): three small contractions, the last a matmul
    T = np.einsum("abc,kc->abk", c, Z)
    T = np.einsum("abk,jb->ajk", T, Y)
    f = X @ T.reshape(4, N * N)
    return f.reshape(N, N, N).astype(dtype)


@dataclass(frozen=True)
class ServingRequest:
    """Arrival time (s from the start of the stream), what is asked, and the
    seed of its right-hand side (elliptic) or the run (PKS)."""

    t: float
    kind: str          # "solve" or "pks"
    model: int         # index into the elliptic catalog or the PKS catalog
    rhs_seed: int


def serving_stream(seed: int, n: int, rate_hz: float, n_models: int, n_pks_models: int = 0,
                   pks_fraction: float = 0.0, rhs_pool: int = 2) -> list:
    """Poisson arrivals at rate_hz; each request picks a catalog entry uniformly
    and one of `rhs_pool` right-hand sides of that entry."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    out = []
    for i in range(n):
        if n_pks_models and rng.uniform() < pks_fraction:
            out.append(ServingRequest(float(t[i]), "pks", int(rng.integers(0, n_pks_models)), 0))
        else:
            m = int(rng.integers(0, n_models))
            out.append(ServingRequest(float(t[i]), "solve", m, m * 1000 + int(rng.integers(0, rhs_pool))))
    return out


def pks_run_catalog(seed: int, n_models: int, Ns=(32, 64, 128), K_range=(4, 8), steps=10) -> list:
    rng = np.random.default_rng(seed)
    return [PksRunModel(int(rng.choice(np.asarray(Ns))), int(rng.integers(K_range[0], K_range[1] + 1)),
                        steps) for _ in range(n_models)]


__all__ = [
    "Gaussian", "Geometry", "Workload", "WORKLOADS", "TEST_A_RHO0", "TEST_A_C0",
    "TEST_B_RHO0", "TEST_B_C0", "OFFC_RHO0", "OFFC_C0", "manufactured_u",
    "manufactured_grad", "random_rhs", "random_field", "ServingModel", "PksRunModel",
    "serving_catalog", "poly_gauss_coeffs", "poly_gauss_rhs", "ServingRequest", "serving_stream",
    "pks_run_catalog",
]
