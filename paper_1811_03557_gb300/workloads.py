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


def serving_requests(seed: int, n: int, rate_hz: float = 2000.0):
    """Poisson-arrival stream of elliptic-solve requests (shapes only)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    out = []
    for i in range(n):
        N = int(rng.choice([32, 64, 128, 256]))
        K = int(rng.integers(4, 13))
        sigma = float(10.0 ** rng.uniform(2.0, 5.0))
        r = float(rng.uniform(0.5, 1.0))
        ell = bool(rng.integers(0, 2))
        if ell:
            ax = (r, r * float(rng.uniform(0.7, 1.0)), r * float(rng.uniform(0.6, 1.0)))
        else:
            ax = (r, r, r)
        half = 1.25 * r * (N + 1) / max(N - 5, 1) if N > 8 else 1.5 * r
        out.append(dict(t=float(t[i]), N=N, K=K, sigma=sigma,
                        geom=Geometry(1 if ell else 0, (0.0, 0.0, 0.0), ax),
                        lo=-half, hi=half,
                        poly=rng.uniform(-1, 1, size=20).tolist(),
                        gauss=float(rng.uniform(0.5, 3.0))))
    return out


__all__ = [
    "Gaussian", "Geometry", "Workload", "WORKLOADS", "TEST_A_RHO0", "TEST_A_C0",
    "TEST_B_RHO0", "TEST_B_C0", "OFFC_RHO0", "OFFC_C0", "manufactured_u",
    "manufactured_grad", "random_rhs", "random_field", "serving_requests",
]
