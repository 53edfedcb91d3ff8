"""Pin of the whole elliptic DPM oracle: second-order convergence to a
manufactured exact solution (Proposition 2.7 conjectures O(h^2) in space).

u = exp(x) sin(y) cos(z) has Lap u = -u, so (sigma - Lap) u = (sigma + 1) u;
its Neumann data du/dn is evaluated at the foot points.  A dropped term, a
wrong sign or index anywhere in the AP, the point sets, the basis, the BEP,
the least squares or the Green's formula destroys the rate.
"""
import numpy as np
import pytest

from oracle import dpm_oracle as O
from paper_1811_03557_gb300.workloads import Geometry, manufactured_grad, manufactured_u


def solve_error(N, K=8, sigma=1.0, lo=-1.25, hi=1.25):
    s = O.DPMSetup(Geometry.sphere(1.0), N, lo, hi, K, 1, sigma)
    X, Y, Z = O.mesh(N, lo, hi)
    uex = manufactured_u(X, Y, Z)
    gn = np.sum(manufactured_grad(s.xf[:, 0], s.xf[:, 1], s.xf[:, 2]) * s.normal, axis=1)
    u, C, ug = O.dpm_elliptic_solve(s, (sigma + 1.0) * uex, gn)
    return float(np.max(np.abs(np.where(s.sets["Mp"], u - uex, 0.0))))


def test_second_order_in_space():
    Ns = (24, 32, 48)
    errs = [solve_error(N) for N in Ns]
    rates = [np.log(errs[i] / errs[i + 1]) / np.log((Ns[i + 1] + 1) / (Ns[i] + 1)) for i in range(2)]
    assert all(r > 1.6 for r in rates), (errs, rates)
    assert errs[-1] < 3e-4


def test_exact_for_discrete_solution_of_the_extension():
    """If the data are a combination of the basis densities the LSQ residual is
    zero and Green's formula returns the difference-equation solution."""
    s = O.DPMSetup(Geometry.sphere(1.0), 20, -1.3, 1.3, 2, 1, 5.0)
    Cwant = np.random.default_rng(0).normal(size=s.ncol)
    ug = s.extend(Cwant)
    # build f so that u = P u_gamma + G f with u solving the BEP exactly: take f = 0
    b = s.i_minus_p_gin(ug)                  # A @ Cwant
    C = s.lstsq(b)
    assert np.allclose(C, Cwant, atol=1e-8)
