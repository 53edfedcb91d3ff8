"""Plain FP64 CPU oracle of the Difference Potentials Method hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this module.  The
product path (the CUDA library and its Python binding) never calls it, and this
module shares no code with it.

Every function restates one definition of Epshteyn & Xia, "Efficient Numerical
Algorithms based on Difference Potentials for Chemotaxis Systems in 3D"
(arXiv:1811.03557), in the paper's order and notation, using numpy in float64.
No blocking, fusion or reordering beyond what the definition states: the
auxiliary problem is the dense 3D DST-I written out with the explicit sine
matrix (a library matmul per axis), the point sets are the literal set unions
of Definition 2.1, and so on.

Readings where the paper is silent or ambiguous:
  * grid: N interior nodes per axis of the cube [lo, hi]^3, x_j = lo + j*h,
    j = 1..N, h = (hi - lo)/(N + 1); the Dirichlet ghost layer j = 0, N+1 is
    the set N^0 \\ M^0.
  * M^+ is the strict interior: F(x) < 1 with F the ellipsoid form evaluated
    in a fixed order, so nodes exactly on Gamma belong to M^-.
  * the AP operator is sigma - Lap_h; the paper's L_{h,dt} = I - dt Lap_h is
    dt*(sigma - Lap_h) with sigma = 1/dt, so the PKS right-hand side is f/dt.
  * basis: real orthonormal spherical harmonics without the Condon-Shortley
    phase, theta from +z and phi = atan2(y, x) of the foot point relative to
    the domain centre; column order nu = l^2 + l + m, then the (d^2/2) copies.
  * a minmod slope whose stencil leaves N^+ is 0.
  * after the extension the PKS densities are clamped at 0 (Theorem 2.4,
    condition 3).

Parity pins: every function here is checked by tests/test_oracle_*.py against
closed forms, brute force, library routines or the paper's theorems.  The
ellipsoid foot point is pinned by its optimality conditions (a stationary
point of the distance), the brute-force global minimum over a fine
parametric sample, the sphere limit and the closed forms on the principal
axes.
"""
from __future__ import annotations

import math

import numpy as np

# Label bits of a node (one uint8 per node of M^0).
LBL_MPLUS = 1     # x in M^+            (Definition 2.1)
LBL_GIN = 2       # x in gamma_in       (Definition 2.1)
LBL_GEX = 4       # x in gamma_ex       (Definition 2.1)


# ---------------------------------------------------------------------------
# Grid (Section 2, "Introduction of the Auxiliary Domain"; reading: node grid)
# ---------------------------------------------------------------------------
def grid_spacing(N: int, lo: float, hi: float) -> float:
    """h of the uniform mesh with N interior nodes per axis on [lo, hi]."""
    return (hi - lo) / (N + 1)


def node_coords(N: int, lo: float, hi: float) -> np.ndarray:
    """x_j = lo + j*h for j = 1..N (float64, evaluated as lo + (j*h))."""
    h = grid_spacing(N, lo, hi)
    j = np.arange(1, N + 1, dtype=np.float64)
    return lo + j * h


def mesh(N, lo, hi):
    x = node_coords(N, lo, hi)
    return np.meshgrid(x, x, x, indexing="ij")


# ---------------------------------------------------------------------------
# Point sets (Definition 2.1)
# ---------------------------------------------------------------------------
def ellipsoid_form(geom, X, Y, Z):
    """F = ((x-cx)/ax)^2 + ((y-cy)/ay)^2 + ((z-cz)/az)^2, summed as (Fx+Fy)+Fz."""
    (cx, cy, cz), (ax, ay, az) = geom.center, geom.axes
    tx = (X - cx) / ax
    ty = (Y - cy) / ay
    tz = (Z - cz) / az
    return (tx * tx + ty * ty) + tz * tz


def inside_mask(geom, N, lo, hi) -> np.ndarray:
    """Membership of each node of M^0 in the open domain Omega: F < 1 for a
    sphere or ellipsoid; for a spherical shell (kind 2, radii axes[0] > axes[1])
    F < 1 for the outer sphere and F > 1 for the inner one."""
    x = node_coords(N, lo, hi)
    X, Y, Z = x[:, None, None], x[None, :, None], x[None, None, :]
    if geom.kind == 2:
        c, (ro, ri, _) = geom.center, geom.axes
        outer = ellipsoid_form(_Sph(c, ro), X, Y, Z) < 1.0
        inner = ellipsoid_form(_Sph(c, ri), X, Y, Z) > 1.0
        return outer & inner
    if geom.kind in (3, 4):
        return _two_sphere_inside(geom, X, Y, Z)
    return ellipsoid_form(geom, X, Y, Z) < 1.0


class _Sph:
    """A sphere as the (centre, axes) pair ellipsoid_form reads."""

    def __init__(self, c, r):
        self.kind, self.center, self.axes = 0, tuple(c), (r, r, r)


def _stencil_union(S: np.ndarray) -> np.ndarray:
    """Union of the 7-point stencils (eq. stencil:7-point) centred at the nodes of S."""
    U = S.copy()
    for ax in range(3):
        U |= np.roll(S, 1, axis=ax) & _not_wrapped(S.shape, ax, +1)
        U |= np.roll(S, -1, axis=ax) & _not_wrapped(S.shape, ax, -1)
    return U


def _not_wrapped(shape, ax, s):
    m = np.ones(shape, dtype=bool)
    idx = [slice(None)] * 3
    idx[ax] = 0 if s > 0 else shape[ax] - 1
    m[tuple(idx)] = False
    return m


def point_sets(inside: np.ndarray) -> dict:
    """Definition 2.1 written out on the grid padded with the ghost layer N^0\\M^0.

    Returns boolean arrays (shape N^3) for M^+, M^-, N^+, N^-, gamma,
    gamma_in and gamma_ex (the ghost layer itself is cut off).
    """
    N = inside.shape[0]
    M0 = np.zeros((N + 2,) * 3, dtype=bool)
    M0[1:-1, 1:-1, 1:-1] = True
    In = np.zeros_like(M0)
    In[1:-1, 1:-1, 1:-1] = inside
    Mp = M0 & In
    Mm = M0 & ~In
    Np = _stencil_union(Mp)
    Nm = _stencil_union(Mm)
    gamma = Np & Nm
    gin = Mp & gamma
    gex = Mm & gamma
    core = (slice(1, -1),) * 3
    return dict(Mp=Mp[core], Mm=Mm[core], Np=Np[core], Nm=Nm[core], gamma=gamma[core],
                gin=gin[core], gex=gex[core])


def labels_from_sets(sets) -> np.ndarray:
    lab = np.zeros(sets["Mp"].shape, dtype=np.uint8)
    lab[sets["Mp"]] |= LBL_MPLUS
    lab[sets["gin"]] |= LBL_GIN
    lab[sets["gex"]] |= LBL_GEX
    return lab


def classify(geom, N, lo, hi):
    """Labels and the ascending linear-index lists of gamma_in and gamma_ex."""
    sets = point_sets(inside_mask(geom, N, lo, hi))
    lab = labels_from_sets(sets)
    flat = lab.reshape(-1)
    gin = np.flatnonzero(flat & LBL_GIN).astype(np.int64)
    gex = np.flatnonzero(flat & LBL_GEX).astype(np.int64)
    return lab, gin, gex


def margin_ok(lab: np.ndarray, margin: int = 2) -> bool:
    """True when no node of M^+ lies within ``margin`` nodes of a cube face."""
    idx = np.argwhere(lab & LBL_MPLUS)
    if idx.size == 0:
        return False
    N = lab.shape[0]
    return bool(idx.min() >= margin and idx.max() <= N - 1 - margin)


# ---------------------------------------------------------------------------
# Orthogonal projection on Gamma, signed distance, normal (Definition 2.6)
# ---------------------------------------------------------------------------
def foot_point(geom, P: np.ndarray, tol: float = 1e-15, maxit: int = 200):
    """Closest point x' on Gamma to each row of P, the signed distance d (> 0
    outside Omega, along the outward normal) and the unit outward normal at x'.

    Sphere: x' = c + r (p-c)/|p-c|, d = |p-c| - r.
    Ellipsoid: x'_i = c_i + (p_i-c_i) a_i^2/(a_i^2 + mu), with mu the root in
    (-min a_i^2, inf) of sum (p_i-c_i)^2 a_i^2/(a_i^2+mu)^2 = 1, found by plain
    bisection (slow, monotone, no starting-guess logic).
    """
    P = np.asarray(P, dtype=np.float64)
    c = np.asarray(geom.center, dtype=np.float64)
    a = np.asarray(geom.axes, dtype=np.float64)
    q = P - c
    if geom.kind == 2:
        # spherical shell: the nearer of the two spheres; normal (x - c)/|x - c| and
        # d = |x - c| - r on both (outward from the centre, also on the inner sphere)
        rho = np.linalg.norm(q, axis=1)
        n = q / rho[:, None]
        r = np.where(np.abs(rho - a[0]) <= np.abs(rho - a[1]), a[0], a[1])
        return c + r[:, None] * n, rho - r, n
    if geom.kind == 0:
        r = a[0]
        rho = np.linalg.norm(q, axis=1)
        n = q / rho[:, None]
        xf = c + r * n
        return xf, rho - r, n
    a2 = a * a

    def F(mu):
        return np.sum(q * q * a2 / (a2 + mu[:, None]) ** 2, axis=1) - 1.0

    lo = np.full(len(P), -a2.min() * (1 - 1e-15))
    hi = np.full(len(P), 1.0)
    while np.any(F(hi) > 0):
        hi = np.where(F(hi) > 0, 2 * hi + 1.0, hi)
    # F is decreasing on (-min a^2, inf): bisection to full double precision.
    for _ in range(maxit):
        mid = 0.5 * (lo + hi)
        pos = F(mid) > 0
        lo = np.where(pos, mid, lo)
        hi = np.where(pos, hi, mid)
        if np.all(hi - lo <= tol * np.maximum(1.0, np.abs(mid))):
            break
    mu = 0.5 * (lo + hi)
    xf = c + q * a2 / (a2 + mu[:, None])
    g = (xf - c) / a2
    n = g / np.linalg.norm(g, axis=1)[:, None]
    outside = np.sum(q * q / a2, axis=1) > 1.0
    d = np.linalg.norm(P - xf, axis=1) * np.where(outside, 1.0, -1.0)
    return xf, d, n


# ---------------------------------------------------------------------------
# Spherical harmonics (eq. spectral_approximation_sd)
# ---------------------------------------------------------------------------
def assoc_legendre(K: int, x: np.ndarray) -> np.ndarray:
    """P_l^m(x) for 0 <= m <= l <= K without the Condon-Shortley phase, by the
    textbook three-term recurrence in l.  Returns shape (K+1, K+1, len(x))."""
    x = np.asarray(x, dtype=np.float64)
    P = np.zeros((K + 1, K + 1) + x.shape)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    for m in range(K + 1):
        # P_m^m = (2m-1)!! (1-x^2)^{m/2}
        dfact = 1.0
        for k in range(1, 2 * m, 2):
            dfact *= k
        P[m, m] = dfact * s ** m
        if m + 1 <= K:
            P[m + 1, m] = x * (2 * m + 1) * P[m, m]
        for l in range(m + 2, K + 1):
            P[l, m] = ((2 * l - 1) * x * P[l - 1, m] - (l + m - 1) * P[l - 2, m]) / (l - m)
    return P


def real_sph_harm(K: int, cos_theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonics phi_nu, nu = l^2 + l + m, for
    l <= K, -l <= m <= l.  Returns shape (n_points, (K+1)^2).

    Y_l0 = N_l0 P_l^0, Y_lm = sqrt(2) N_lm P_l^m cos(m phi) (m > 0),
    Y_l,-m = sqrt(2) N_lm P_l^m sin(m phi), N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).
    """
    P = assoc_legendre(K, cos_theta)
    out = np.zeros((len(cos_theta), (K + 1) ** 2))
    for l in range(K + 1):
        for m in range(0, l + 1):
            Nlm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
            if m == 0:
                out[:, l * l + l] = Nlm * P[l, 0]
            else:
                out[:, l * l + l + m] = math.sqrt(2.0) * Nlm * P[l, m] * np.cos(m * phi)
                out[:, l * l + l - m] = math.sqrt(2.0) * Nlm * P[l, m] * np.sin(m * phi)
    return out


def boundary_basis(geom, xf: np.ndarray, K: int) -> np.ndarray:
    """phi_nu(theta, phi) at foot points xf (angles relative to the centre)."""
    q = xf - np.asarray(geom.center)
    rad = np.linalg.norm(q, axis=1)
    cos_t = q[:, 2] / rad
    ph = np.arctan2(q[:, 1], q[:, 0])
    return real_sph_harm(K, cos_t, ph)


# ---------------------------------------------------------------------------
# The Auxiliary Problem (Definition 2.4): (sigma - Lap_h) v = q on M^0,
# v = 0 on N^0 \ M^0, diagonalised by the 3D DST-I.
# ---------------------------------------------------------------------------
def dst1_matrix(N: int) -> np.ndarray:
    """S[a, m] = sin(pi a m / (N+1)), a, m = 1..N."""
    a = np.arange(1, N + 1, dtype=np.float64)
    return np.sin(np.pi * np.outer(a, a) / (N + 1))


def ap_eigenvalues(N: int, h: float, sigma: float) -> np.ndarray:
    """lambda_abc = sigma + (4/h^2)(sin^2(pi a/2(N+1)) + sin^2(pi b/..) + sin^2(pi c/..))."""
    a = np.arange(1, N + 1, dtype=np.float64)
    s2 = np.sin(np.pi * a / (2 * (N + 1))) ** 2
    return sigma + (4.0 / (h * h)) * (s2[:, None, None] + s2[None, :, None] + s2[None, None, :])


def dst3(X: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Apply S along each of the three axes (one matmul per axis)."""
    Y = np.einsum("ai,ijk->ajk", S, X, optimize=True)
    Y = np.einsum("bj,ajk->abk", S, Y, optimize=True)
    return np.einsum("ck,abk->abc", S, Y, optimize=True)


def aux_solve(q: np.ndarray, h: float, sigma: float) -> np.ndarray:
    """Solve the AP for one right-hand side q (N^3 array on M^0).

    Forward DST-I on x, y, z; divide by lambda_abc; inverse DST-I (the same
    sine matrix times 2/(N+1) per axis)."""
    N = q.shape[0]
    S = dst1_matrix(N)
    qh = dst3(np.asarray(q, dtype=np.float64), S)
    uh = qh / ap_eigenvalues(N, h, sigma)
    return (2.0 / (N + 1)) ** 3 * dst3(uh, S)


def apply_L(v: np.ndarray, h: float, sigma: float) -> np.ndarray:
    """(sigma - Lap_h) v at every node of M^0 with v = 0 on the ghost layer
    (the 7-point operator of eq. discrete_chemotaxis, shifted form)."""
    vp = np.pad(np.asarray(v, dtype=np.float64), 1)
    c = vp[1:-1, 1:-1, 1:-1]
    nb = (vp[2:, 1:-1, 1:-1] + vp[:-2, 1:-1, 1:-1] + vp[1:-1, 2:, 1:-1] + vp[1:-1, :-2, 1:-1]
          + vp[1:-1, 1:-1, 2:] + vp[1:-1, 1:-1, :-2])
    return sigma * c - (nb - 6.0 * c) / (h * h)


# ---------------------------------------------------------------------------
# Particular solution, difference potential, trace (eqs. rhs:particular_solution,
# rhs:difference_potentials; Definition 2.5; trace operators)
# ---------------------------------------------------------------------------
def particular_solution(f, sets, h, sigma):
    """G f: AP with q = f on M^+, 0 on M^-; restricted to N^+ (zero elsewhere)."""
    q = np.where(sets["Mp"], f, 0.0)
    return np.where(sets["Np"], aux_solve(q, h, sigma), 0.0)


def gamma_density_grid(v_gamma, gamma_idx, N):
    """A density on gamma extended by zero to the whole grid."""
    g = np.zeros(N ** 3)
    g[gamma_idx] = v_gamma
    return g.reshape(N, N, N)


def difference_potential(vgrid, sets, h, sigma):
    """P_{N+gamma} v_gamma: AP with q = 0 on M^+, L[v_gamma] on M^-; on N^+."""
    q = np.where(sets["Mm"], apply_L(vgrid, h, sigma), 0.0)
    return np.where(sets["Np"], aux_solve(q, h, sigma), 0.0)


# ---------------------------------------------------------------------------
# DPM setup: gamma geometry, basis, BEP matrix (eq. BEP_recast), QR
# ---------------------------------------------------------------------------
class DPMSetup:
    """Everything of Steps 1-2 that depends only on (geometry, grid, K, beta, sigma)."""

    def __init__(self, geom, N, lo, hi, K, beta, sigma, build_bep=True):
        self.geom, self.N, self.lo, self.hi = geom, N, lo, hi
        self.K, self.beta, self.sigma = K, beta, sigma
        self.h = grid_spacing(N, lo, hi)
        self.sets = point_sets(inside_mask(geom, N, lo, hi))
        self.labels = labels_from_sets(self.sets)
        flat_gamma = self.sets["gamma"].reshape(-1)
        self.gamma_idx = np.flatnonzero(flat_gamma)                 # ascending
        self.gin_idx = np.flatnonzero(self.sets["gin"].reshape(-1))
        self.gex_idx = np.flatnonzero(self.sets["gex"].reshape(-1))
        # positions of gamma_in inside the gamma list
        self.gin_pos = np.searchsorted(self.gamma_idx, self.gin_idx)
        X, Y, Z = mesh(N, lo, hi)
        self.P = np.stack([X.reshape(-1)[self.gamma_idx], Y.reshape(-1)[self.gamma_idx],
                           Z.reshape(-1)[self.gamma_idx]], axis=1)
        self.xf, self.d, self.normal = foot_point(geom, self.P)
        self.phi = boundary_basis(geom, self.xf, K)                    # |gamma| x (K+1)^2
        self.nsh = (K + 1) ** 2
        self.ncol = (beta + 1) * self.nsh
        if build_bep:
            self.A = self.bep_matrix()
            self.Q, self.R = np.linalg.qr(self.A)

    def basis_densities(self) -> np.ndarray:
        """Columns psi_k on gamma: phi_nu, then beta * (d^2/2) phi_nu (eq. extension_operator_recast)."""
        cols = [self.phi]
        if self.beta:
            cols.append(0.5 * self.d[:, None] ** 2 * self.phi)
        return np.concatenate(cols, axis=1)

    def i_minus_p_gin(self, v_gamma) -> np.ndarray:
        """Tr_{gamma_in} (v_gamma - P_{N+gamma} v_gamma)."""
        vg = gamma_density_grid(v_gamma, self.gamma_idx, self.N)
        Pv = difference_potential(vg, self.sets, self.h, self.sigma)
        return v_gamma[self.gin_pos] - Pv.reshape(-1)[self.gin_idx]

    def bep_matrix(self) -> np.ndarray:
        """|gamma_in| x ncol matrix of eq. BEP_recast, one AP per column (Step 2)."""
        Psi = self.basis_densities()
        return np.stack([self.i_minus_p_gin(Psi[:, k]) for k in range(self.ncol)], axis=1)

    def lstsq(self, b) -> np.ndarray:
        """C = R^{-1} Q^T b with the precomputed QR (Steps 2 and 5)."""
        from scipy.linalg import solve_triangular
        return solve_triangular(self.R, self.Q.T @ b)

    def extend(self, C, neumann=None) -> np.ndarray:
        """u_gamma = sum C0 phi + d g_N + beta (d^2/2) sum C2 phi (eq. extension_operator)."""
        u = self.phi @ C[: self.nsh]
        if self.beta:
            u = u + 0.5 * self.d ** 2 * (self.phi @ C[self.nsh:])
        if neumann is not None:
            u = u + self.d * neumann
        return u

    def gamma_grid(self, v_gamma):
        return gamma_density_grid(v_gamma, self.gamma_idx, self.N)


def dpm_elliptic_solve(setup: DPMSetup, f, neumann=None):
    """Solve (sigma - Lap) u = f in Omega with du/dn = neumann on Gamma.

    Step 4a: particular solution; Step 5: BEP least squares + extension;
    Steps 6-7: Green's formula u = P u_gamma + G f on N^+ (eq.
    generalized_greens_formula).  Returns (u on N^+, C, u_gamma)."""
    s = setup
    G = particular_solution(f, s.sets, s.h, s.sigma)
    b = G.reshape(-1)[s.gin_idx]
    if neumann is not None:
        b = b - s.i_minus_p_gin(s.d * neumann)
    C = s.lstsq(b)
    ug = s.extend(C, neumann)
    u = G + difference_potential(s.gamma_grid(ug), s.sets, s.h, s.sigma)
    return u, C, ug


# ---------------------------------------------------------------------------
# Domain decomposition, Case 1 (Section 3): Omega_1 = ball |x - c| < r1,
# Omega_2 = shell r1 < |x - c| < r2, each embedded in its own cubic box and
# grid.  The interface Z (|x - c| = r1) carries three spherical-harmonic
# series -- u, du/dnu, d2u/dnu2 with nu = (x - c)/|x - c| -- shared by both
# sub-domains, which is how the interface conditions (continuity of u and of
# its normal derivatives across Z) enter; Gamma (|x - c| = r2) carries u and
# d2u/dn2 with du/dn the Neumann data (2-term extension of the single domain).
# The reduced BEPs of both sub-domains (eqs. reduced_DD1_BEP1,
# reduced_DD1_BEP2) are stacked into one least-squares problem.
# ---------------------------------------------------------------------------
class Shell:
    """Spherical shell r_in < |x - c| < r_out (kind 2; axes = (r_out, r_in, 0))."""

    def __init__(self, r_out, r_in, center=(0.0, 0.0, 0.0)):
        self.kind, self.center, self.axes = 2, tuple(center), (r_out, r_in, 0.0)


class DDSubdomain:
    """Point sets and gamma geometry of one sub-domain; `surf` = 1 for the grid
    boundary nodes whose foot point lies on Z, 0 for those on Gamma."""

    def __init__(self, geom, N, lo, hi, r_z, K):
        self.geom, self.N, self.lo, self.hi = geom, N, lo, hi
        self.h = grid_spacing(N, lo, hi)
        self.sets = point_sets(inside_mask(geom, N, lo, hi))
        self.labels = labels_from_sets(self.sets)
        self.gamma_idx = np.flatnonzero(self.sets["gamma"].reshape(-1))
        self.gin_idx = np.flatnonzero(self.sets["gin"].reshape(-1))
        self.gin_pos = np.searchsorted(self.gamma_idx, self.gin_idx)
        X, Y, Z = mesh(N, lo, hi)
        P = np.stack([X.reshape(-1)[self.gamma_idx], Y.reshape(-1)[self.gamma_idx],
                      Z.reshape(-1)[self.gamma_idx]], axis=1)
        self.xf, self.d, self.normal = foot_point(geom, P)
        rf = np.linalg.norm(self.xf - np.asarray(geom.center), axis=1)
        self.surf = (np.abs(rf - r_z) < 1e-9 * max(1.0, r_z)).astype(np.int64)
        self.phi = boundary_basis(geom, self.xf, K)

    def i_minus_p_gin(self, v_gamma, sigma):
        """Tr_{gamma_in} (v_gamma - P v_gamma) on this sub-domain's grid."""
        vg = gamma_density_grid(v_gamma, self.gamma_idx, self.N)
        Pv = difference_potential(vg, self.sets, self.h, sigma)
        return v_gamma[self.gin_pos] - Pv.reshape(-1)[self.gin_idx]


class DDSetup:
    """Steps 1-2 of the two-sub-domain method: both sub-domains, the column
    densities of the shared Z series and the Gamma series, and the stacked
    reduced BEP matrix with its QR decomposition."""

    def __init__(self, center, r1, r2, N1, lo1, hi1, N2, lo2, hi2, KZ, KG, sigma, build_bep=True):
        self.r1, self.r2, self.KZ, self.KG, self.sigma = r1, r2, KZ, KG, sigma
        self.nz, self.ng = (KZ + 1) ** 2, (KG + 1) ** 2
        self.ncol = 3 * self.nz + 2 * self.ng
        K = max(KZ, KG)
        self.sub = [DDSubdomain(_Sph(center, r1), N1, lo1, hi1, r1, KZ),
                    DDSubdomain(Shell(r2, r1, center), N2, lo2, hi2, r1, K)]
        if build_bep:
            self.A = self.bep_matrix()
            self.Q, self.R = np.linalg.qr(self.A)

    def column_density(self, l, k):
        """Density of unknown k on sub-domain l's grid boundary: Z columns
        (3 terms x nz harmonics: phi, s phi, s^2/2 phi with s the signed distance
        from Z along nu) on its Z nodes, Gamma columns (2 terms x ng: phi,
        d^2/2 phi) on its Gamma nodes; zero on the other nodes."""
        sd = self.sub[l]
        out = np.zeros(len(sd.gamma_idx))
        if k < 3 * self.nz:
            t, nu = divmod(k, self.nz)
            m = sd.surf == 1
            fac = (np.ones_like(sd.d), sd.d, 0.5 * sd.d ** 2)[t]
        else:
            t, nu = divmod(k - 3 * self.nz, self.ng)
            m = sd.surf == 0
            fac = (np.ones_like(sd.d), 0.5 * sd.d ** 2)[t]
        out[m] = fac[m] * sd.phi[m, nu]
        return out

    def bep_matrix(self):
        """Rows gamma_in of Omega_1, then gamma_in of Omega_2 (Z and Gamma nodes);
        one column per unknown coefficient."""
        blocks = []
        for l, sd in enumerate(self.sub):
            cols = []
            for k in range(self.ncol):
                psi = self.column_density(l, k)
                cols.append(sd.i_minus_p_gin(psi, self.sigma) if np.any(psi) else np.zeros(len(sd.gin_idx)))
            blocks.append(np.stack(cols, axis=1))
        return np.vstack(blocks)

    def lstsq(self, b):
        from scipy.linalg import solve_triangular
        return solve_triangular(self.R, self.Q.T @ b)

    def densities(self, C, neumann2=None):
        """u on each grid boundary from the coefficients (+ d g_N on Gamma nodes)."""
        out = []
        for l, sd in enumerate(self.sub):
            u = np.zeros(len(sd.gamma_idx))
            for k in range(self.ncol):
                u += C[k] * self.column_density(l, k)
            if l == 1 and neumann2 is not None:
                m = sd.surf == 0
                u[m] += sd.d[m] * neumann2[m]
            out.append(u)
        return out


def dd_elliptic_solve(setup: DDSetup, f1, f2, neumann2=None):
    """(sigma - Lap) u = f in Omega = Omega_1 + Omega_2, du/dn = g_N on Gamma
    (neumann2: values at the grid boundary nodes of Omega_2, used on its Gamma
    nodes), by the coupled reduced BEPs, then Green's formula in each sub-domain.
    Returns (u1 on N^+_1, u2 on N^+_2, C)."""
    S1, S2 = setup.sub
    G1 = particular_solution(f1, S1.sets, S1.h, setup.sigma)
    G2 = particular_solution(f2, S2.sets, S2.h, setup.sigma)
    b1 = G1.reshape(-1)[S1.gin_idx]
    b2 = G2.reshape(-1)[S2.gin_idx]
    if neumann2 is not None:
        v = np.where(S2.surf == 0, S2.d * neumann2, 0.0)
        b2 = b2 - S2.i_minus_p_gin(v, setup.sigma)
    C = setup.lstsq(np.concatenate([b1, b2]))
    ug1, ug2 = setup.densities(C, neumann2)
    u1 = G1 + difference_potential(gamma_density_grid(ug1, S1.gamma_idx, S1.N), S1.sets, S1.h, setup.sigma)
    u2 = G2 + difference_potential(gamma_density_grid(ug2, S2.gamma_idx, S2.N), S2.sets, S2.h, setup.sigma)
    return u1, u2, C


# ---------------------------------------------------------------------------
# Domain decomposition into L concentric sub-domains, Case 1 generalised: the
# ball |x - c| < rho_1 and the shells rho_l < |x - c| < rho_{l+1} (rho_L = R), each
# on its own grid.  Interface Z_m (|x - c| = rho_m, m = 1..L-1) carries its own
# three series (u, du/dnu, d2u/dnu2, nu = (x - c)/|x - c|, degree K_m) shared by
# the two sub-domains it separates; Gamma carries the two series of the
# outermost shell.  A shell's grid-boundary node belongs to the nearer of its
# two spheres (the outer one on a tie), as in Case 1.  The reduced BEPs of all
# sub-domains are stacked; each involves only the series of its own surfaces.
# ---------------------------------------------------------------------------
class MLSubdomain:
    """Sub-domain l of the layered decomposition: point sets, the sphere index
    of each grid-boundary node (m = 1..L; L is Gamma), its signed distance s
    from that sphere along nu, and the harmonics of its direction."""

    def __init__(self, l, center, radii, N, lo, hi, Kmax):
        self.l, self.N, self.lo, self.hi = l, N, lo, hi
        c = np.asarray(center, dtype=np.float64)
        self.geom = _Sph(center, radii[0]) if l == 0 else Shell(radii[l], radii[l - 1], center)
        self.h = grid_spacing(N, lo, hi)
        self.sets = point_sets(inside_mask(self.geom, N, lo, hi))
        self.labels = labels_from_sets(self.sets)
        self.gamma_idx = np.flatnonzero(self.sets["gamma"].reshape(-1))
        self.gin_idx = np.flatnonzero(self.sets["gin"].reshape(-1))
        self.gin_pos = np.searchsorted(self.gamma_idx, self.gin_idx)
        X, Y, Z = mesh(N, lo, hi)
        P = np.stack([X.reshape(-1)[self.gamma_idx], Y.reshape(-1)[self.gamma_idx],
                      Z.reshape(-1)[self.gamma_idx]], axis=1)
        self.xf, _, self.normal = foot_point(self.geom, P)
        rho = np.linalg.norm(P - c, axis=1)
        if l == 0:
            self.sphere = np.ones(len(P), dtype=np.int64)
        else:
            outer = np.abs(rho - radii[l]) <= np.abs(rho - radii[l - 1])
            self.sphere = np.where(outer, l + 1, l)
        self.s = rho - np.asarray(radii)[self.sphere - 1]
        self.phi = boundary_basis(self.geom, self.xf, Kmax)

    def i_minus_p_gin(self, v_gamma, sigma):
        vg = gamma_density_grid(v_gamma, self.gamma_idx, self.N)
        Pv = difference_potential(vg, self.sets, self.h, sigma)
        return v_gamma[self.gin_pos] - Pv.reshape(-1)[self.gin_idx]


class MLSetup:
    """Steps 1-2 of the layered decomposition: the L sub-domains, the columns
    (interface m: 3 (K_m + 1)^2, term-major; then Gamma: 2 (K_G + 1)^2), the
    stacked reduced BEP matrix and its QR decomposition."""

    def __init__(self, center, radii, grids, K, KG, sigma, build_bep=True):
        # radii: rho_1 .. rho_{L-1}, R; grids: (N, lo, hi) per sub-domain; K: K_m per interface
        self.L = len(radii)
        self.radii, self.K, self.KG, self.sigma = list(radii), list(K), KG, sigma
        self.n = [(k + 1) ** 2 for k in self.K] + [(KG + 1) ** 2]
        self.terms = [3] * (self.L - 1) + [2]
        self.off = np.concatenate([[0], np.cumsum([t * n for t, n in zip(self.terms, self.n)])]).astype(int)
        self.ncol = int(self.off[-1])
        Kmax = max(self.K + [KG])
        self.sub = [MLSubdomain(l, center, radii, *grids[l], Kmax) for l in range(self.L)]
        if build_bep:
            self.A = self.bep_matrix()
            self.Q, self.R = np.linalg.qr(self.A)

    def column_sphere(self, k):
        m = int(np.searchsorted(self.off, k, side="right"))  # 1-based sphere index
        t, nu = divmod(k - self.off[m - 1], self.n[m - 1])
        return m, t, nu

    def column_density(self, l, k):
        sd = self.sub[l]
        m, t, nu = self.column_sphere(k)
        on = sd.sphere == m
        out = np.zeros(len(sd.gamma_idx))
        if not np.any(on):
            return out
        s = sd.s[on]
        fac = (np.ones_like(s), s, 0.5 * s * s)[t] if m < self.L else (np.ones_like(s), 0.5 * s * s)[t]
        out[on] = fac * sd.phi[on, nu]
        return out

    def bep_matrix(self):
        blocks = []
        for l, sd in enumerate(self.sub):
            cols = []
            for k in range(self.ncol):
                psi = self.column_density(l, k)
                cols.append(sd.i_minus_p_gin(psi, self.sigma) if np.any(psi) else np.zeros(len(sd.gin_idx)))
            blocks.append(np.stack(cols, axis=1))
        return np.vstack(blocks)

    def lstsq(self, b):
        from scipy.linalg import solve_triangular
        return solve_triangular(self.R, self.Q.T @ b)

    def densities(self, C, neumann=None, clamp=False):
        out = []
        for l, sd in enumerate(self.sub):
            u = np.zeros(len(sd.gamma_idx))
            for k in range(self.ncol):
                u += C[k] * self.column_density(l, k)
            if l == self.L - 1 and neumann is not None:
                g = sd.sphere == self.L
                u[g] += sd.s[g] * neumann[g]
            out.append(np.maximum(u, 0.0) if clamp else u)
        return out


def ml_elliptic_solve(setup: MLSetup, fs, neumann=None):
    """(sigma - Lap) u = f on the union of the sub-domains, du/dn = g_N on Gamma
    (neumann: values at the outermost sub-domain's grid-boundary nodes, read on
    its Gamma nodes).  Returns ([u_l on N^+_l], C)."""
    G, b = [], []
    L = setup.L
    for l, (sd, f) in enumerate(zip(setup.sub, fs)):
        g = particular_solution(f, sd.sets, sd.h, setup.sigma)
        bl = g.reshape(-1)[sd.gin_idx]
        if l == L - 1 and neumann is not None:
            v = np.where(sd.sphere == L, sd.s * neumann, 0.0)
            bl = bl - sd.i_minus_p_gin(v, setup.sigma)
        G.append(g)
        b.append(bl)
    C = setup.lstsq(np.concatenate(b))
    dens = setup.densities(C, neumann)
    us = [g + difference_potential(gamma_density_grid(u, sd.gamma_idx, sd.N), sd.sets, sd.h, setup.sigma)
          for g, u, sd in zip(G, dens, setup.sub)]
    return us, C


class MLPKSState:
    """Oracle of the time loop on the layered decomposition: dt from the smallest
    CFL bound of all grids (and dt_max, dt_prev), the stacked BEP rebuilt when dt
    changes, one least squares for the particular traces of all sub-domains."""

    def __init__(self, center, radii, grids, K, KG, chi, dt_max, rho0, c0, dt_mode="cfl", clamp=True):
        self.args = (center, radii, grids, K, KG)
        self.chi, self.dt_max, self.dt_mode, self.clamp = chi, dt_max, dt_mode, clamp
        base = MLSetup(*self.args, 1.0 / dt_max, build_bep=False)
        self.sub = base.sub
        self.setup, self.dt, self.t = None, None, 0.0
        self.rho, self.c = [], []
        for sd in self.sub:
            X, Y, Z = mesh(sd.N, sd.lo, sd.hi)
            r = np.where(sd.sets["Mp"], rho0(X, Y, Z), 0.0)
            c = np.where(sd.sets["Mp"], c0(X, Y, Z), 0.0)
            ex = sd.labels.reshape(-1)[sd.gamma_idx] & LBL_GEX > 0
            xf = sd.xf[ex]
            r.reshape(-1)[sd.gamma_idx[ex]] = rho0(xf[:, 0], xf[:, 1], xf[:, 2])
            c.reshape(-1)[sd.gamma_idx[ex]] = c0(xf[:, 0], xf[:, 1], xf[:, 2])
            self.rho.append(r)
            self.c.append(c)

    def choose_dt(self):
        if self.dt_mode == "fixed":
            return self.dt_max
        cand = min([self.dt_max] + [cfl_dt(c, sd.sets, sd.h, self.chi) for c, sd in zip(self.c, self.sub)])
        return cand if self.dt is None else min(self.dt, cand)

    def step(self):
        dt = self.choose_dt()
        if self.setup is None or dt != self.dt:
            self.setup = MLSetup(*self.args, 1.0 / dt)
        self.dt = dt
        S = self.setup
        rhs = [pks_rhs(r, c, sd.sets, sd.h, self.chi, dt) for r, c, sd in zip(self.rho, self.c, S.sub)]
        new = []
        for f in range(2):  # rho, c
            G = [particular_solution(rhs[l][f] / dt, sd.sets, sd.h, S.sigma) for l, sd in enumerate(S.sub)]
            b = np.concatenate([G[l].reshape(-1)[sd.gin_idx] for l, sd in enumerate(S.sub)])
            C = S.lstsq(b)
            dens = S.densities(C, clamp=self.clamp)
            new.append([G[l] + difference_potential(gamma_density_grid(dens[l], sd.gamma_idx, sd.N), sd.sets,
                                                    sd.h, S.sigma) for l, sd in enumerate(S.sub)])
        self.rho, self.c = new
        self.t += dt
        return dt

    def diagnostics(self):
        parts = [diagnostics(r, c, sd.sets, sd.h, sd.N, sd.lo, sd.hi) for r, c, sd in zip(self.rho, self.c, self.sub)]
        return dict(mass=sum(p["mass"] for p in parts), max_rho=max(p["max_rho"] for p in parts),
                    min_rho=min(p["min_rho"] for p in parts), min_c=min(p["min_c"] for p in parts),
                    m2=sum(p["m2"] for p in parts), free_energy=sum(p["free_energy"] for p in parts))


# ---------------------------------------------------------------------------
# Domain decomposition, Case 2 (Section 3): the interface Z meets Gamma.
# Omega is the sphere |x - c| < R; Z is the sphere |x - c_Z| = r_Z with
# c_Z = c + (0, 0, z_off); Omega_1 = Omega inside Z (a lens around the north
# pole when z_off = R), Omega_2 = Omega outside Z.  Each sub-domain has its own
# cubic box and grid, described in a local frame: global x = origin + local x,
# the box is [lo, hi]^3 in local coordinates, and its geometry's centres are
# the global ones minus the origin.
# Reading of the grid boundary split (gamma_l, zeta_l of Section 3): a node of
# sub-domain l's grid boundary (Definition 2.1 on Omega_l) belongs to gamma_l
# when it is a grid-boundary node of the whole sphere Omega on the same grid,
# and to zeta_l when it is a grid-boundary node of the ball inside Z; a node in
# both lies in the layer at the wedge Z n Gamma and carries two values (the
# "extra layer" of the paper's angle window is this one grid layer).  A node in
# neither (possible only for nodes exactly on a sphere) is given to the nearer
# surface.  Its effective density is the mean of its values; every node of
# gamma_l,in gives one BEP row per surface it belongs to (eq. reduced_DD2_BEP).
# Basis: zonal harmonics about the z axis through each surface's centre,
# Y_nu(theta) = sqrt((2 nu + 1)/(4 pi)) P_nu(cos theta), nu < M (Section 4 uses
# zonal harmonics; on Z the cosine is first mapped from the range the part of Z
# inside Omega spans to [-1, 1], the same polynomials in a basis that stays
# well conditioned there), M_Z per term of the 3-term series on Z (u, du/dnu,
# d2u/dnu2, nu = (x - c_Z)/|x - c_Z|, shared by both sub-domains) and M_G per
# term of the 2-term series on Gamma (u, d2u/dn2; du/dn the Neumann data).
# ---------------------------------------------------------------------------
def zonal_harmonics(M: int, cos_theta: np.ndarray) -> np.ndarray:
    """sqrt((2 nu + 1)/(4 pi)) P_nu(x), nu = 0..M-1, by Bonnet's recurrence
    (nu + 1) P_{nu+1} = (2 nu + 1) x P_nu - nu P_{nu-1}.  Shape (len(x), M)."""
    x = np.asarray(cos_theta, dtype=np.float64)
    P = np.zeros((len(x), max(M, 1)))
    P[:, 0] = 1.0
    if M > 1:
        P[:, 1] = x
    for nu in range(1, M - 1):
        P[:, nu + 1] = ((2 * nu + 1) * x * P[:, nu] - nu * P[:, nu - 1]) / (nu + 1)
    norm = np.sqrt((2 * np.arange(M) + 1) / (4 * math.pi))
    return P[:, :M] * norm


class Lens:
    """Omega_1 of Case 2: |x - c| < R and |x - c_Z| < r_Z, c_Z = c + (0, 0, z_off)
    (kind 3; axes = (R, r_Z, z_off))."""

    def __init__(self, R, r_z, z_off, center=(0.0, 0.0, 0.0)):
        self.kind, self.center, self.axes = 3, tuple(center), (R, r_z, z_off)


class OutsideZ:
    """Omega_2 of Case 2: |x - c| < R and |x - c_Z| > r_Z (kind 4; axes as Lens)."""

    def __init__(self, R, r_z, z_off, center=(0.0, 0.0, 0.0)):
        self.kind, self.center, self.axes = 4, tuple(center), (R, r_z, z_off)


def _z_centre(geom):
    c = geom.center
    return (c[0], c[1], c[2] + geom.axes[2])


def _two_sphere_inside(geom, X, Y, Z):
    R, rz, _ = geom.axes
    inO = ellipsoid_form(_Sph(geom.center, R), X, Y, Z) < 1.0
    fz = ellipsoid_form(_Sph(_z_centre(geom), rz), X, Y, Z)
    return inO & ((fz < 1.0) if geom.kind == 3 else (fz > 1.0))


def _radial(P, c):
    """|p - c| summed as (qx^2 + qy^2) + qz^2, and q = p - c."""
    q = P - np.asarray(c, dtype=np.float64)
    return np.sqrt((q[:, 0] * q[:, 0] + q[:, 1] * q[:, 1]) + q[:, 2] * q[:, 2]), q


class DD2Subdomain:
    """Point sets, the gamma_l / zeta_l split, distances, zonal harmonics and
    the BEP rows of one sub-domain of Case 2."""

    def __init__(self, geom, N, lo, hi, origin, MZ, MG):
        self.geom, self.N, self.lo, self.hi = geom, N, lo, hi
        self.origin = np.asarray(origin, dtype=np.float64)
        self.h = grid_spacing(N, lo, hi)
        X, Y, Z = mesh(N, lo, hi)
        self.sets = point_sets(inside_mask(geom, N, lo, hi))
        self.labels = labels_from_sets(self.sets)
        self.gamma_idx = np.flatnonzero(self.sets["gamma"].reshape(-1))
        self.gin_idx = np.flatnonzero(self.sets["gin"].reshape(-1))
        self.gin_pos = np.searchsorted(self.gamma_idx, self.gin_idx)
        R, rz, _ = geom.axes
        c0, cz = geom.center, _z_centre(geom)
        on_g = point_sets(inside_mask(_Sph(c0, R), N, lo, hi))["gamma"].reshape(-1)[self.gamma_idx]
        on_z = point_sets(inside_mask(_Sph(cz, rz), N, lo, hi))["gamma"].reshape(-1)[self.gamma_idx]
        P = np.stack([X.reshape(-1)[self.gamma_idx], Y.reshape(-1)[self.gamma_idx],
                      Z.reshape(-1)[self.gamma_idx]], axis=1)
        rg, qg = _radial(P, c0)
        rzz, qz = _radial(P, cz)
        self.dG, self.dZ = rg - R, rzz - rz
        neither = ~on_g & ~on_z
        near_g = np.abs(self.dG) <= np.abs(self.dZ)
        self.on_g = on_g | (neither & near_g)
        self.on_z = on_z | (neither & ~near_g)
        cnt = self.on_g.astype(np.float64) + self.on_z.astype(np.float64)
        self.wG, self.wZ = self.on_g / cnt, self.on_z / cnt
        # a node at a sphere's centre carries no value of that sphere (cosine 1)
        rg1, rz1 = np.where(rg > 0, rg, 1.0), np.where(rzz > 0, rzz, 1.0)
        cos_g = np.where(rg > 0, qg[:, 2] / rg1, 1.0)
        cos_z = np.where(rzz > 0, qz[:, 2] / rz1, 1.0)
        self.phiG = zonal_harmonics(MG, cos_g)
        # Z inside Omega spans cos theta_Z in [-1, c*] (z_off > 0; [c*, 1] otherwise),
        # c* the cosine at the circle Z n Gamma; its series uses P_nu of cos theta_Z
        # mapped from that range to [-1, 1] (the same polynomials of degree < MZ)
        zoff = geom.axes[2]
        cstar = (R * R - zoff * zoff - rz * rz) / (2.0 * zoff * rz)
        a, b = (-1.0, cstar) if zoff > 0 else (cstar, 1.0)
        self.phiZ = zonal_harmonics(MZ, (2.0 * cos_z - (a + b)) / (b - a))
        self.footG = np.asarray(c0) + R * (qg / rg1[:, None])
        self.footZ = np.asarray(cz) + rz * (qz / rz1[:, None])
        self.normalG = qg / rg1[:, None]
        # rows: gamma_in nodes in ascending order; a Gamma row before a Z row
        rows = []
        for i, e in enumerate(self.gin_pos):
            if self.on_g[e]:
                rows.append((i, e, 0))
            if self.on_z[e]:
                rows.append((i, e, 1))
        self.rows = np.array(rows, dtype=np.int64).reshape(-1, 3)

    def value(self, k, surf, MZ, MG):
        """Value of unknown k's basis density at every node of gamma_l as the
        given surface's series (1 = Z, 0 = Gamma) would give it.  Gamma unknowns
        k - 3 MZ = t MG + nu: t = 0 the series of u, t = 1 that of d^2u/dn^2."""
        if k < 3 * MZ:
            if surf == 0:
                return np.zeros(len(self.gamma_idx))
            t, nu = divmod(k, MZ)
            fac = (np.ones_like(self.dZ), self.dZ, 0.5 * self.dZ ** 2)[t]
            return fac * self.phiZ[:, nu]
        if surf == 1:
            return np.zeros(len(self.gamma_idx))
        t, nu = divmod(k - 3 * MZ, MG)
        fac = (np.ones_like(self.dG), 0.5 * self.dG ** 2)[t]
        return fac * self.phiG[:, nu]

    def rows_minus_potential(self, own, eff, sigma):
        """Row values own(surface of row)[node] - Tr P_{N+gamma} eff at the row's node."""
        Pv = difference_potential(gamma_density_grid(eff, self.gamma_idx, self.N), self.sets, self.h, sigma)
        tr = Pv.reshape(-1)[self.gin_idx]
        i, e, sf = self.rows[:, 0], self.rows[:, 1], self.rows[:, 2]
        return np.where(sf == 1, own[1][e], own[0][e]) - tr[i]


class DD2Setup:
    """Steps 1-2 of Case 2: both sub-domains, the stacked reduced BEPs
    (eq. reduced_DD2_BEP, l = 1, 2) over the shared Z and Gamma series, and the
    QR decomposition.  gamma_series: the unknown series on Gamma, 2 for the
    3-term extension u + d g_N + (d^2/2) d^2u/dn^2, 1 for the 2-term extension
    u + d g_N that the paper uses on the boundary for Test (B) (Section 4, "Basis
    functions, extension operators and BEPs")."""

    def __init__(self, center, R, r_z, z_off, N1, lo1, hi1, origin1, N2, lo2, hi2, origin2, MZ, MG, sigma,
                 build_bep=True, gamma_series=2):
        self.R, self.r_z, self.z_off, self.MZ, self.MG, self.sigma = R, r_z, z_off, MZ, MG, sigma
        self.gamma_series = gamma_series
        self.ncol = 3 * MZ + gamma_series * MG
        # the sphere's centre in each sub-domain's local frame
        c1 = np.asarray(center, dtype=np.float64) - np.asarray(origin1, dtype=np.float64)
        c2 = np.asarray(center, dtype=np.float64) - np.asarray(origin2, dtype=np.float64)
        self.sub = [DD2Subdomain(Lens(R, r_z, z_off, tuple(c1)), N1, lo1, hi1, origin1, MZ, MG),
                    DD2Subdomain(OutsideZ(R, r_z, z_off, tuple(c2)), N2, lo2, hi2, origin2, MZ, MG)]
        if build_bep:
            self.A = self.bep_matrix()
            self.Q, self.R_ = np.linalg.qr(self.A)

    def column(self, l, k):
        sd = self.sub[l]
        vz = sd.value(k, 1, self.MZ, self.MG)
        vg = sd.value(k, 0, self.MZ, self.MG)
        return (vg, vz), sd.wG * vg + sd.wZ * vz

    def bep_matrix(self):
        blocks = []
        for l, sd in enumerate(self.sub):
            cols = []
            for k in range(self.ncol):
                own, eff = self.column(l, k)
                cols.append(sd.rows_minus_potential(own, eff, self.sigma))
            blocks.append(np.stack(cols, axis=1))
        return np.vstack(blocks)

    def lstsq(self, b):
        from scipy.linalg import solve_triangular
        return solve_triangular(self.R_, self.Q.T @ b)

    def densities(self, C, neumann=None, clamp=False):
        """Effective density of each sub-domain from the coefficients: the mean of
        the Gamma series value (+ d g_N) and the Z series value at wedge nodes."""
        out = []
        for l, sd in enumerate(self.sub):
            ug = np.zeros(len(sd.gamma_idx))
            uz = np.zeros(len(sd.gamma_idx))
            for k in range(self.ncol):
                ug += C[k] * sd.value(k, 0, self.MZ, self.MG)
                uz += C[k] * sd.value(k, 1, self.MZ, self.MG)
            if neumann is not None:
                ug = ug + sd.dG * neumann[l]
            u = sd.wG * ug + sd.wZ * uz
            out.append(np.maximum(u, 0.0) if clamp else u)
        return out


def dd2_elliptic_solve(setup: DD2Setup, f1, f2, neumann=None):
    """(sigma - Lap) u = f on Omega_1 + Omega_2 with du/dn = g_N on Gamma
    (neumann[l]: g_N at the Gamma foot points of sub-domain l's grid boundary
    nodes), by the stacked BEPs of Case 2 and Green's formula per sub-domain.
    Returns (u1, u2, C)."""
    G, b = [], []
    for l, (sd, f) in enumerate(zip(setup.sub, (f1, f2))):
        g = particular_solution(f, sd.sets, sd.h, setup.sigma)
        bl = g.reshape(-1)[sd.gin_idx][sd.rows[:, 0]]
        if neumann is not None:
            vg = sd.dG * neumann[l]
            bl = bl - sd.rows_minus_potential((vg, np.zeros_like(vg)), sd.wG * vg, setup.sigma)
        G.append(g)
        b.append(bl)
    C = setup.lstsq(np.concatenate(b))
    dens = setup.densities(C, neumann)
    us = [g + difference_potential(gamma_density_grid(u, sd.gamma_idx, sd.N), sd.sets, sd.h, setup.sigma)
          for g, u, sd in zip(G, dens, setup.sub)]
    return us[0], us[1], C


# ---------------------------------------------------------------------------
# PKS discretisation (eqs. discrete_chemotaxis .. slope_limiter, cfl_condition)
# ---------------------------------------------------------------------------
def minmod(*xs):
    """eq. slope_limiter: min if all > 0, max if all < 0, else 0."""
    X = np.stack(np.broadcast_arrays(*xs))
    allpos = np.all(X > 0, axis=0)
    allneg = np.all(X < 0, axis=0)
    return np.where(allpos, X.min(axis=0), np.where(allneg, X.max(axis=0), 0.0))


def _shift(a, ax, s, fill=0.0):
    """b[p] = a[p + s e_ax] (fill outside the grid)."""
    out = np.full_like(a, fill)
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    if s > 0:
        src[ax] = slice(s, None)
        dst[ax] = slice(None, -s)
    else:
        src[ax] = slice(None, s)
        dst[ax] = slice(-s, None)
    out[tuple(dst)] = a[tuple(src)]
    return out


def limited_slopes(rho, Np, h, ax):
    """minmod slope of rho along axis ax at every node of N^+; 0 where one of
    the two neighbours is not in N^+ (reading of the paper's silence)."""
    rp, rm = _shift(rho, ax, 1), _shift(rho, ax, -1)
    ok = Np & _shift(Np, ax, 1, False) & _shift(Np, ax, -1, False)
    s = minmod(2.0 * (rp - rho) / h, (rp - rm) / (2.0 * h), 2.0 * (rho - rm) / h)
    return np.where(ok, s, 0.0)


def convective_term(rho, c, sets, h, chi):
    """g of eq. discrete_convective_term on M^+ (0 elsewhere).

    Face gradients by eq. c-central-difference; face densities upwinded by eq.
    upwind_approximation from the piecewise-linear reconstruction with minmod
    slopes (eq. truncated_taylor_expansion)."""
    Np, Mp = sets["Np"], sets["Mp"]
    g = np.zeros_like(rho)
    for ax in range(3):
        s = limited_slopes(rho, Np, h, ax)
        rE = rho + 0.5 * h * s          # reconstruction at x_{j+1/2} - 0
        rW = rho - 0.5 * h * s          # reconstruction at x_{j-1/2} + 0
        gp = (_shift(c, ax, 1) - c) / h                 # grad c at j+1/2
        gm = (c - _shift(c, ax, -1)) / h                # grad c at j-1/2
        rho_p = np.where(gp > 0, rE, _shift(rW, ax, 1))
        rho_m = np.where(gm > 0, _shift(rE, ax, -1), rW)
        g += (chi * rho_p * gp - chi * rho_m * gm) / h
    return np.where(Mp, g, 0.0)


def max_face_gradients(c, sets, h):
    """max over M^+ of |grad_h c| at the j+-1/2 faces, per axis (eq. cfl_condition)."""
    Mp = sets["Mp"]
    out = []
    for ax in range(3):
        gp = np.abs(_shift(c, ax, 1) - c) / h
        gm = np.abs(c - _shift(c, ax, -1)) / h
        out.append(float(np.max(np.where(Mp, np.maximum(gp, gm), 0.0))))
    return out


def cfl_dt(c, sets, h, chi):
    """min over axes of h / (6 chi max|grad c|) (eq. cfl_condition)."""
    m = max_face_gradients(c, sets, h)
    return min(h / (6.0 * chi * g) if g > 0 else math.inf for g in m)


def pks_rhs(rho, c, sets, h, chi, dt):
    """f for both equations of eq. discrete_chemotaxis on M^+ (alpha = gamma_rho = gamma_c = 1)."""
    g = convective_term(rho, c, sets, h, chi)
    Mp = sets["Mp"]
    f_rho = np.where(Mp, rho - dt * g, 0.0)
    f_c = np.where(Mp, (1.0 - dt) * c + dt * rho, 0.0)
    return f_rho, f_c


def diagnostics(rho, c, sets, h, N, lo, hi):
    """Mass h^3 sum rho, max rho (eq. sd-norm:max), min rho / min c on N^+,
    second moment (eq. sd-norm:second-moment) and free energy (eq. sd-norm:free-energy)."""
    Mp, Np = sets["Mp"], sets["Np"]
    X, Y, Z = mesh(N, lo, hi)
    h3 = h ** 3
    r = np.where(Mp, rho, 0.0)
    mass = h3 * np.sum(r)
    m2 = h3 * np.sum(np.where(Mp, (X * X + Y * Y + Z * Z) * rho, 0.0))
    rlogr = np.where(rho > 0, rho * np.log(np.where(rho > 0, rho, 1.0)), 0.0)
    grad2 = np.zeros_like(c)
    for ax in range(3):
        grad2 += (_shift(c, ax, 1) - _shift(c, ax, -1)) ** 2
    dens = rlogr - rho * c + 0.5 * c * c + grad2 / (8.0 * h * h)
    F = h3 * np.sum(np.where(Mp, dens, 0.0))
    return dict(mass=mass, max_rho=float(np.max(np.where(Mp, rho, -np.inf))),
                min_rho=float(np.min(np.where(Np, rho, np.inf))),
                min_c=float(np.min(np.where(Np, c, np.inf))), m2=m2, free_energy=F)


class PKSState:
    """Oracle of the time loop, Steps 3-7, for the PKS model on one domain."""

    def __init__(self, geom, N, lo, hi, K, beta, chi, dt_max, rho0=None, c0=None,
                 dt_mode="fixed", clamp=True, rho=None, c=None):
        self.geom, self.N, self.lo, self.hi = geom, N, lo, hi
        self.K, self.beta, self.chi, self.dt_max = K, beta, chi, dt_max
        self.dt_mode, self.clamp = dt_mode, clamp
        self.h = grid_spacing(N, lo, hi)
        self.setup = None
        self.dt = None
        self.t = 0.0
        base = DPMSetup(geom, N, lo, hi, K, beta, 1.0 / dt_max, build_bep=False)
        self.sets = base.sets
        self._geo = base
        if rho is None:
            rho, c = self.initial_state(rho0, c0)
        self.rho = np.asarray(rho, dtype=np.float64)
        self.c = np.asarray(c, dtype=np.float64)

    def initial_state(self, rho0, c0):
        """rho^0, c^0 at the nodes of M^+ and at the foot points of gamma_ex
        (2-term extension with zero Neumann data, Remark 2.1)."""
        X, Y, Z = mesh(self.N, self.lo, self.hi)
        rho = np.where(self.sets["Mp"], rho0(X, Y, Z), 0.0)
        c = np.where(self.sets["Mp"], c0(X, Y, Z), 0.0)
        g = self._geo
        ex = g.labels.reshape(-1)[g.gamma_idx] & LBL_GEX > 0
        xf = g.xf[ex]
        rho.reshape(-1)[g.gamma_idx[ex]] = rho0(xf[:, 0], xf[:, 1], xf[:, 2])
        c.reshape(-1)[g.gamma_idx[ex]] = c0(xf[:, 0], xf[:, 1], xf[:, 2])
        return rho, c

    def choose_dt(self):
        """Step 3: fixed mode uses dt_max; cfl mode dt = min(dt_prev, dt_cfl, dt_max)."""
        if self.dt_mode == "fixed":
            return self.dt_max
        cand = min(self.dt_max, cfl_dt(self.c, self.sets, self.h, self.chi))
        return cand if self.dt is None else min(self.dt, cand)

    def step(self):
        dt = self.choose_dt()
        if self.setup is None or dt != self.dt:           # Step 2 / Step 4b
            self.setup = DPMSetup(self.geom, self.N, self.lo, self.hi, self.K, self.beta, 1.0 / dt)
        self.dt = dt
        s = self.setup
        f_rho, f_c = pks_rhs(self.rho, self.c, self.sets, self.h, self.chi, dt)   # Step 4a
        out = []
        for f in (f_rho, f_c):
            q = f / dt                                   # L_{h,dt} = dt (sigma - Lap_h)
            G = particular_solution(q, s.sets, s.h, s.sigma)
            C = s.lstsq(G.reshape(-1)[s.gin_idx])        # Step 5
            ug = s.extend(C)
            if self.clamp:
                ug = np.maximum(ug, 0.0)
            u = G + difference_potential(s.gamma_grid(ug), s.sets, s.h, s.sigma)   # Steps 6-7
            out.append(u)
        self.rho, self.c = out
        self.t += dt
        return dt


class DDPKSState:
    """Oracle of the time loop (Steps 3-7) on the two sub-domains of Case 1:
    each sub-domain keeps rho and c on its own grid; Step 3's dt is the
    smaller CFL bound of the two grids (and dt_max, and dt_prev); the coupled
    BEP is rebuilt whenever dt changes (Step 4b); every solve stacks the
    particular-solution traces of both sub-domains into one least squares."""

    def __init__(self, center, r1, r2, N1, lo1, hi1, N2, lo2, hi2, KZ, KG, chi, dt_max, rho0, c0,
                 dt_mode="cfl", clamp=True):
        self.args = (center, r1, r2, N1, lo1, hi1, N2, lo2, hi2, KZ, KG)
        self.chi, self.dt_max, self.dt_mode, self.clamp = chi, dt_max, dt_mode, clamp
        base = DDSetup(*self.args, 1.0 / dt_max, build_bep=False)
        self.sub = base.sub
        self.setup, self.dt, self.t = None, None, 0.0
        self.rho, self.c = [], []
        for sd in self.sub:
            X, Y, Z = mesh(sd.N, sd.lo, sd.hi)
            r = np.where(sd.sets["Mp"], rho0(X, Y, Z), 0.0)
            c = np.where(sd.sets["Mp"], c0(X, Y, Z), 0.0)
            ex = sd.labels.reshape(-1)[sd.gamma_idx] & LBL_GEX > 0
            xf = sd.xf[ex]
            r.reshape(-1)[sd.gamma_idx[ex]] = rho0(xf[:, 0], xf[:, 1], xf[:, 2])
            c.reshape(-1)[sd.gamma_idx[ex]] = c0(xf[:, 0], xf[:, 1], xf[:, 2])
            self.rho.append(r)
            self.c.append(c)

    def choose_dt(self):
        if self.dt_mode == "fixed":
            return self.dt_max
        cand = min([self.dt_max] + [cfl_dt(c, sd.sets, sd.h, self.chi) for c, sd in zip(self.c, self.sub)])
        return cand if self.dt is None else min(self.dt, cand)

    def step(self):
        dt = self.choose_dt()
        if self.setup is None or dt != self.dt:
            self.setup = DDSetup(*self.args, 1.0 / dt)
        self.dt = dt
        S = self.setup
        rhs = [pks_rhs(r, c, sd.sets, sd.h, self.chi, dt) for r, c, sd in zip(self.rho, self.c, S.sub)]
        new = []
        for f in range(2):  # rho, c
            G = [particular_solution(rhs[l][f] / dt, sd.sets, sd.h, S.sigma) for l, sd in enumerate(S.sub)]
            b = np.concatenate([G[l].reshape(-1)[sd.gin_idx] for l, sd in enumerate(S.sub)])
            C = S.lstsq(b)
            dens = S.densities(C)
            out = []
            for l, sd in enumerate(S.sub):
                ug = np.maximum(dens[l], 0.0) if self.clamp else dens[l]
                out.append(G[l] + difference_potential(gamma_density_grid(ug, sd.gamma_idx, sd.N),
                                                       sd.sets, sd.h, S.sigma))
            new.append(out)
        self.rho, self.c = new
        self.t += dt
        return dt

    def diagnostics(self):
        """diagnostics() of each sub-domain combined: sums of mass, second moment
        and free energy; max / min over both."""
        parts = [diagnostics(r, c, sd.sets, sd.h, sd.N, sd.lo, sd.hi)
                 for r, c, sd in zip(self.rho, self.c, self.sub)]
        return dict(mass=sum(p["mass"] for p in parts), max_rho=max(p["max_rho"] for p in parts),
                    min_rho=min(p["min_rho"] for p in parts), min_c=min(p["min_c"] for p in parts),
                    m2=sum(p["m2"] for p in parts), free_energy=sum(p["free_energy"] for p in parts))


class DD2PKSState:
    """Oracle of the time loop (Steps 3-7) on the two sub-domains of Case 2:
    rho and c on each sub-domain's grid (local frames), Step 3's dt from the
    smaller CFL bound of the two grids, the stacked BEP rebuilt whenever dt
    changes, one least squares for the particular traces of both sub-domains
    (wedge rows duplicated), effective densities clamped at 0."""

    def __init__(self, center, R, r_z, z_off, N1, lo1, hi1, origin1, N2, lo2, hi2, origin2, MZ, MG, chi,
                 dt_max, rho0, c0, dt_mode="cfl", clamp=True, gamma_series=2):
        self.args = (center, R, r_z, z_off, N1, lo1, hi1, origin1, N2, lo2, hi2, origin2, MZ, MG)
        self.gamma_series = gamma_series
        self.chi, self.dt_max, self.dt_mode, self.clamp = chi, dt_max, dt_mode, clamp
        base = DD2Setup(*self.args, 1.0 / dt_max, build_bep=False, gamma_series=gamma_series)
        self.sub = base.sub
        self.setup, self.dt, self.t = None, None, 0.0
        self.rho, self.c = [], []
        for sd in self.sub:
            X, Y, Z = mesh(sd.N, sd.lo, sd.hi)
            o = sd.origin
            X, Y, Z = X + o[0], Y + o[1], Z + o[2]
            r = np.where(sd.sets["Mp"], rho0(X, Y, Z), 0.0)
            c = np.where(sd.sets["Mp"], c0(X, Y, Z), 0.0)
            # gamma_ex: the data at the foot point on the node's first surface
            # (Gamma when it belongs to gamma_l, else Z)
            ex = sd.labels.reshape(-1)[sd.gamma_idx] & LBL_GEX > 0
            xf = np.where(sd.on_g[:, None], sd.footG, sd.footZ)[ex] + o
            r.reshape(-1)[sd.gamma_idx[ex]] = rho0(xf[:, 0], xf[:, 1], xf[:, 2])
            c.reshape(-1)[sd.gamma_idx[ex]] = c0(xf[:, 0], xf[:, 1], xf[:, 2])
            self.rho.append(r)
            self.c.append(c)

    def choose_dt(self):
        if self.dt_mode == "fixed":
            return self.dt_max
        cand = min([self.dt_max] + [cfl_dt(c, sd.sets, sd.h, self.chi) for c, sd in zip(self.c, self.sub)])
        return cand if self.dt is None else min(self.dt, cand)

    def step(self):
        dt = self.choose_dt()
        if self.setup is None or dt != self.dt:
            self.setup = DD2Setup(*self.args, 1.0 / dt, gamma_series=self.gamma_series)
        self.dt = dt
        S = self.setup
        rhs = [pks_rhs(r, c, sd.sets, sd.h, self.chi, dt) for r, c, sd in zip(self.rho, self.c, S.sub)]
        new = []
        for f in range(2):  # rho, c
            G = [particular_solution(rhs[l][f] / dt, sd.sets, sd.h, S.sigma) for l, sd in enumerate(S.sub)]
            b = np.concatenate([G[l].reshape(-1)[sd.gin_idx][sd.rows[:, 0]] for l, sd in enumerate(S.sub)])
            C = S.lstsq(b)
            dens = S.densities(C, clamp=self.clamp)
            new.append([G[l] + difference_potential(gamma_density_grid(dens[l], sd.gamma_idx, sd.N), sd.sets,
                                                    sd.h, S.sigma) for l, sd in enumerate(S.sub)])
        self.rho, self.c = new
        self.t += dt
        return dt

    def diagnostics(self):
        """Sums over both sub-domains of mass, second moment (global
        coordinates: local + origin) and free energy; max / min over both."""
        parts = []
        for r, c, sd in zip(self.rho, self.c, self.sub):
            d = diagnostics(r, c, sd.sets, sd.h, sd.N, sd.lo, sd.hi)
            X, Y, Z = mesh(sd.N, sd.lo, sd.hi)
            o = sd.origin
            X, Y, Z = X + o[0], Y + o[1], Z + o[2]
            d["m2"] = sd.h ** 3 * np.sum(np.where(sd.sets["Mp"], (X * X + Y * Y + Z * Z) * r, 0.0))
            parts.append(d)
        return dict(mass=sum(p["mass"] for p in parts), max_rho=max(p["max_rho"] for p in parts),
                    min_rho=min(p["min_rho"] for p in parts), min_c=min(p["min_c"] for p in parts),
                    m2=sum(p["m2"] for p in parts), free_energy=sum(p["free_energy"] for p in parts))

