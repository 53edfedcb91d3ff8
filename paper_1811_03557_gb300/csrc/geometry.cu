// Orthogonal projection of the nodes of gamma on Gamma (Definition 2.6) and
// the real orthonormal spherical harmonics at the foot points (eq.
// spectral_approximation_sd), in FP64.  Setup work, run once per geometry.
//
// Sphere: x' = c + r (p - c)/|p - c|, d = |p - c| - r, n = (p - c)/|p - c|.
// Ellipsoid: x'_i = c_i + q_i a_i^2/(a_i^2 + mu), q = p - c, where mu is the
// root in (-min a_i^2, inf) of F(mu) = sum q_i^2 a_i^2/(a_i^2+mu)^2 - 1 (the
// Lagrange condition of the closest point); F is convex and decreasing there,
// so Newton's method safeguarded by a bisection bracket converges to it.
// d = +-|p - x'| (> 0 outside), n = grad(sum (x_i-c_i)^2/a_i^2)/|.| at x'.
//
// Basis: Y_l0 = N_l0 P_l^0(cos t), Y_lm = sqrt2 N_lm P_l^m cos(m ph),
// Y_l,-m = sqrt2 N_lm P_l^m sin(m ph), N_lm = sqrt((2l+1)/(4pi) (l-m)!/(l+m)!),
// P_l^m without the Condon-Shortley phase; column nu = l^2 + l + m.
#include <math.h>

#include "dpm_internal.cuh"

namespace dpm {
namespace {

constexpr int kMaxK = 16;
__constant__ double c_nlm[(kMaxK + 1) * (kMaxK + 1)];

__device__ void project(int kind, const double c[3], const double a[3], const double p[3],
                        double xf[3], double nrm[3], double *dist) {
    double q[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
    if (kind == 2) {
        // spherical shell (radii a[0] > a[1]): the nearer sphere; normal (p - c)/|p - c|
        // and d = |p - c| - r on both spheres
        double rho = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        const double r = fabs(rho - a[0]) <= fabs(rho - a[1]) ? a[0] : a[1];
        for (int t = 0; t < 3; ++t) {
            nrm[t] = q[t] / rho;
            xf[t] = c[t] + r * nrm[t];
        }
        *dist = rho - r;
        return;
    }
    if (kind == 0) {
        double rho = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        for (int t = 0; t < 3; ++t) {
            nrm[t] = q[t] / rho;
            xf[t] = c[t] + a[0] * nrm[t];
        }
        *dist = rho - a[0];
        return;
    }
    double a2[3] = {a[0] * a[0], a[1] * a[1], a[2] * a[2]};
    double amin2 = fmin(a2[0], fmin(a2[1], a2[2]));
    double lo = -amin2, hi = 1.0;
    auto F = [&](double mu, double *dF) {
        double f = -1.0, df = 0.0;
        for (int t = 0; t < 3; ++t) {
            double w = 1.0 / (a2[t] + mu);
            double u = q[t] * q[t] * a2[t] * w * w;
            f += u;
            df -= 2.0 * u * w;
        }
        *dF = df;
        return f;
    };
    double dF;
    for (int it = 0; it < 200 && F(hi, &dF) > 0; ++it) hi = 2.0 * hi + 1.0;
    double mu = 0.0;
    if (!(mu > lo && mu < hi)) mu = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double f = F(mu, &dF);
        if (f > 0) lo = mu; else hi = mu;
        double nxt = mu - f / dF;
        if (!(nxt > lo && nxt < hi)) nxt = 0.5 * (lo + hi);
        double step = fabs(nxt - mu);
        mu = nxt;
        if (step <= 1e-16 * fmax(1.0, fabs(mu)) || hi - lo <= 1e-16 * fmax(1.0, fabs(mu))) break;
    }
    double g[3], gn = 0.0, dd = 0.0, s = 0.0;
    for (int t = 0; t < 3; ++t) {
        xf[t] = c[t] + q[t] * a2[t] / (a2[t] + mu);
        g[t] = (xf[t] - c[t]) / a2[t];
        gn += g[t] * g[t];
        dd += (p[t] - xf[t]) * (p[t] - xf[t]);
        s += q[t] * q[t] / a2[t];
    }
    gn = sqrt(gn);
    for (int t = 0; t < 3; ++t) nrm[t] = g[t] / gn;
    *dist = (s > 1.0 ? 1.0 : -1.0) * sqrt(dd);
}

__global__ void k_gamma_geom(int n, int N, double lo, double h, int kind, double cx, double cy,
                             double cz, double ax, double ay, double az, int K, const int *gamma,
                             double *foot, double *normal, double *dist, double *phi) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    int p = gamma[e];
    int k = p % N, j = (p / N) % N, i = p / (N * N);
    double P[3] = {lo + (double)(i + 1) * h, lo + (double)(j + 1) * h, lo + (double)(k + 1) * h};
    double c[3] = {cx, cy, cz}, a[3] = {ax, ay, az};
    double xf[3], nr[3], d;
    project(kind, c, a, P, xf, nr, &d);
    for (int t = 0; t < 3; ++t) {
        foot[3 * e + t] = xf[t];
        normal[3 * e + t] = nr[t];
    }
    dist[e] = d;
    // angles of the foot point about the centre
    double v0 = xf[0] - cx, v1 = xf[1] - cy, v2 = xf[2] - cz;
    double rad = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
    double x = v2 / rad;
    double ph = atan2(v1, v0);
    double st = sqrt(fmax(0.0, 1.0 - x * x));
    int nsh = (K + 1) * (K + 1);
    double *out = phi + (int64_t)e * nsh;
    double pmm = 1.0;  // P_m^m, built up as (2m-1)!! st^m
    for (int m = 0; m <= K; ++m) {
        if (m > 0) pmm *= (double)(2 * m - 1) * st;
        double cm = 1.0, sm = 0.0;
        if (m > 0) sincos((double)m * ph, &sm, &cm);
        double p2 = 0.0, p1 = 0.0;  // P_{l-2}^m, P_{l-1}^m
        for (int l = m; l <= K; ++l) {
            double plm;
            if (l == m) plm = pmm;
            else if (l == m + 1) plm = x * (2 * m + 1) * pmm;
            else plm = ((2 * l - 1) * x * p1 - (l + m - 1) * p2) / (double)(l - m);
            p2 = p1;
            p1 = plm;
            double nl = c_nlm[l * (kMaxK + 1) + m];
            if (m == 0) {
                out[l * l + l] = nl * plm;
            } else {
                out[l * l + l + m] = M_SQRT2 * nl * plm * cm;
                out[l * l + l - m] = M_SQRT2 * nl * plm * sm;
            }
        }
    }
}

template <class T>
__global__ void k_basis(int n, int nsh, int beta, const double *phi, const double *dist, T *psi) {
    // psi[k][g]: k < nsh -> phi[g][k]; k >= nsh -> (d^2/2) phi[g][k-nsh]
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    int k = blockIdx.y;
    if (g >= n) return;
    int kk = k < nsh ? k : k - nsh;
    double v = phi[(int64_t)g * nsh + kk];
    if (k >= nsh) v *= 0.5 * dist[g] * dist[g];
    psi[(int64_t)k * n + g] = (T)v;
}

__global__ void k_basis_in(int m, int n, int nsh, const int *gin_pos, const double *phi,
                           const double *dist, double *psi_in) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    int k = blockIdx.y;
    if (r >= m) return;
    int g = gin_pos[r];
    int kk = k < nsh ? k : k - nsh;
    double v = phi[(int64_t)g * nsh + kk];
    if (k >= nsh) v *= 0.5 * dist[g] * dist[g];
    psi_in[(int64_t)k * m + r] = v;
}

bool g_nlm_ready = false;

int ensure_nlm() {
    if (g_nlm_ready) return DPM_OK;
    double tab[(kMaxK + 1) * (kMaxK + 1)] = {0};
    for (int l = 0; l <= kMaxK; ++l)
        for (int m = 0; m <= l; ++m) {
            double r = 1.0;  // (l-m)!/(l+m)!
            for (int t = l - m + 1; t <= l + m; ++t) r /= (double)t;
            tab[l * (kMaxK + 1) + m] = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * r);
        }
    DPM_CUDA(cudaMemcpyToSymbol(c_nlm, tab, sizeof(tab)));
    g_nlm_ready = true;
    return DPM_OK;
}

}  // namespace

int build_gamma_geom(const dpm_geom &g, const GridIndex &gi, int K, GammaGeom &gg,
                     cudaStream_t s) {
    if (K < 0 || K > kMaxK) { set_error("K=%d out of range [0,%d]", K, kMaxK); return DPM_EINVAL; }
    if (g.kind < 0 || g.kind > 2) {
        set_error("geometry kind %d: the single-domain and Case 1 paths take kinds 0-2 (kinds 3/4 are "
                  "the sub-domains of dpm_dd2_*)", g.kind);
        return DPM_EINVAL;
    }
    DPM_RET(ensure_nlm());
    gg.K = K;
    gg.nsh = (K + 1) * (K + 1);
    int64_t n = gi.n_gamma;
    DPM_RET(gg.foot.alloc(sizeof(double) * 3 * n));
    DPM_RET(gg.normal.alloc(sizeof(double) * 3 * n));
    DPM_RET(gg.dist.alloc(sizeof(double) * n));
    DPM_RET(gg.phi.alloc(sizeof(double) * gg.nsh * n));
    double ax = g.axes[0], ay = g.kind == 0 ? g.axes[0] : g.axes[1],
           az = g.kind == 0 ? g.axes[0] : g.axes[2];  // kind 2: (r_out, r_in, -)
    int blocks = (int)((n + 127) / 128);
    k_gamma_geom<<<blocks, 128, 0, s>>>((int)n, gi.N, gi.lo, gi.h, g.kind, g.center[0], g.center[1],
                                        g.center[2], ax, ay, az, K, gi.gamma.as<int>(),
                                        gg.foot.as<double>(), gg.normal.as<double>(),
                                        gg.dist.as<double>(), gg.phi.as<double>());
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int make_basis_densities(const GammaGeom &gg, const GridIndex &gi, int beta, T *psi,
                         double *psi_in, cudaStream_t s) {
    int ncol = (beta + 1) * gg.nsh;
    int64_t n = gi.n_gamma, m = gi.n_gin;
    if (psi) {
        dim3 grid((unsigned)((n + 255) / 256), ncol);
        k_basis<T><<<grid, 256, 0, s>>>((int)n, gg.nsh, beta, gg.phi.as<double>(),
                                        gg.dist.as<double>(), psi);
        DPM_LAUNCHED();
    }
    if (psi_in) {
        dim3 grid((unsigned)((m + 255) / 256), ncol);
        k_basis_in<<<grid, 256, 0, s>>>((int)m, (int)n, gg.nsh, gi.gin_pos.as<int>(),
                                        gg.phi.as<double>(), gg.dist.as<double>(), psi_in);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

template int make_basis_densities<float>(const GammaGeom &, const GridIndex &, int, float *,
                                         double *, cudaStream_t);
template int make_basis_densities<double>(const GammaGeom &, const GridIndex &, int, double *,
                                          double *, cudaStream_t);

}  // namespace dpm
