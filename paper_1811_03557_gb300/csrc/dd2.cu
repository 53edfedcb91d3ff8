// Domain decomposition, Case 2 (Section 3): the kernels specific to an
// interface Z that meets Gamma.
//
// Omega is the sphere |x - c| < R, Z the sphere |x - c_Z| = rz.  On each
// sub-domain's grid (local frame) a grid-boundary node carries a Gamma value,
// a Z value, or both (the wedge layer): flag bit 0 = Gamma, bit 1 = Z.  Its
// effective density is the mean of the values it carries; every node of
// gamma_in gives one BEP row per surface (eq. reduced_DD2_BEP).  Unknown k:
// k < 3 MZ is term t = k / MZ, harmonic nu = k % MZ of the Z series (value
// {1, s, s^2/2}[t] Y_nu(cos theta_Z), s = |x - c_Z| - rz); else term
// t = (k - 3 MZ) / MG of the Gamma series ({1, d^2/2}[t] Y_nu(cos theta_G); t = 0 only
// with one Gamma series, the 2-term extension u + d g_N,
// d = |x - c| - R), with the zonal harmonics Y_nu = sqrt((2 nu + 1)/(4 pi)) P_nu.
// On Z the argument of P_nu is cos theta_Z mapped from the range that the part
// of Z inside Omega spans to [-1, 1]: the same polynomials of degree < MZ in
// cos theta_Z, in a basis that stays well conditioned on the partial sphere.
#include "dpm_internal.cuh"

namespace dpm {

namespace {

__device__ __forceinline__ double node_coord(double lo, double h, int j) {
    return __dadd_rn(lo, __dmul_rn((double)(j + 1), h));
}

// |p - c| as sqrt((qx^2 + qy^2) + qz^2), q = p - c.
__device__ __forceinline__ double radial(const double p[3], const double c[3], double q[3]) {
    for (int t = 0; t < 3; ++t) q[t] = __dsub_rn(p[t], c[t]);
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(q[0], q[0]), __dmul_rn(q[1], q[1])), __dmul_rn(q[2], q[2])));
}

__global__ void k_dd2_split(int n, int N, double lo, double h, const int *gamma, const uint8_t *lab_o,
                            const uint8_t *lab_b, double c0x, double c0y, double c0z, double R, double czx,
                            double czy, double czz, double rz, uint8_t *flags, double *dG, double *dZ,
                            double *cosG, double *cosZ, double *footG, double *footZ) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int p = gamma[e];
    const int k = p % N, j = (p / N) % N, i = p / (N * N);
    const double P[3] = {node_coord(lo, h, i), node_coord(lo, h, j), node_coord(lo, h, k)};
    const double c0[3] = {c0x, c0y, c0z}, cz[3] = {czx, czy, czz};
    double qg[3], qz[3];
    const double rg = radial(P, c0, qg), rzz = radial(P, cz, qz);
    const double dg = rg - R, dz = rzz - rz;
    const uint8_t gb = DPM_LBL_GIN | DPM_LBL_GEX;
    uint8_t f = (uint8_t)(((lab_o[p] & gb) ? 1 : 0) | ((lab_b[p] & gb) ? 2 : 0));
    if (!f) f = fabs(dg) <= fabs(dz) ? 1 : 2;
    flags[e] = f;
    dG[e] = dg;
    dZ[e] = dz;
    cosG[e] = rg > 0.0 ? qg[2] / rg : 1.0;  // a node at a centre carries no value of that sphere
    cosZ[e] = rzz > 0.0 ? qz[2] / rzz : 1.0;
    for (int t = 0; t < 3; ++t) {
        footG[3 * (size_t)e + t] = rg > 0.0 ? c0[t] + R * (qg[t] / rg) : c0[t];
        footZ[3 * (size_t)e + t] = rzz > 0.0 ? cz[t] + rz * (qz[t] / rzz) : cz[t];
    }
}

// Y_nu(t) = sqrt((2 nu + 1)/(4 pi)) P_nu(t), nu < M, Bonnet's recurrence in FP64,
// at t = (2 x - (a + b))/(b - a): x mapped from [a, b] to [-1, 1].
__global__ void k_zonal(int n, int M, const double *x, double a, double b, double *Y) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double c = (2.0 * x[e] - (a + b)) / (b - a);
    double pm = 1.0, p = c;  // P_0, P_1
    double *y = Y + (size_t)e * M;
    const double inv4pi = 0.25 / 3.14159265358979323846;
    y[0] = sqrt(inv4pi);
    if (M > 1) y[1] = sqrt(3.0 * inv4pi) * c;
    for (int nu = 1; nu + 1 < M; ++nu) {
        const double pn = ((2.0 * nu + 1.0) * c * p - nu * pm) / (nu + 1.0);
        pm = p;
        p = pn;
        y[nu + 1] = sqrt((2.0 * nu + 3.0) * inv4pi) * pn;
    }
}

// Value of unknown k at node e as surface `surf` (0 Gamma, 1 Z) gives it.
__device__ __forceinline__ double col_value(int k, int surf, int e, int MZ, int MG, const double *dG,
                                            const double *dZ, const double *YG, const double *YZ) {
    if (k < 3 * MZ) {
        if (surf == 0) return 0.0;
        const int t = k / MZ, nu = k % MZ;
        const double s = dZ[e];
        const double fac = t == 0 ? 1.0 : (t == 1 ? s : 0.5 * s * s);
        return fac * YZ[(size_t)e * MZ + nu];
    }
    if (surf == 1) return 0.0;
    const int k2 = k - 3 * MZ, t = k2 / MG, nu = k2 % MG;
    const double d = dG[e];
    return (t == 0 ? 1.0 : 0.5 * d * d) * YG[(size_t)e * MG + nu];
}

__device__ __forceinline__ double wedge_mean(uint8_t f, double vg, double vz) {
    return f == 3 ? 0.5 * (vg + vz) : (f == 1 ? vg : vz);
}

// Effective column densities psi[k][e] (the AP right-hand side densities).
template <class T>
__global__ void k_dd2_psi(int n, int MZ, int MG, const uint8_t *flags, const double *dG, const double *dZ,
                          const double *YG, const double *YZ, T *psi) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (e >= n) return;
    const uint8_t f = flags[e];
    const double vg = (f & 1) ? col_value(k, 0, e, MZ, MG, dG, dZ, YG, YZ) : 0.0;
    const double vz = (f & 2) ? col_value(k, 1, e, MZ, MG, dG, dZ, YG, YZ) : 0.0;
    psi[(size_t)k * n + e] = (T)wedge_mean(f, vg, vz);
}

// Row values own[k][r]: column k at row r's node as row r's surface gives it.
__global__ void k_dd2_rows(int m, int MZ, int MG, const int *row_e, const uint8_t *row_s, const double *dG,
                           const double *dZ, const double *YG, const double *YZ, double *own) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (r >= m) return;
    own[(size_t)k * m + r] = col_value(k, row_s[r], row_e[r], MZ, MG, dG, dZ, YG, YZ);
}

// Stacked BEP (column-major, rows of sub-domain 0 then 1):
// A[k][off_l + r] = own_l[k][r] - trace_l[k][row_i_l[r]].
template <class T>
__global__ void k_dd2_assemble(int m1, int m2, int ncol, const double *own1, const T *tr1, int g1,
                               const int *ri1, const double *own2, const T *tr2, int g2, const int *ri2,
                               double *A) {
    const int m = m1 + m2;
    const int64_t total = (int64_t)m * ncol;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(q / m), r = (int)(q % m);
        A[q] = r < m1 ? own1[(size_t)k * m1 + r] - (double)tr1[(size_t)k * g1 + ri1[r]]
                      : own2[(size_t)k * m2 + (r - m1)] - (double)tr2[(size_t)k * g2 + ri2[r - m1]];
    }
}

// b[r] = trace_p[row_i[r]] - (vG at a Gamma row - trace_v[row_i[r]]) for one
// right-hand side of one sub-domain; the Neumann part only when vG is given.
template <class T>
__global__ void k_dd2_rhs(int m, const int *row_i, const int *row_e, const uint8_t *row_s, const T *trp,
                          const double *vG, const T *trv, T *b) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    double x = (double)trp[row_i[r]];
    if (vG) x -= (row_s[r] == 0 ? vG[row_e[r]] : 0.0) - (double)trv[row_i[r]];
    b[r] = (T)x;
}

// Neumann density: vG[e] = d g_N on Gamma nodes (0 elsewhere) and its effective
// (wedge-averaged) value as an AP density.
template <class T>
__global__ void k_dd2_neumann(int n, const uint8_t *flags, const double *dG, const double *gn, double *vG,
                              T *veff) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const uint8_t f = flags[e];
    const double v = (f & 1) ? dG[e] * gn[e] : 0.0;
    vG[e] = v;
    veff[e] = (T)wedge_mean(f, v, 0.0);
}

// Effective density from the coefficients (nr sets, stride ldc): one warp per
// node, FP64 sums over the harmonics of each series it carries, + d g_N on
// Gamma values when gn is given, the wedge mean, optional clamp at 0.
template <class T>
__global__ void k_dd2_extend(int n, int MZ, int MG, int GS, const uint8_t *flags, const double *dG, const double *dZ,
                             const double *YG, const double *YZ, const double *C, int ldc, const double *gn,
                             T *dens, int ldd, int nr, int clamp) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int e = warp;
    const uint8_t f = flags[e];
    const double s = dZ[e], d = dG[e];
    const double *yz = YZ + (size_t)e * MZ, *yg = YG + (size_t)e * MG;
    for (int q = 0; q < nr; ++q) {
        const double *cq = C + (size_t)q * ldc;
        double sz = 0.0, sg = 0.0;
        if (f & 2)
            for (int nu = lane; nu < MZ; nu += 32)
                sz += (cq[nu] + s * cq[MZ + nu] + 0.5 * s * s * cq[2 * MZ + nu]) * yz[nu];
        if (f & 1)
            for (int nu = lane; nu < MG; nu += 32)
                sg += (cq[3 * MZ + nu] + (GS == 2 ? 0.5 * d * d * cq[3 * MZ + MG + nu] : 0.0)) * yg[nu];
        for (int o = 16; o > 0; o >>= 1) {
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
            sg += __shfl_xor_sync(0xffffffffu, sg, o);
        }
        if (lane == 0) {
            if ((f & 1) && gn) sg += d * gn[e];
            double u = wedge_mean(f, sg, sz);
            if (clamp && u < 0.0) u = 0.0;
            dens[(size_t)q * ldd + e] = (T)u;
        }
    }
}

// The foot point a gamma_ex node takes its initial data from: on Gamma when the
// node carries a Gamma value, else on Z.
__global__ void k_dd2_init_foot(int n, const uint8_t *flags, const double *footG, const double *footZ,
                                double *foot) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double *src = (flags[e] & 1) ? footG : footZ;
    for (int t = 0; t < 3; ++t) foot[3 * (size_t)e + t] = src[3 * (size_t)e + t];
}

unsigned blocks1(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int dd2_split(const GridIndex &gi, const uint8_t *lab_o, const uint8_t *lab_b, const double c0[3], double R,
              const double cz[3], double rz, uint8_t *flags, double *dG, double *dZ, double *cosG,
              double *cosZ, double *footG, double *footZ, cudaStream_t s) {
    const int64_t n = gi.n_gamma;
    if (n == 0) return DPM_OK;
    k_dd2_split<<<blocks1(n, 128), 128, 0, s>>>((int)n, gi.N, gi.lo, gi.h, gi.gamma.as<int>(), lab_o, lab_b,
                                                c0[0], c0[1], c0[2], R, cz[0], cz[1], cz[2], rz, flags, dG,
                                                dZ, cosG, cosZ, footG, footZ);
    DPM_LAUNCHED();
    return DPM_OK;
}

int dd2_zonal(int64_t n, int M, const double *x, double a, double b, double *Y, cudaStream_t s) {
    if (n == 0) return DPM_OK;
    k_zonal<<<blocks1(n, 128), 128, 0, s>>>((int)n, M, x, a, b, Y);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int dd2_columns(int64_t n, int64_t m, int MZ, int MG, int GS, const uint8_t *flags, const double *dG,
                const double *dZ, const double *YG, const double *YZ, const int *row_e, const uint8_t *row_s,
                T *psi, double *own, cudaStream_t s) {
    const int ncol = 3 * MZ + GS * MG;
    if (n > 0) {
        k_dd2_psi<T><<<dim3(blocks1(n, 256), ncol), 256, 0, s>>>((int)n, MZ, MG, flags, dG, dZ, YG, YZ, psi);
        DPM_LAUNCHED();
    }
    if (m > 0) {
        k_dd2_rows<<<dim3(blocks1(m, 256), ncol), 256, 0, s>>>((int)m, MZ, MG, row_e, row_s, dG, dZ, YG, YZ,
                                                               own);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

template <class T>
int dd2_assemble(int64_t m1, int64_t m2, int ncol, const double *own1, const T *tr1, int64_t g1,
                 const int *ri1, const double *own2, const T *tr2, int64_t g2, const int *ri2, double *A,
                 cudaStream_t s) {
    k_dd2_assemble<T><<<4 * 152, 256, 0, s>>>((int)m1, (int)m2, ncol, own1, tr1, (int)g1, ri1, own2, tr2,
                                              (int)g2, ri2, A);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int dd2_rhs(int64_t m, const int *row_i, const int *row_e, const uint8_t *row_s, const T *trp,
            const double *vG, const T *trv, T *b, cudaStream_t s) {
    if (m == 0) return DPM_OK;
    k_dd2_rhs<T><<<blocks1(m, 256), 256, 0, s>>>((int)m, row_i, row_e, row_s, trp, vG, trv, b);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int dd2_neumann(int64_t n, const uint8_t *flags, const double *dG, const double *gn, double *vG, T *veff,
                cudaStream_t s) {
    if (n == 0) return DPM_OK;
    k_dd2_neumann<T><<<blocks1(n, 256), 256, 0, s>>>((int)n, flags, dG, gn, vG, veff);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int dd2_extend(int64_t n, int MZ, int MG, int GS, const uint8_t *flags, const double *dG, const double *dZ,
               const double *YG, const double *YZ, const double *C, int ldc, const double *gn, T *dens,
               int ldd, int nr, int clamp, cudaStream_t s) {
    if (n == 0) return DPM_OK;
    k_dd2_extend<T><<<blocks1(n * 32, 256), 256, 0, s>>>((int)n, MZ, MG, GS, flags, dG, dZ, YG, YZ, C, ldc, gn,
                                                         dens, ldd, nr, clamp);
    DPM_LAUNCHED();
    return DPM_OK;
}

int dd2_init_foot(int64_t n, const uint8_t *flags, const double *footG, const double *footZ, double *foot,
                  cudaStream_t s) {
    if (n == 0) return DPM_OK;
    k_dd2_init_foot<<<blocks1(n, 256), 256, 0, s>>>((int)n, flags, footG, footZ, foot);
    DPM_LAUNCHED();
    return DPM_OK;
}

#define DD2_INST(T)                                                                                        \
    template int dd2_columns<T>(int64_t, int64_t, int, int, int, const uint8_t *, const double *,           \
                                const double *, const double *, const double *, const int *, const uint8_t *, \
                                T *, double *, cudaStream_t);                                              \
    template int dd2_assemble<T>(int64_t, int64_t, int, const double *, const T *, int64_t, const int *,     \
                                 const double *, const T *, int64_t, const int *, double *, cudaStream_t);  \
    template int dd2_rhs<T>(int64_t, const int *, const int *, const uint8_t *, const T *, const double *,  \
                            const T *, T *, cudaStream_t);                                                 \
    template int dd2_neumann<T>(int64_t, const uint8_t *, const double *, const double *, double *, T *,    \
                                cudaStream_t);                                                             \
    template int dd2_extend<T>(int64_t, int, int, int, const uint8_t *, const double *, const double *,     \
                               const double *, const double *, const double *, int, const double *, T *,   \
                               int, int, int, cudaStream_t);
DD2_INST(float)
DD2_INST(double)
#undef DD2_INST

}  // namespace dpm
