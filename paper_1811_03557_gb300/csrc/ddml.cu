// Layered domain decomposition (Section 3's Case 1 with more than one
// interface): the ball |x - c| < rho_1 and the shells rho_l < |x - c| < rho_{l+1}
// (rho_L = R), each on its own grid.  Sphere m (1..L; m = L is Gamma) carries
// its series: three terms (u, du/dnu, d2u/dnu2, nu = (x - c)/|x - c|) of n_m
// harmonics on an interface, two (u, d2u/dn2) on Gamma.  A sub-domain's
// grid-boundary node belongs to one sphere (the nearer of the shell's two; the
// ball's only one), with s = |x - c| - rho_m; column k = (sphere m, term t,
// harmonic nu) has the density {1, s, s^2/2}[t] phi_nu (Gamma: {1, s^2/2}[t])
// on the nodes of sphere m and zero elsewhere.
#include <algorithm>

#include "dpm_internal.cuh"

namespace dpm {

namespace {

__device__ __forceinline__ void column_of(const MlColumns &cm, int k, int *m, int *t, int *nu) {
    int q = 1;
    while (q < cm.L && k >= cm.off[q]) ++q;  // sphere q: columns [off[q-1], off[q])
    const int r = k - cm.off[q - 1];
    *m = q;
    *t = r / cm.n[q - 1];
    *nu = r % cm.n[q - 1];
}

__device__ __forceinline__ double column_value(const MlColumns &cm, int k, int m_node, double s, const double *ph) {
    int m, t, nu;
    column_of(cm, k, &m, &t, &nu);
    if (m != m_node) return 0.0;
    const double fac = m < cm.L ? (t == 0 ? 1.0 : (t == 1 ? s : 0.5 * s * s)) : (t == 0 ? 1.0 : 0.5 * s * s);
    return fac * ph[nu];
}

// psi[j][e] (local column j = global column cols[j]) and psi_in[j][r] at gamma_in.
template <class T>
__global__ void k_ml_psi(int n, int nsh, MlColumns cm, const int *cols, const uint8_t *sphere, const double *dist,
                         const double *phi, T *psi) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (e >= n) return;
    psi[(size_t)j * n + e] = (T)column_value(cm, cols[j], sphere[e], dist[e], phi + (size_t)e * nsh);
}

__global__ void k_ml_psi_in(int m, int nsh, MlColumns cm, const int *cols, const int *gin_pos, const uint8_t *sphere,
                            const double *dist, const double *phi, double *psi_in) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (r >= m) return;
    const int e = gin_pos[r];
    psi_in[(size_t)j * m + r] = column_value(cm, cols[j], sphere[e], dist[e], phi + (size_t)e * nsh);
}

// A[cols[j]][row0 + r] = psi_in[j][r] - trace[j][r]  (A column-major, ld = mtot; zeroed before)
template <class T>
__global__ void k_ml_assemble(int m, int ncl, int64_t mtot, int64_t row0, const int *cols, const double *psi_in,
                              const T *trace, double *A) {
    const int64_t total = (int64_t)m * ncl;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / m), r = (int)(q % m);
        A[(int64_t)cols[j] * mtot + row0 + r] = psi_in[q] - (double)trace[q];
    }
}

// u on the grid boundary from the coefficients (nr sets, stride ldc): one warp per
// node over its sphere's series; + s g_N on Gamma nodes when gn is given; clamp.
constexpr int kMlExtQ = 4;  // right-hand sides per pass over the FP32 table

template <class T>
__global__ void k_ml_extend(int n, int nsh, MlColumns cm, const uint8_t *sphere, const double *dist, const double *phi,
                            const double *C, int ldc, const double *gn, T *dens, int ldd, int nr, int clamp) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int e = warp, m = sphere[e];
    const double s = dist[e];
    const double *ph = phi + (size_t)e * nsh;
    const int nm = cm.n[m - 1], o = cm.off[m - 1];
    for (int q = 0; q < nr; ++q) {
        const double *cq = C + (size_t)q * ldc + o;
        double acc = 0.0;
        if (m < cm.L) {
            for (int nu = lane; nu < nm; nu += 32)
                acc += (cq[nu] + s * cq[nm + nu] + 0.5 * s * s * cq[2 * nm + nu]) * ph[nu];
        } else {
            for (int nu = lane; nu < nm; nu += 32) acc += (cq[nu] + 0.5 * s * s * cq[nm + nu]) * ph[nu];
        }
        for (int w = 16; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
        if (lane == 0) {
            double u = acc;
            if (m == cm.L && gn) u += s * gn[e];
            if (clamp && u < 0.0) u = 0.0;
            dens[(size_t)q * ldd + e] = (T)u;
        }
    }
}

// FP32 paths: one thread per grid-boundary node, its sphere's harmonics in
// order from the transposed FP32 table (coalesced loads), the coefficients of
// the block's spheres mlo..mhi converted to FP32 in shared memory; the three
// series (two on Gamma) are summed separately in FP32 and combined in FP64,
// as the single-domain extension does.
template <class T>
__global__ void k_ml_extend32(int n, MlColumns cm, int mlo, int mhi, const uint8_t *sphere, const double *dist,
                              const float *__restrict__ phit, const double *__restrict__ C, int ldc,
                              const double *gn, T *dens, int ldd, int nr, int clamp) {
    extern __shared__ float cs32[];
    const int c0 = cm.off[mlo - 1], ncs = cm.off[mhi] - c0;
    for (int i = threadIdx.x; i < nr * ncs; i += blockDim.x) cs32[i] = (float)C[(size_t)(i / ncs) * ldc + c0 + i % ncs];
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int m = sphere[g], nm = cm.n[m - 1], base = cm.off[m - 1] - c0;
    const bool gam = m == cm.L;  // Gamma: u and d^2u/dn^2 only
    const double d = dist[g];
    for (int q0 = 0; q0 < nr; q0 += kMlExtQ) {
        const int nq = min(kMlExtQ, nr - q0);
        float s0[kMlExtQ] = {}, s1[kMlExtQ] = {}, s2[kMlExtQ] = {};
        for (int nu = 0; nu < nm; ++nu) {
            const float f = phit[(size_t)nu * n + g];
#pragma unroll
            for (int q = 0; q < kMlExtQ; ++q)
                if (q < nq) {
                    const float *cp = cs32 + (size_t)(q0 + q) * ncs + base;
                    s0[q] = fmaf(cp[nu], f, s0[q]);
                    if (gam) {
                        s2[q] = fmaf(cp[nm + nu], f, s2[q]);
                    } else {
                        s1[q] = fmaf(cp[nm + nu], f, s1[q]);
                        s2[q] = fmaf(cp[2 * nm + nu], f, s2[q]);
                    }
                }
        }
#pragma unroll
        for (int q = 0; q < kMlExtQ; ++q)
            if (q < nq) {
                double u = (double)s0[q] + d * (double)s1[q] + 0.5 * d * d * (double)s2[q];
                if (gam && gn) u += d * gn[g];
                if (clamp && u < 0.0) u = 0.0;
                dens[(size_t)(q0 + q) * ldd + g] = (T)u;
            }
    }
}

// sphere index of each grid-boundary node from its foot point: the ball's nodes
// all lie on sphere 1; a shell's on its inner sphere m_in or outer m_in + 1.
__global__ void k_ml_sphere(int n, const double *foot, double cx, double cy, double cz, double r_mid, int m_in,
                            int ball, uint8_t *sphere) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    if (ball) {
        sphere[e] = 1;
        return;
    }
    const double *f = foot + 3 * (size_t)e;
    const double x = f[0] - cx, y = f[1] - cy, z = f[2] - cz;
    sphere[e] = (uint8_t)(sqrt(x * x + y * y + z * z) < r_mid ? m_in : m_in + 1);
}

// d g_N on the Gamma nodes (sphere L), zero elsewhere.
template <class T>
__global__ void k_ml_neumann(int n, int L, const uint8_t *sphere, const double *dist, const double *gn, T *v) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    v[e] = sphere[e] == L ? (T)(dist[e] * gn[e]) : (T)0;
}

// b[row0 + r] = tr_p[r] - (v|gamma_in - tr_v)[r] (the last term with Neumann data only)
template <class T>
__global__ void k_ml_rhs(int m, const T *trp, const T *v, const int *gin_pos, const T *trv, T *b) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    T x = trp[r];
    if (v) x -= v[gin_pos[r]] - trv[r];
    b[r] = x;
}

unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int ml_sphere_flags(int64_t n, const double *foot, const double c[3], double r_mid, int m_in, int ball,
                    uint8_t *sphere, cudaStream_t s) {
    if (n == 0) return DPM_OK;
    k_ml_sphere<<<nblk(n, 256), 256, 0, s>>>((int)n, foot, c[0], c[1], c[2], r_mid, m_in, ball, sphere);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int ml_columns(int64_t n, int64_t m, int nsh, const MlColumns &cm, int ncl, const int *cols, const uint8_t *sphere,
               const double *dist, const double *phi, const int *gin_pos, T *psi, double *psi_in, cudaStream_t s) {
    if (n > 0 && ncl > 0) {
        k_ml_psi<T><<<dim3(nblk(n, 256), ncl), 256, 0, s>>>((int)n, nsh, cm, cols, sphere, dist, phi, psi);
        DPM_LAUNCHED();
    }
    if (m > 0 && ncl > 0) {
        k_ml_psi_in<<<dim3(nblk(m, 256), ncl), 256, 0, s>>>((int)m, nsh, cm, cols, gin_pos, sphere, dist, phi, psi_in);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

template <class T>
int ml_assemble(int64_t m, int ncl, int64_t mtot, int64_t row0, const int *cols, const double *psi_in, const T *trace,
                double *A, cudaStream_t s) {
    if (m == 0 || ncl == 0) return DPM_OK;
    k_ml_assemble<T><<<4 * 152, 256, 0, s>>>((int)m, ncl, mtot, row0, cols, psi_in, trace, A);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int ml_extend(int64_t n, int nsh, const MlColumns &cm, const uint8_t *sphere, const double *dist, const double *phi,
              const float *phit, int mlo, int mhi, const double *C, int ldc, const double *gn, T *dens, int ldd,
              int nr, int clamp, cudaStream_t s) {
    if (n == 0) return DPM_OK;
    if (phit && sizeof(T) == 4) {
        // right-hand sides in groups whose FP32 coefficients fit in 48 KB of shared memory
        const size_t per = sizeof(float) * (size_t)(cm.off[mhi] - cm.off[mlo - 1]);
        const int grp = (int)std::max<size_t>(1, (48 * 1024) / std::max<size_t>(per, 1));
        for (int q0 = 0; q0 < nr; q0 += grp) {
            const int nq = std::min(grp, nr - q0);
            k_ml_extend32<T><<<nblk(n, 128), 128, per * nq, s>>>((int)n, cm, mlo, mhi, sphere, dist, phit,
                                                                 C + (size_t)q0 * ldc, ldc, gn,
                                                                 dens + (size_t)q0 * ldd, ldd, nq, clamp);
            DPM_LAUNCHED();
        }
        return DPM_OK;
    }
    k_ml_extend<T><<<nblk(n * 32, 256), 256, 0, s>>>((int)n, nsh, cm, sphere, dist, phi, C, ldc, gn, dens, ldd, nr,
                                                     clamp);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int ml_neumann(int64_t n, int L, const uint8_t *sphere, const double *dist, const double *gn, T *v, cudaStream_t s) {
    if (n == 0) return DPM_OK;
    k_ml_neumann<T><<<nblk(n, 256), 256, 0, s>>>((int)n, L, sphere, dist, gn, v);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int ml_rhs(int64_t m, const T *trp, const T *v, const int *gin_pos, const T *trv, T *b, cudaStream_t s) {
    if (m == 0) return DPM_OK;
    k_ml_rhs<T><<<nblk(m, 256), 256, 0, s>>>((int)m, trp, v, gin_pos, trv, b);
    DPM_LAUNCHED();
    return DPM_OK;
}

#define ML_INST(T)                                                                                               \
    template int ml_columns<T>(int64_t, int64_t, int, const MlColumns &, int, const int *, const uint8_t *,       \
                               const double *, const double *, const int *, T *, double *, cudaStream_t);        \
    template int ml_assemble<T>(int64_t, int, int64_t, int64_t, const int *, const double *, const T *, double *, \
                                cudaStream_t);                                                                   \
    template int ml_extend<T>(int64_t, int, const MlColumns &, const uint8_t *, const double *, const double *,    \
                              const float *, int, int, const double *, int, const double *, T *, int, int, int,  \
                              cudaStream_t);                                                                     \
    template int ml_neumann<T>(int64_t, int, const uint8_t *, const double *, const double *, T *, cudaStream_t); \
    template int ml_rhs<T>(int64_t, const T *, const T *, const int *, const T *, T *, cudaStream_t);
ML_INST(float)
ML_INST(double)
#undef ML_INST

}  // namespace dpm
