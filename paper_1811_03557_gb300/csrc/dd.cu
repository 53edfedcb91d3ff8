// Domain decomposition, Case 1 (Section 3): the kernels that are specific to
// two sub-domains coupled through the interface Z.
//
// Omega_1 is the ball |x - c| < r1, Omega_2 the shell r1 < |x - c| < r2, each
// with its own grid.  The unknowns are three spherical-harmonic series on Z
// (u, du/dnu, d2u/dnu2 with nu = (x - c)/|x - c|, shared by both sub-domains:
// the interface conditions) and two on Gamma (u, d2u/dn2; du/dn is the
// Neumann data).  Column k of the stacked BEP (eqs. reduced_DD1_BEP1 and
// reduced_DD1_BEP2) has, on a grid-boundary node whose foot point lies on Z,
// the density phi_nu, s phi_nu or s^2/2 phi_nu (s the signed distance from Z
// along nu), on a node of Gamma phi_nu or d^2/2 phi_nu, and zero on the nodes
// of the other surface.
#include "dpm_internal.cuh"

namespace dpm {

namespace {

// Value of column k at a node with signed distance d, surface flag z (1: Z),
// harmonics ph[0..nsh).
__device__ __forceinline__ double dd_column(int k, int nz, int ng, int z, double d, const double *ph) {
    if (k < 3 * nz) {
        if (!z) return 0.0;
        const int t = k / nz, nu = k % nz;
        const double fac = t == 0 ? 1.0 : (t == 1 ? d : 0.5 * d * d);
        return fac * ph[nu];
    }
    if (z) return 0.0;
    const int k2 = k - 3 * nz;
    const int t = k2 / ng, nu = k2 % ng;
    return (t == 0 ? 1.0 : 0.5 * d * d) * ph[nu];
}

__global__ void k_dd_surf(int n, const double *foot, double cx, double cy, double cz, double r_mid,
                          uint8_t *surf) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double *f = foot + 3 * (size_t)e;
    const double x = f[0] - cx, y = f[1] - cy, z = f[2] - cz;
    surf[e] = sqrt(x * x + y * y + z * z) < r_mid ? 1 : 0;
}

template <class T>
__global__ void k_dd_psi(int n, int nsh, int nz, int ng, const double *phi, const double *dist,
                         const uint8_t *surf, T *psi) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (e >= n) return;
    psi[(size_t)k * n + e] = (T)dd_column(k, nz, ng, surf[e], dist[e], phi + (size_t)e * nsh);
}

__global__ void k_dd_psi_in(int m, int nsh, int nz, int ng, const int *gin_pos, const double *phi,
                            const double *dist, const uint8_t *surf, double *psi_in) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (r >= m) return;
    const int e = gin_pos[r];
    psi_in[(size_t)k * m + r] = dd_column(k, nz, ng, surf[e], dist[e], phi + (size_t)e * nsh);
}

// Stacked BEP (column-major, m1 + m2 rows): rows of Omega_1 then of Omega_2;
// Omega_1 has only the Z columns (k < nzc).
template <class T>
__global__ void k_dd_assemble(int m1, int m2, int nzc, int ncol, const double *psi_in1, const T *tr1,
                              const double *psi_in2, const T *tr2, double *A) {
    const int m = m1 + m2;
    const int64_t total = (int64_t)m * ncol;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(q / m), r = (int)(q % m);
        double v;
        if (r < m1) {
            v = k < nzc ? psi_in1[(size_t)k * m1 + r] - (double)tr1[(size_t)k * m1 + r] : 0.0;
        } else {
            const int r2 = r - m1;
            v = psi_in2[(size_t)k * m2 + r2] - (double)tr2[(size_t)k * m2 + r2];
        }
        A[q] = v;
    }
}

// u on the grid boundary of one sub-domain from the coefficients (nr sets,
// stride ldc): one warp per node, FP64 sums; + d g_N on Gamma nodes when
// neumann is given; optional clamp at 0.
template <class T>
__global__ void k_dd_extend(int n, int nsh, int nz, int ng, const double *phi, const double *dist,
                            const uint8_t *surf, const double *C, int ldc, const double *neumann,
                            T *dens, int ldd, int nr, int clamp) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double *ph = phi + (size_t)warp * nsh;
    const double d = dist[warp];
    const int z = surf[warp];
    for (int q = 0; q < nr; ++q) {
        const double *cq = C + (size_t)q * ldc;
        double s = 0.0;
        if (z) {
            for (int nu = lane; nu < nz; nu += 32)
                s += (cq[nu] + d * cq[nz + nu] + 0.5 * d * d * cq[2 * nz + nu]) * ph[nu];
        } else {
            for (int nu = lane; nu < ng; nu += 32)
                s += (cq[3 * nz + nu] + 0.5 * d * d * cq[3 * nz + ng + nu]) * ph[nu];
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            double u = s;
            if (!z && neumann) u += d * neumann[warp];
            if (clamp && u < 0.0) u = 0.0;
            dens[(size_t)q * ldd + warp] = (T)u;
        }
    }
}

// d g_N on the Gamma nodes of the shell, zero on its Z nodes.
template <class T>
__global__ void k_dd_neumann_dens(int n, const double *dist, const uint8_t *surf, const double *gn,
                                  T *v) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    v[e] = surf[e] ? (T)0 : (T)(dist[e] * gn[e]);
}

// b = [tr_p1 ; tr_p2 - (v|in - tr_v2)] for one right-hand side (the last term
// only with Neumann data).
template <class T>
__global__ void k_dd_rhs(int m1, int m2, const T *tr_p1, const T *tr_p2, const T *v, const int *gin_pos2,
                         const T *tr_v2, T *b) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m1 + m2) return;
    if (r < m1) {
        b[r] = tr_p1[r];
    } else {
        const int r2 = r - m1;
        T x = tr_p2[r2];
        if (v) x -= v[gin_pos2[r2]] - tr_v2[r2];
        b[r] = x;
    }
}

}  // namespace

int dd_surface_flags(int64_t n, const double *foot, const double c[3], double r_mid, uint8_t *surf,
                     cudaStream_t s) {
    if (n == 0) return DPM_OK;
    k_dd_surf<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((int)n, foot, c[0], c[1], c[2], r_mid, surf);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int dd_columns(int64_t n, int64_t m, int nsh, int nz, int ng, int ncol_l, const double *phi,
               const double *dist, const uint8_t *surf, const int *gin_pos, T *psi, double *psi_in,
               cudaStream_t s) {
    if (n > 0) {
        k_dd_psi<T><<<dim3((unsigned)((n + 255) / 256), ncol_l), 256, 0, s>>>((int)n, nsh, nz, ng, phi,
                                                                             dist, surf, psi);
        DPM_LAUNCHED();
    }
    if (m > 0) {
        k_dd_psi_in<<<dim3((unsigned)((m + 255) / 256), ncol_l), 256, 0, s>>>((int)m, nsh, nz, ng, gin_pos,
                                                                              phi, dist, surf, psi_in);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

template <class T>
int dd_assemble(int64_t m1, int64_t m2, int nzc, int ncol, const double *psi_in1, const T *tr1,
                const double *psi_in2, const T *tr2, double *A, cudaStream_t s) {
    k_dd_assemble<T><<<4 * 152, 256, 0, s>>>((int)m1, (int)m2, nzc, ncol, psi_in1, tr1, psi_in2, tr2, A);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int dd_extend(int64_t n, int nsh, int nz, int ng, const double *phi, const double *dist,
              const uint8_t *surf, const double *C, int ldc, const double *neumann, T *dens, int ldd,
              int nr, int clamp, cudaStream_t s) {
    if (n == 0) return DPM_OK;
    const int64_t threads = n * 32;
    k_dd_extend<T><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>((int)n, nsh, nz, ng, phi, dist, surf,
                                                                      C, ldc, neumann, dens, ldd, nr, clamp);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int dd_neumann_density(int64_t n, const double *dist, const uint8_t *surf, const double *gn, T *v,
                       cudaStream_t s) {
    if (n == 0) return DPM_OK;
    k_dd_neumann_dens<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>((int)n, dist, surf, gn, v);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int dd_rhs(int64_t m1, int64_t m2, const T *tr_p1, const T *tr_p2, const T *v, const int *gin_pos2,
           const T *tr_v2, T *b, cudaStream_t s) {
    const int64_t m = m1 + m2;
    k_dd_rhs<T><<<(unsigned)((m + 255) / 256), 256, 0, s>>>((int)m1, (int)m2, tr_p1, tr_p2, v, gin_pos2,
                                                            tr_v2, b);
    DPM_LAUNCHED();
    return DPM_OK;
}

#define DD_INST(T)                                                                                     \
    template int dd_columns<T>(int64_t, int64_t, int, int, int, int, const double *, const double *,   \
                               const uint8_t *, const int *, T *, double *, cudaStream_t);             \
    template int dd_assemble<T>(int64_t, int64_t, int, int, const double *, const T *, const double *, \
                                const T *, double *, cudaStream_t);                                    \
    template int dd_extend<T>(int64_t, int, int, int, const double *, const double *, const uint8_t *, \
                              const double *, int, const double *, T *, int, int, int, cudaStream_t);   \
    template int dd_neumann_density<T>(int64_t, const double *, const uint8_t *, const double *, T *,  \
                                       cudaStream_t);                                                  \
    template int dd_rhs<T>(int64_t, int64_t, const T *, const T *, const T *, const int *, const T *,  \
                           T *, cudaStream_t);
DD_INST(float)
DD_INST(double)
#undef DD_INST

}  // namespace dpm
