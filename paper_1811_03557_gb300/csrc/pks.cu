// PKS step kernels and the BEP assembly / extension helpers.
//
//  * k_flux: the convective term g of eq. discrete_convective_term on M^+,
//    with face gradients of c by eq. c-central-difference, face densities
//    upwinded (eq. upwind_approximation) from the piecewise-linear
//    reconstruction (eq. truncated_taylor_expansion) with minmod slopes
//    (eq. slope_limiter); a slope whose stencil leaves N^+ is 0.  Then the
//    IMEX right-hand sides of eq. discrete_chemotaxis (alpha = gamma_rho =
//    gamma_c = 1): f_rho = rho - dt g, f_c = (1 - dt) c + dt rho.
//  * k_cfl: max over M^+ of |grad_h c| at the j +- 1/2 faces per axis
//    (eq. cfl_condition).
//  * k_diag: mass, max/min, second moment (eq. sd-norm:second-moment) and
//    free energy (eq. sd-norm:free-energy), per-block FP64 partial sums
//    reduced in a fixed order.
//  * extension: u_gamma = sum C0 phi + beta (d^2/2) sum C2 phi + d g_N
//    (eqs. extension_operator, extension_operator_recast): FP32 paths one
//    thread per node of gamma over a transposed FP32 table, the FP64 path one
//    warp per node with a shuffle reduction over the harmonics.
#include <math.h>

#include <algorithm>

#include "dpm_internal.cuh"

namespace dpm {
namespace {

__device__ __forceinline__ bool in_np(uint8_t l) { return l & (DPM_LBL_MPLUS | DPM_LBL_GEX); }

// (i, j, k) of node p = (i N + j) N + k in 32-bit arithmetic (N^3 < 2^32; a
// 64-bit division costs about ten times as many instructions)
__device__ __forceinline__ void node_ijk(int64_t p, int N, int &i, int &j, int &k) {
    const unsigned q = (unsigned)p, n = (unsigned)N, ij = q / n, ii = ij / n;
    k = (int)(q - ij * n);
    j = (int)(ij - ii * n);
    i = (int)ii;
}

template <class T> __device__ __forceinline__ T minmod3(T a, T b, T c) {
    if (a > 0 && b > 0 && c > 0) return fmin(a, fmin(b, c));
    if (a < 0 && b < 0 && c < 0) return fmax(a, fmax(b, c));
    return (T)0;
}

// slope of rho at a node from its value and its two neighbours' along one axis
// (ok: the node and both neighbours on N^+, the node's coordinate in [1, N-2];
// else 0)
template <class T>
__device__ __forceinline__ T slope_of(bool ok, T rm, T r0, T rp, T inv_h) {
    return ok ? minmod3<T>((T)2 * (rp - r0) * inv_h, (rp - rm) * ((T)0.5 * inv_h), (T)2 * (r0 - rm) * inv_h)
              : (T)0;
}

template <class T>
__global__ void k_flux(int N, T h, T chi, double dt_d, const double *dt_dev, const uint8_t *lab,
                       const T *rho, const T *c, T *f_rho, T *f_c) {
    const int64_t n3 = (int64_t)N * N * N;
    const T dt = (T)(dt_dev ? *dt_dev : dt_d), inv_h = (T)1 / h, half_h = (T)0.5 * h;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n3;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (!(lab[p] & DPM_LBL_MPLUS)) {
            f_rho[p] = (T)0;
            f_c[p] = (T)0;
            continue;
        }
        int coord[3];
        node_ijk(p, N, coord[0], coord[1], coord[2]);
        int64_t st[3] = {(int64_t)N * N, (int64_t)N, 1};
        T r0 = rho[p], c0 = c[p];
        T g = (T)0;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            int64_t s = st[ax];
            int cc = coord[ax];
            // the labels and densities at p +- s and p +- 2s that the three
            // slopes (at p, p - s, p + s) read, loaded at once; those at p +- 2s
            // only where that slope's node has a coordinate in [1, N-2]
            const bool in_c = cc >= 1 && cc <= N - 2, in_l = cc >= 2 && cc <= N - 1,
                       in_r = cc >= 0 && cc <= N - 3;
            const uint8_t lm1 = (in_c || in_l) ? lab[p - s] : 0, lp1 = (in_c || in_r) ? lab[p + s] : 0;
            const uint8_t lm2 = in_l ? lab[p - 2 * s] : 0, lp2 = in_r ? lab[p + 2 * s] : 0;
            const T rm1 = rho[p - s], rp1 = rho[p + s];
            const T rm2 = in_l ? rho[p - 2 * s] : (T)0, rp2 = in_r ? rho[p + 2 * s] : (T)0;
            const T cp1 = c[p + s], cm1 = c[p - s];
            // p is on M^+, hence on N^+
            T sp = slope_of<T>(in_c && in_np(lm1) && in_np(lp1), rm1, r0, rp1, inv_h);
            T sL = slope_of<T>(in_l && in_np(lm1) && in_np(lm2), rm2, rm1, r0, inv_h);
            T sR = slope_of<T>(in_r && in_np(lp1) && in_np(lp2), r0, rp1, rp2, inv_h);
            T gp = (cp1 - c0) * inv_h;  // grad c at j+1/2
            T gm = (c0 - cm1) * inv_h;  // grad c at j-1/2
            T east = r0 + half_h * sp, west = r0 - half_h * sp;
            T rho_p = gp > 0 ? east : rp1 - half_h * sR;
            T rho_m = gm > 0 ? rm1 + half_h * sL : west;
            g += (chi * rho_p * gp - chi * rho_m * gm) * inv_h;
        }
        f_rho[p] = r0 - dt * g;
        f_c[p] = ((T)1 - dt) * c0 + dt * r0;
    }
}

// gmax[ax] = max |c(p+e) - c(p)|, |c(p) - c(p-e)| over M^+ (as float bits).
// The maxima are taken in the state precision (|difference| of two state
// values, as the oracle takes them) and published as the bits of a
// non-negative double: non-negative IEEE doubles order like their bit
// patterns, so an integer atomicMax is an exact max and the FP64 path's
// CFL bound is the oracle's to the last bit for the same c.
template <class T>
__global__ void k_cfl(int N, const uint8_t *lab, const T *c, unsigned long long *gmax) {
    const int64_t n3 = (int64_t)N * N * N;
    T m[3] = {T(0), T(0), T(0)};
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n3;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (!(lab[p] & DPM_LBL_MPLUS)) continue;
        int64_t st[3] = {(int64_t)N * N, (int64_t)N, 1};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const T a = fabs(c[p + st[ax]] - c[p]);
            const T b = fabs(c[p] - c[p - st[ax]]);
            m[ax] = fmax(m[ax], fmax(a, b));
        }
    }
    __shared__ T shm[3][32];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        T v = m[ax];
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0) shm[ax][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        T v = T(0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, shm[threadIdx.x][w]);
        atomicMax(gmax + threadIdx.x, (unsigned long long)__double_as_longlong((double)v));
    }
}

constexpr int kDiagThreads = 256;
constexpr int kDiag = 6;  // mass, max rho, min rho, min c, m2, free energy

// Per-thread partials in T (a thread folds ~14 nodes of the 128^3 grid, so
// FP32 sums lose ~1e-7 on the FP32 paths and the FP64 pipe, 1/64 of the FP32
// rate here, is left to the block and final sums).
template <class T>
__global__ void k_diag(int N, double lo, double h, const uint8_t *lab, const T *rho, const T *c,
                       double *part, double ox, double oy, double oz) {
    const int64_t n3 = (int64_t)N * N * N;
    T a[kDiag] = {(T)0, (T)-INFINITY, (T)INFINITY, (T)INFINITY, (T)0, (T)0};
    const T inv8h2 = (T)(1.0 / (8.0 * h * h)), ht = (T)h;
    const T x0 = (T)(lo + ox), y0 = (T)(lo + oy), z0 = (T)(lo + oz);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n3;
         p += (int64_t)gridDim.x * blockDim.x) {
        uint8_t l = lab[p];
        if (!in_np(l)) continue;
        T r = rho[p], cc = c[p];
        a[2] = fmin(a[2], r);
        a[3] = fmin(a[3], cc);
        if (!(l & DPM_LBL_MPLUS)) continue;
        int i, j, k;
        node_ijk(p, N, i, j, k);
        // global coordinates: the grid's local frame plus its origin (0 unless
        // the grid belongs to a shifted sub-domain box)
        const T x = x0 + (T)(i + 1) * ht, y = y0 + (T)(j + 1) * ht, z = z0 + (T)(k + 1) * ht;
        a[0] += r;
        a[1] = fmax(a[1], r);
        a[4] += (x * x + y * y + z * z) * r;
        int64_t st[3] = {(int64_t)N * N, (int64_t)N, 1};
        T g2 = (T)0;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            T d = c[p + st[ax]] - c[p - st[ax]];
            g2 += d * d;
        }
        T rlr = r > (T)0 ? r * log(r) : (T)0;
        a[5] += rlr - r * cc + (T)0.5 * cc * cc + g2 * inv8h2;
    }
    // warp reduction: max / min in T (exact), the three sums in FP64
    __shared__ double sh[kDiag][kDiagThreads / 32];
    T mx = a[1], mn_r = a[2], mn_c = a[3];
    double s_m = (double)a[0], s_2 = (double)a[4], s_f = (double)a[5];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn_r = fmin(mn_r, __shfl_xor_sync(0xffffffffu, mn_r, o));
        mn_c = fmin(mn_c, __shfl_xor_sync(0xffffffffu, mn_c, o));
        s_m += __shfl_xor_sync(0xffffffffu, s_m, o);
        s_2 += __shfl_xor_sync(0xffffffffu, s_2, o);
        s_f += __shfl_xor_sync(0xffffffffu, s_f, o);
    }
    if ((threadIdx.x & 31) == 0) {
        const int w = threadIdx.x >> 5;
        sh[0][w] = s_m;
        sh[1][w] = (double)mx;
        sh[2][w] = (double)mn_r;
        sh[3][w] = (double)mn_c;
        sh[4][w] = s_2;
        sh[5][w] = s_f;
    }
    __syncthreads();
    if (threadIdx.x < kDiag) {
        int q = threadIdx.x;
        double x = sh[q][0];
        for (int w = 1; w < kDiagThreads / 32; ++w)
            x = (q == 1) ? fmax(x, sh[q][w]) : (q == 2 || q == 3) ? fmin(x, sh[q][w]) : x + sh[q][w];
        part[blockIdx.x * kDiag + q] = x;
    }
}

// Final reduction of the per-block partials: each thread folds a strided set of
// blocks in increasing order, then a fixed pairwise tree (deterministic).
__global__ void k_diag_final(int nblk, double h, const double *part, double *out) {
    constexpr int T = 256;
    __shared__ double sh[kDiag][T];
    const int t = threadIdx.x;
    double v[kDiag] = {0.0, -INFINITY, INFINITY, INFINITY, 0.0, 0.0};
    for (int b = t; b < nblk; b += T) {
        const double *pp = part + b * kDiag;
        v[0] += pp[0];
        v[1] = fmax(v[1], pp[1]);
        v[2] = fmin(v[2], pp[2]);
        v[3] = fmin(v[3], pp[3]);
        v[4] += pp[4];
        v[5] += pp[5];
    }
#pragma unroll
    for (int q = 0; q < kDiag; ++q) sh[q][t] = v[q];
    __syncthreads();
    for (int w = T / 2; w > 0; w >>= 1) {
        if (t < w) {
            sh[0][t] += sh[0][t + w];
            sh[1][t] = fmax(sh[1][t], sh[1][t + w]);
            sh[2][t] = fmin(sh[2][t], sh[2][t + w]);
            sh[3][t] = fmin(sh[3][t], sh[3][t + w]);
            sh[4][t] += sh[4][t + w];
            sh[5][t] += sh[5][t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        double h3 = h * h * h;
        out[0] = h3 * sh[0][0];
        out[1] = sh[1][0];
        out[2] = sh[2][0];
        out[3] = sh[3][0];
        out[4] = h3 * sh[4][0];
        out[5] = h3 * sh[5][0];
    }
}

__device__ __forceinline__ double gauss(const dpm_gaussian &g, double x, double y, double z) {
    double dx = x - g.center[0], dy = y - g.center[1], dz = z - g.center[2];
    return g.amp * exp(-g.alpha * (dx * dx + dy * dy + g.zscale * dz * dz));
}

template <class T>
__global__ void k_init_nodes(int N, double lo, double h, const uint8_t *lab, dpm_gaussian g0,
                             dpm_gaussian g1, T *rho, T *c) {
    const int64_t n3 = (int64_t)N * N * N;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n3;
         p += (int64_t)gridDim.x * blockDim.x) {
        T a = (T)0, b = (T)0;
        if (lab[p] & DPM_LBL_MPLUS) {
            int i, j, k;
            node_ijk(p, N, i, j, k);
            double x = lo + (double)(i + 1) * h, y = lo + (double)(j + 1) * h,
                   z = lo + (double)(k + 1) * h;
            a = (T)gauss(g0, x, y, z);
            b = (T)gauss(g1, x, y, z);
        }
        rho[p] = a;
        c[p] = b;
    }
}

template <class T>
__global__ void k_init_gex(int n, const int *gex, const int *gex_pos, const double *foot,
                           dpm_gaussian g0, dpm_gaussian g1, T *rho, T *c) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    int p = gex[e], g = gex_pos[e];
    const double *x = foot + 3 * (size_t)g;
    rho[p] = (T)gauss(g0, x[0], x[1], x[2]);
    c[p] = (T)gauss(g1, x[0], x[1], x[2]);
}

template <class T>
__global__ void k_mask_copy(int64_t n3, const uint8_t *lab, const T *src, T *dst) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n3;
         p += (int64_t)gridDim.x * blockDim.x)
        dst[p] = in_np(lab[p]) ? src[p] : (T)0;
}

template <class T>
__global__ void k_assemble(int64_t total, const double *psi_in, const T *trace, double *A) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        A[i] = psi_in[i] - (double)trace[i];
}

// One warp per node of gamma: u[q][g] = sum_nu C0 phi + beta d^2/2 sum_nu C2 phi + d gN,
// accumulated in P (the FP64 path: P = double).
template <class T, class P>
__global__ void k_extend(int n, int nsh, int beta, const P *phi, const double *dist,
                         const double *C, int ldc, const double *neumann, T *dens, int ldd,
                         int nr, int clamp, int cs_ok) {
    // the coefficients in P, converted once per block (cs_ok: they fit in shared memory)
    extern __shared__ unsigned char ext_sm[];
    P *cs = reinterpret_cast<P *>(ext_sm);
    const int ncu = (beta ? 2 : 1) * nsh;
    if (cs_ok) {
        for (int i = threadIdx.x; i < nr * ncu; i += blockDim.x)
            cs[i] = (P)C[(size_t)(i / ncu) * ldc + i % ncu];
        __syncthreads();
    }
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const P *ph = phi + (size_t)warp * nsh;
    const double d = dist[warp];
    for (int q = 0; q < nr; ++q) {
        const double *cq = C + (size_t)q * ldc;
        const P *cp = cs + (size_t)q * ncu;
        P s0 = (P)0, s2 = (P)0;
        for (int nu = lane; nu < nsh; nu += 32) {
            const P f = ph[nu];
            s0 += (cs_ok ? cp[nu] : (P)cq[nu]) * f;
            if (beta) s2 += (cs_ok ? cp[nsh + nu] : (P)cq[nsh + nu]) * f;
        }
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            double u = (double)s0 + 0.5 * d * d * (double)s2;
            if (neumann) u += d * neumann[warp];
            if (clamp && u < 0.0) u = 0.0;
            dens[(size_t)q * ldd + warp] = (T)u;
        }
    }
}

// FP32 paths: one thread per node of gamma, the harmonics in order (the FP32
// table is stored transposed, [nu][node], so the loads are coalesced), up to
// kExtQ right-hand sides per pass over the table; the coefficients converted
// to FP32 once per block into shared memory.
constexpr int kExtQ = 4;
template <class T>
__global__ void k_extend32(int n, int nsh, int beta, const float *__restrict__ phit,
                           const double *__restrict__ dist, const double *__restrict__ C, int ldc,
                           const double *__restrict__ neumann, T *dens, int ldd, int nr, int clamp) {
    extern __shared__ float cs32[];
    const int ncu = (beta ? 2 : 1) * nsh;
    for (int i = threadIdx.x; i < nr * ncu; i += blockDim.x) cs32[i] = (float)C[(size_t)(i / ncu) * ldc + i % ncu];
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const double d = dist[g];
    for (int q0 = 0; q0 < nr; q0 += kExtQ) {
        const int nq = min(kExtQ, nr - q0);
        float s0[kExtQ] = {}, s2[kExtQ] = {};
#pragma unroll 8
        for (int nu = 0; nu < nsh; ++nu) {
            const float f = phit[(size_t)nu * n + g];
#pragma unroll
            for (int q = 0; q < kExtQ; ++q)
                if (q < nq) {
                    const float *cp = cs32 + (size_t)(q0 + q) * ncu;
                    s0[q] = fmaf(cp[nu], f, s0[q]);
                    if (beta) s2[q] = fmaf(cp[nsh + nu], f, s2[q]);
                }
        }
#pragma unroll
        for (int q = 0; q < kExtQ; ++q)
            if (q < nq) {
                double u = (double)s0[q] + 0.5 * d * d * (double)s2[q];
                if (neumann) u += d * neumann[g];
                if (clamp && u < 0.0) u = 0.0;
                dens[(size_t)(q0 + q) * ldd + g] = (T)u;
            }
    }
}

// phit[nu][g] = float(phi[g][nu])
__global__ void k_phi32t(int n, int nsh, const double *phi, float *phit) {
    const int64_t total = (int64_t)n * nsh;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t nu = e / n, g = e - nu * n;
        phit[e] = (float)phi[g * nsh + nu];
    }
}

int blocks_for(int64_t n, int t) {
    int64_t b = (n + t - 1) / t;
    return (int)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}

// grid for the reductions over N^3 (a few nodes per thread, few partials)
int reduce_blocks(int64_t n, int t) {
    int64_t b = (n + t - 1) / t;
    return (int)(b > 152 * 4 ? 152 * 4 : (b < 1 ? 1 : b));
}

}  // namespace

template <class T>
int assemble_bep(const double *psi_in, const T *trace, double *A, int64_t m, int ncol,
                 const int *cond_flag, cudaStream_t s) {
    (void)cond_flag;
    DPM_PROF("assemble", s);
    int64_t total = m * ncol;
    k_assemble<T><<<blocks_for(total, 256), 256, 0, s>>>(total, psi_in, trace, A);
    DPM_LAUNCHED();
    return DPM_OK;
}
template int assemble_bep<float>(const double *, const float *, double *, int64_t, int, const int *,
                                 cudaStream_t);
template int assemble_bep<double>(const double *, const double *, double *, int64_t, int,
                                  const int *, cudaStream_t);

int gamma_phi32(const GammaGeom &gg, int64_t n_gamma, cudaStream_t s) {
    GammaGeom &g = const_cast<GammaGeom &>(gg);
    const size_t elems = (size_t)n_gamma * gg.nsh;
    if (elems == 0 || g.phi32.bytes >= elems * sizeof(float)) return DPM_OK;
    DPM_RET(g.phi32.alloc(elems * sizeof(float)));
    k_phi32t<<<blocks_for((int64_t)elems, 256), 256, 0, s>>>((int)n_gamma, gg.nsh, gg.phi.as<double>(),
                                                              g.phi32.as<float>());
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int extend_density(const GammaGeom &gg, int64_t n_gamma, int beta, const double *C, int ldc,
                   const double *neumann, T *dens, int ldd, int nr, int clamp, cudaStream_t s) {
    DPM_PROF("extend", s);
    int64_t threads = n_gamma * 32;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (sizeof(T) == 4) {
        const GammaGeom &g = gg;
        DPM_RET(gamma_phi32(gg, n_gamma, s));
        // right-hand sides in groups whose FP32 coefficients fit in 48 KB of shared memory
        const size_t per = sizeof(float) * (size_t)(beta ? 2 : 1) * gg.nsh;
        const int grp = (int)std::max<size_t>(1, (48 * 1024) / per);
        for (int q0 = 0; q0 < nr; q0 += grp) {
            const int nq = std::min(grp, nr - q0);
            k_extend32<T><<<(unsigned)((n_gamma + 127) / 128), 128, per * nq, s>>>(
                (int)n_gamma, gg.nsh, beta, g.phi32.as<float>(), gg.dist.as<double>(), C + (size_t)q0 * ldc, ldc,
                neumann, dens + (size_t)q0 * ldd, ldd, nq, clamp);
            if (q0 + grp < nr) DPM_LAUNCHED();
        }
    } else {
        const size_t sm = sizeof(double) * (size_t)nr * (beta ? 2 : 1) * gg.nsh;
        const int ok = sm <= 32 * 1024;
        k_extend<T, double><<<blocks, 256, ok ? sm : 0, s>>>((int)n_gamma, gg.nsh, beta, gg.phi.as<double>(),
                                                   gg.dist.as<double>(), C, ldc, neumann, dens, ldd, nr, clamp, ok);
    }
    DPM_LAUNCHED();
    return DPM_OK;
}
template int extend_density<float>(const GammaGeom &, int64_t, int, const double *, int,
                                   const double *, float *, int, int, int, cudaStream_t);
template int extend_density<double>(const GammaGeom &, int64_t, int, const double *, int,
                                    const double *, double *, int, int, int, cudaStream_t);

// ---- PKS helpers used by the API layer ------------------------------------
template <class T>
int pks_flux(int N, double h, double chi, double dt, const double *dt_dev, const uint8_t *lab,
             const T *rho, const T *c, T *f_rho, T *f_c, cudaStream_t s) {
    DPM_PROF("pks_flux", s);
    int64_t n3 = (int64_t)N * N * N;
    k_flux<T><<<blocks_for(n3, 256), 256, 0, s>>>(N, (T)h, (T)chi, dt, dt_dev, lab, rho, c, f_rho,
                                                  f_c);
    DPM_LAUNCHED();
    return DPM_OK;
}
template int pks_flux<float>(int, double, double, double, const double *, const uint8_t *,
                             const float *, const float *, float *, float *, cudaStream_t);
template int pks_flux<double>(int, double, double, double, const double *, const uint8_t *,
                              const double *, const double *, double *, double *, cudaStream_t);

// Step 3 on the device: dt = min(dt_max, CFL bound from the face-gradient
// maxima, dt_prev) (dt_mode 1; dt_max alone in dt_mode 0), sigma = 1/dt.
// The arithmetic is the host path's, in FP64.
__global__ void k_step_dt(const unsigned long long *gmax, double h, double chi, double dt_max, int mode,
                          StepScalars *sc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double dt = dt_max;
    if (mode == 1) {
        for (int ax = 0; ax < 3; ++ax) {
            const double gm = __longlong_as_double((long long)gmax[ax]) / h;
            if (gm > 0) dt = fmin(dt, h / (6.0 * chi * gm));
        }
        if (sc->step > 0) dt = fmin(dt, sc->dt_prev);
    }
    if (!(dt > 0) || !isfinite(dt)) {
        sc->bad = 1;
        dt = dt_max;
    }
    sc->rebuild_now = (sc->need_build || dt < sc->dt_prev) ? 1 : 0;
    sc->dt = dt;
    sc->sigma = 1.0 / dt;
}

__global__ void k_step_dt_grids(StepGrids g, double chi, double dt_max, int mode, StepScalars *sc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double dt = dt_max;
    if (mode == 1) {
        for (int l = 0; l < g.n; ++l)
            for (int ax = 0; ax < 3; ++ax) {
                const double gm = __longlong_as_double((long long)g.gmax[l][ax]) / g.h[l];
                if (gm > 0) dt = fmin(dt, g.h[l] / (6.0 * chi * gm));
            }
        if (sc->step > 0) dt = fmin(dt, sc->dt_prev);
    }
    if (!(dt > 0) || !isfinite(dt)) {
        sc->bad = 1;
        dt = dt_max;
    }
    sc->rebuild_now = (sc->need_build || dt < sc->dt_prev) ? 1 : 0;
    sc->dt = dt;
    sc->sigma = 1.0 / dt;
}

__global__ void k_step_end(StepScalars *sc, int rebuilt) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    sc->t += sc->dt;
    sc->dt_prev = sc->dt;
    sc->step += 1;
    sc->rebuilt = rebuilt < 0 ? sc->rebuild_now : rebuilt;
    if (sc->rebuilt) sc->need_build = 0;
}

__global__ void k_rebuild_cond(cudaGraphConditionalHandle h, const StepScalars *sc) {
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, sc->rebuild_now ? 1u : 0u);
}

int pks_step_dt(const unsigned long long *gmax, double h, double chi, double dt_max, int mode,
                StepScalars *sc, cudaStream_t s) {
    k_step_dt<<<1, 32, 0, s>>>(gmax, h, chi, dt_max, mode, sc);
    DPM_LAUNCHED();
    return DPM_OK;
}

int pks_step_dt_grids(const StepGrids &g, double chi, double dt_max, int mode, StepScalars *sc, cudaStream_t s) {
    if (g.n < 1 || g.n > kMaxStepGrids) { set_error("step dt: 1..%d grids", kMaxStepGrids); return DPM_EINVAL; }
    k_step_dt_grids<<<1, 32, 0, s>>>(g, chi, dt_max, mode, sc);
    DPM_LAUNCHED();
    return DPM_OK;
}

int pks_set_rebuild_cond(cudaGraphConditionalHandle h, const StepScalars *sc, cudaStream_t s) {
    k_rebuild_cond<<<1, 32, 0, s>>>(h, sc);
    DPM_LAUNCHED();
    return DPM_OK;
}

int pks_step_end(StepScalars *sc, int rebuilt, cudaStream_t s) {
    k_step_end<<<1, 32, 0, s>>>(sc, rebuilt);
    DPM_LAUNCHED();
    return DPM_OK;
}

template <class T>
int pks_cfl(int N, const uint8_t *lab, const T *c, unsigned long long *gmax, cudaStream_t s) {
    DPM_PROF("pks_cfl", s);
    int64_t n3 = (int64_t)N * N * N;
    DPM_CUDA(cudaMemsetAsync(gmax, 0, 3 * sizeof(unsigned long long), s));
    k_cfl<T><<<reduce_blocks(n3, 256), 256, 0, s>>>(N, lab, c, gmax);
    DPM_LAUNCHED();
    return DPM_OK;
}
template int pks_cfl<float>(int, const uint8_t *, const float *, unsigned long long *, cudaStream_t);
template int pks_cfl<double>(int, const uint8_t *, const double *, unsigned long long *, cudaStream_t);

int pks_diag_blocks(int N) { return reduce_blocks((int64_t)N * N * N, kDiagThreads); }

template <class T>
int pks_diag(int N, double lo, double h, const uint8_t *lab, const T *rho, const T *c,
             double *part, double *out, cudaStream_t s, const double *origin) {
    DPM_PROF("pks_diag", s);
    int nb = pks_diag_blocks(N);
    const double ox = origin ? origin[0] : 0.0, oy = origin ? origin[1] : 0.0, oz = origin ? origin[2] : 0.0;
    k_diag<T><<<nb, kDiagThreads, 0, s>>>(N, lo, h, lab, rho, c, part, ox, oy, oz);
    DPM_LAUNCHED();
    k_diag_final<<<1, 256, 0, s>>>(nb, h, part, out);
    DPM_LAUNCHED();
    return DPM_OK;
}
template int pks_diag<float>(int, double, double, const uint8_t *, const float *, const float *,
                             double *, double *, cudaStream_t, const double *);
template int pks_diag<double>(int, double, double, const uint8_t *, const double *,
                              const double *, double *, double *, cudaStream_t, const double *);

template <class T>
int pks_init(const GridIndex &gi, const GammaGeom &gg, const dpm_gaussian &g0,
             const dpm_gaussian &g1, T *rho, T *c, cudaStream_t s) {
    int64_t n3 = (int64_t)gi.N * gi.N * gi.N;
    k_init_nodes<T><<<blocks_for(n3, 256), 256, 0, s>>>(gi.N, gi.lo, gi.h, gi.labels.as<uint8_t>(),
                                                        g0, g1, rho, c);
    DPM_LAUNCHED();
    if (gi.n_gex > 0) {
        k_init_gex<T><<<(unsigned)((gi.n_gex + 255) / 256), 256, 0, s>>>(
            (int)gi.n_gex, gi.gex.as<int>(), gi.gex_pos.as<int>(), gg.foot.as<double>(), g0, g1,
            rho, c);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}
template int pks_init<float>(const GridIndex &, const GammaGeom &, const dpm_gaussian &,
                             const dpm_gaussian &, float *, float *, cudaStream_t);
template int pks_init<double>(const GridIndex &, const GammaGeom &, const dpm_gaussian &,
                              const dpm_gaussian &, double *, double *, cudaStream_t);

template <class T>
int mask_copy(int N, const uint8_t *lab, const T *src, T *dst, cudaStream_t s) {
    int64_t n3 = (int64_t)N * N * N;
    k_mask_copy<T><<<blocks_for(n3, 256), 256, 0, s>>>(n3, lab, src, dst);
    DPM_LAUNCHED();
    return DPM_OK;
}
template int mask_copy<float>(int, const uint8_t *, const float *, float *, cudaStream_t);
template int mask_copy<double>(int, const uint8_t *, const double *, double *, cudaStream_t);

}  // namespace dpm
