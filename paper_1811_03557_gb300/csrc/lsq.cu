// Least squares for the spectral coefficients of the BEP (eq. BEP_recast,
// Steps 2 and 5 of the main algorithm), refined to FP64 accuracy.
//
// Factor (once per BEP, Step 2 / 4b): an upper-triangular R with R^T R =
// A^T A (up to column equilibration D), A m x n column-major, m >> n:
//   * mixed precision (the FP32 paths): Gram of an FP32 copy of A over all
//     SMs (chunk sums in FP64, fixed order), equilibrated by its diagonal and
//     factored in FP32 in one CTA, R^{-1} kept in FP32 (n <= 168); for
//     larger n the Gram of an FP32 copy of A D (D from the column norms),
//     factored in FP64, with that copy kept for the solves' products with A^T;
//   * CholeskyQR in FP64 (FP64 SYRK, FP64 Cholesky; optionally equilibrated
//     with a small diagonal shift);
//   * Householder QR, one reflector H_j = I - tau_j v_j v_j^T per column
//     (three dependent launches per column; kept as the reference method).
// Solve (every step): C = D R^{-1} R^{-T} D A^T b (the semi-normal equations
// with the original A), then iterative refinement on r = b - A C, the
// residual always in FP64.  With the factor as a preconditioner the refined C
// agrees with a backward-stable QR solve; Q is never formed.  A block-banded
// A (lsq_set_band: the stacked BEPs of the layered decomposition) is stored
// dense, but the solves' products skip its zero blocks.
#include <math.h>

#include <algorithm>

#include "dpm_internal.cuh"

namespace dpm {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) t += sh[i];
    return t;
}

// Reflector for column j: v_j stored in A[j:m, j] (v_j[0] = x0 - alpha),
// alpha = -sign(x0) |x| is R[j][j]; tau = 2 / (v^T v).  Also clears w.
__global__ void k_house(int m, int n, int j, double *A, double *tau, double *rdiag, double *w,
                        int *status) {
    __shared__ double sh[32];
    double *col = A + (size_t)j * m;
    double s = 0.0;
    for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) s += col[r] * col[r];
    s = block_sum(s, sh);
    for (int c = threadIdx.x; c < n; c += blockDim.x) w[c] = 0.0;
    if (threadIdx.x == 0) {
        double x0 = col[j];
        double nrm = sqrt(x0 * x0 + s);
        if (!(nrm > 0.0) || !isfinite(nrm)) {
            tau[j] = 0.0;
            rdiag[j] = 0.0;
            status[0] = 1;
        } else {
            double alpha = x0 >= 0.0 ? -nrm : nrm;
            double v0 = x0 - alpha;
            col[j] = v0;
            tau[j] = 2.0 / (s + v0 * v0);
            rdiag[j] = alpha;
        }
    }
}

// w[c] += sum_{r in chunk, r >= j} v[r] A[r][c] for trailing columns c > j.
__global__ void k_dot(int m, int n, int j, const double *A, double *w, int rows_per) {
    __shared__ double sh[32];
    int c = j + 1 + blockIdx.x;
    int r0 = j + blockIdx.y * rows_per, r1 = min(m, r0 + rows_per);
    const double *v = A + (size_t)j * m, *a = A + (size_t)c * m;
    double s = 0.0;
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) s += v[r] * a[r];
    s = block_sum(s, sh);
    if (threadIdx.x == 0 && s != 0.0) atomicAdd(w + c, s);
}

__global__ void k_upd(int m, int n, int j, double *A, const double *tau, const double *w,
                      int rows_per) {
    int c = j + 1 + blockIdx.x;
    int r0 = j + blockIdx.y * rows_per, r1 = min(m, r0 + rows_per);
    const double *v = A + (size_t)j * m;
    double *a = A + (size_t)c * m;
    double f = tau[j] * w[c];
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) a[r] -= f * v[r];
}

// Dense upper-triangular R (row-major n x n) from the factored A.
__global__ void k_extract_r(int m, int n, const double *A, const double *rdiag, double *R) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int r = idx / n, c = idx % n;
    R[idx] = (c > r) ? A[(size_t)c * m + r] : (c == r ? rdiag[r] : 0.0);
}

// y[q][c] = sum_r A0[r][c] b[q][r]  (b in T, row stride ldb)
// part[sl][q][c] = sum over the rows of slice sl of A0[r][c] b[q][r]: one CTA
// per (column, row slice, group of up to kAtbQ right-hand sides), so that the
// FP64 work (which runs at a small fraction of the FP32 rate) spreads evenly
// over all SMs; kAtbU rows per thread in flight, fixed-order block sums.  The
// slices are added (in slice order) where y is consumed (k_trimv).
constexpr int kAtbQ = 4, kAtbU = 4, kAtbT = 256, kAtbMaxSlices = 16;
// The rows a CTA of k_atb / k_atb32 visits: its slice [r_begin, r_end), cut to
// the column's nonzero rows [lo, hi) when A is banded.  The first unrolled
// group is the one that holds lo, so every row keeps its thread and its place
// in that thread's sum (the skipped rows hold zeros): the same sums as the
// dense loop.
__device__ __forceinline__ void atb_rows(const int *cband, int c, int r_begin, int &r_start, int &r_end) {
    if (!cband) { r_start = r_begin; return; }
    const int lo = max(r_begin, cband[2 * c]);
    r_end = min(r_end, cband[2 * c + 1]);
    r_start = lo >= r_end ? r_end : r_begin + (lo - r_begin) / (kAtbU * kAtbT) * (kAtbU * kAtbT);
}

__global__ void __launch_bounds__(kAtbT) k_atb(int m, int n, const double *__restrict__ A0,
                                               const double *__restrict__ b, int ldb,
                                               double *__restrict__ part, int nr, int rows_per,
                                               const int *__restrict__ cband) {
    __shared__ double sh[kAtbQ][kAtbT / 32];
    const int c = blockIdx.x, sl = blockIdx.y, q0 = blockIdx.z * kAtbQ, nq = min(kAtbQ, nr - q0);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int r_begin = sl * rows_per;
    int r_end = min(m, r_begin + rows_per), r_start;
    atb_rows(cband, c, r_begin, r_start, r_end);
    const double *a = A0 + (size_t)c * m;
    double acc[kAtbQ] = {};
    for (int r0 = r_start + t; r0 < r_end; r0 += kAtbU * kAtbT) {
        double av[kAtbU];
#pragma unroll
        for (int u = 0; u < kAtbU; ++u) {
            const int r = r0 + u * kAtbT;
            av[u] = r < r_end ? a[r] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < kAtbQ; ++q) {
            if (q < nq) {
                const double *bq = b + (size_t)(q0 + q) * ldb;
#pragma unroll
                for (int u = 0; u < kAtbU; ++u) {
                    const int r = r0 + u * kAtbT;
                    if (r < r_end) acc[q] = fma(av[u], bq[r], acc[q]);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kAtbQ; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[q][warp] = v;
    }
    __syncthreads();
    if (t < nq) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < kAtbT / 32; ++w) v += sh[t][w];
        part[((size_t)sl * nr + q0 + t) * n + c] = v;
    }
}

// The same products from the FP32 copy of A and FP32 right-hand sides (or
// residuals): FP32 products, per-thread and warp sums, FP64 block sums.  Used for
// A^T b and A^T r on the mixed-precision path, where only the residual needs
// FP64 (the preconditioner's own error is larger than these roundings).
__global__ void __launch_bounds__(kAtbT) k_atb32(int m, int n, const float *__restrict__ A32,
                                                 const float *__restrict__ b, int ldb,
                                                 double *__restrict__ part, int nr, int rows_per,
                                                 const int *__restrict__ cband) {
    __shared__ double sh[kAtbQ][kAtbT / 32];
    const int c = blockIdx.x, sl = blockIdx.y, q0 = blockIdx.z * kAtbQ, nq = min(kAtbQ, nr - q0);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int r_begin = sl * rows_per;
    int r_end = min(m, r_begin + rows_per), r_start;
    atb_rows(cband, c, r_begin, r_start, r_end);
    const float *a = A32 + (size_t)c * m;
    float acc[kAtbQ] = {};
    for (int r0 = r_start + t; r0 < r_end; r0 += kAtbU * kAtbT) {
        float av[kAtbU];
#pragma unroll
        for (int u = 0; u < kAtbU; ++u) {
            const int r = r0 + u * kAtbT;
            av[u] = r < r_end ? a[r] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < kAtbQ; ++q) {
            if (q < nq) {
                const float *bq = b + (size_t)(q0 + q) * ldb;
#pragma unroll
                for (int u = 0; u < kAtbU; ++u) {
                    const int r = r0 + u * kAtbT;
                    if (r < r_end) acc[q] = fmaf(av[u], bq[r], acc[q]);
                }
            }
        }
    }
    // warp sums in FP32 (the FP64 pipe runs at 1/64 of the FP32 rate), the
    // block's 8 warp sums in FP64
#pragma unroll
    for (int q = 0; q < kAtbQ; ++q) {
        if (q < nq) {
            float v = acc[q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) sh[q][warp] = (double)v;
        }
    }
    __syncthreads();
    if (t < nq) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < kAtbT / 32; ++w) v += sh[t][w];
        part[((size_t)sl * nr + q0 + t) * n + c] = v;
    }
}

// out[q][r] = (double) b[q][r] (the FP32 right-hand sides, converted once)
__global__ void k_to_double(int m, int nr, const float *__restrict__ b, int ldb, double *__restrict__ out) {
    const size_t total = (size_t)m * nr;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
        out[e] = (double)b[(e / m) * ldb + e % m];
}

// res[q][r] = b[q][r] - sum_c A0[r][c] C[q][c].  A CTA takes 32 rows (the
// lanes) and up to kAtbQ right-hand sides; its 8 warps take the columns
// c = w, w + 8, ... and the 8 partial sums are added in warp order.
constexpr int kResW = 8;
// With a banded A (rband: the column interval of each 32-row group) each warp
// starts at its first column of the interval with the same residue mod kResW:
// the columns left out hold zeros in these rows, so the sums are the dense ones.
template <class T, class R>
__global__ void __launch_bounds__(32 * kResW) k_resid(int m, int n, const double *A0, const T *b, int ldb,
                                                      const double *C, R *res, int nr,
                                                      const int *__restrict__ rband) {
    __shared__ double sh[kResW][kAtbQ][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x * 32 + lane;
    const int q0 = blockIdx.y * kAtbQ, nq = min(kAtbQ, nr - q0);
    int c_lo = 0, c_hi = n;
    if (rband) {
        c_lo = rband[2 * blockIdx.x];
        c_hi = rband[2 * blockIdx.x + 1];
    }
    double s[kAtbQ] = {};
    if (r < m) {
        int c = c_lo + ((warp - c_lo) % kResW + kResW) % kResW;
        for (; c + 3 * kResW < c_hi; c += 4 * kResW) {
            double av[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) av[u] = A0[(size_t)(c + u * kResW) * m + r];
#pragma unroll
            for (int q = 0; q < kAtbQ; ++q)
                if (q < nq) {
                    const double *cq = C + (size_t)(q0 + q) * n;
#pragma unroll
                    for (int u = 0; u < 4; ++u) s[q] = fma(av[u], cq[c + u * kResW], s[q]);
                }
        }
        for (; c < c_hi; c += kResW) {
            const double av = A0[(size_t)c * m + r];
#pragma unroll
            for (int q = 0; q < kAtbQ; ++q)
                if (q < nq) s[q] = fma(av, C[(size_t)(q0 + q) * n + c], s[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < kAtbQ; ++q) sh[warp][q][lane] = s[q];
    __syncthreads();
    if (warp < nq && r < m) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < kResW; ++w) v += sh[w][warp][lane];
        res[(size_t)(q0 + warp) * m + r] = (R)((double)b[(size_t)(q0 + warp) * ldb + r] - v);
    }
}

// G partial sums: part[chunk][i][j] = sum over the chunk's rows of A[r][i] A[r][j]
// for the 64 x 64 tile (bi, bj) with bj >= bi (upper tiles only).
constexpr int kGT = 64, kGR = 16;
__global__ void k_syrk_part(int m, int n, const double *A, int rows_per, double *part) {
    __shared__ double As[kGR][kGT + 1], Bs[kGR][kGT + 1];
    const int nb = (n + kGT - 1) / kGT;
    // decode the upper tile index
    int tile = blockIdx.x, bi = 0;
    while (tile >= nb - bi) { tile -= nb - bi; ++bi; }
    const int bj = bi + tile;
    const int chunk = blockIdx.y;
    const int r0 = chunk * rows_per, r1 = min(m, r0 + rows_per);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 4 x 4 each
    double acc[4][4] = {};
    for (int rs = r0; rs < r1; rs += kGR) {
        for (int q = threadIdx.x; q < kGR * kGT; q += blockDim.x) {
            const int rr = q % kGR, cc = q / kGR;
            const int r = rs + rr;
            const int ci = bi * kGT + cc, cj = bj * kGT + cc;
            As[rr][cc] = (r < r1 && ci < n) ? A[(size_t)ci * m + r] : 0.0;
            Bs[rr][cc] = (r < r1 && cj < n) ? A[(size_t)cj * m + r] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < kGR; ++rr) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[rr][ty * 4 + u];
                b[u] = Bs[rr][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
    double *P = part + (size_t)chunk * n * n;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = bi * kGT + ty * 4 + u, j = bj * kGT + tx * 4 + v;
            if (i < n && j < n) P[(size_t)i * n + j] = acc[u][v];
        }
}

// G[i][j] = sum over chunks of part[chunk][i][j], for j >= i.  A CTA takes 32
// consecutive elements (the lanes); warp w sums the chunks w, w + 8, ... in
// order and the 8 warp sums are added in warp order (fixed, deterministic).
constexpr int kRedW = 8;
template <class P, class O>
__global__ void __launch_bounds__(32 * kRedW) k_syrk_reduce(int n, int nchunks, const P *part, O *G) {
    __shared__ double sh[kRedW][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int idx = blockIdx.x * 32 + lane;
    const int i = idx / n, j = idx % n;
    const bool on = idx < n * n && j >= i;  // upper triangle: only upper tiles were written
    double s = 0.0;
    if (on) {
        const size_t nn = (size_t)n * n;
        int c = warp;
        for (; c + 3 * kRedW < nchunks; c += 4 * kRedW) {
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = (double)part[(size_t)(c + u * kRedW) * nn + idx];
            s += v[0];
            s += v[1];
            s += v[2];
            s += v[3];
        }
        for (; c < nchunks; c += kRedW) s += (double)part[(size_t)c * nn + idx];
    }
    sh[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && on) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < kRedW; ++w) v += sh[w][lane];
        G[idx] = (O)v;
    }
}

// d[j] = 1 / ||A[:, j]||_2 (column equilibration; FP64)
__global__ void k_colscale(int m, const double *A, double *d) {
    __shared__ double sh[32];
    const int j = blockIdx.x;
    const double *a = A + (size_t)j * m;
    const int T_ = blockDim.x;
    double s = 0.0;
    for (int r0 = threadIdx.x; r0 < m; r0 += kAtbU * T_) {
        double av[kAtbU];
#pragma unroll
        for (int u = 0; u < kAtbU; ++u) av[u] = r0 + u * T_ < m ? a[r0 + u * T_] : 0.0;
#pragma unroll
        for (int u = 0; u < kAtbU; ++u) s = fma(av[u], av[u], s);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) d[j] = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
}

// Af = float(A D), column-major like A: the Gram products then read FP32
// operands (FP64 arithmetic runs at a small fraction of the FP32 rate).
__global__ void k_scale32(int m, const double *__restrict__ A, const double *__restrict__ d,
                          float *__restrict__ Af) {
    const int j = blockIdx.y;  // column
    const double dj = d[j];
    const double *a = A + (size_t)j * m;
    float *o = Af + (size_t)j * m;
    const int stride = gridDim.x * blockDim.x;
    for (int r0 = blockIdx.x * blockDim.x + threadIdx.x; r0 < m; r0 += kAtbU * stride) {
        double av[kAtbU];
#pragma unroll
        for (int u = 0; u < kAtbU; ++u) av[u] = r0 + u * stride < m ? a[r0 + u * stride] : 0.0;
#pragma unroll
        for (int u = 0; u < kAtbU; ++u)
            if (r0 + u * stride < m) o[r0 + u * stride] = (float)(av[u] * dj);
    }
}

// Af = float(A), column-major like A (the Gram products read FP32 operands);
// with lo: also lo = float(A - Af), so that A = Af + lo to about 2^-48 relative
__global__ void k_to_float(size_t total, const double *__restrict__ A, float *__restrict__ Af,
                           float *__restrict__ lo) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t e0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e0 < total; e0 += kAtbU * stride) {
        double v[kAtbU];
#pragma unroll
        for (int u = 0; u < kAtbU; ++u) v[u] = e0 + u * stride < total ? A[e0 + u * stride] : 0.0;
#pragma unroll
        for (int u = 0; u < kAtbU; ++u)
            if (e0 + u * stride < total) {
                const float hi = (float)v[u];
                Af[e0 + u * stride] = hi;
                if (lo) lo[e0 + u * stride] = (float)(v[u] - (double)hi);
            }
    }
}

// C as two floats per entry (hi, lo): the residual's coefficients
__global__ void k_split_coef(int total, const double *__restrict__ C, float *__restrict__ hi,
                             float *__restrict__ lo) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const double c = C[e];
        const float h = (float)c;
        hi[e] = h;
        lo[e] = (float)(c - (double)h);
    }
}

// res[q][r] = b[q][r] - sum_c A[r][c] C[q][c] in two-float arithmetic (the FP32
// paths): A = Ahi + Alo and C = Chi + Clo; each product's rounding error from an
// FMA (exact), the small cross terms in FP32, the running sum by TwoSum into a
// (sum, error) pair; the warps' pairs are added in FP64 at the end.  About 2^-44
// of the sums' magnitude, far below the FP32 rounding of the stored residual,
// at the FP32 rate instead of GB300's FP64 rate.  Same CTA and column layout as
// k_resid (32 rows x kResW warps, banded column intervals).
__global__ void __launch_bounds__(32 * kResW) k_resid2f(int m, int n, const float *__restrict__ Ahi,
                                                        const float *__restrict__ Alo, const float *b, int ldb,
                                                        const float *__restrict__ Chi,
                                                        const float *__restrict__ Clo, float *res, int nr,
                                                        const int *__restrict__ rband) {
    __shared__ double sh[kResW][kAtbQ][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x * 32 + lane;
    const int q0 = blockIdx.y * kAtbQ, nq = min(kAtbQ, nr - q0);
    int c_lo = 0, c_hi = n;
    if (rband) {
        c_lo = rband[2 * blockIdx.x];
        c_hi = rband[2 * blockIdx.x + 1];
    }
    float S[kAtbQ] = {}, E[kAtbQ] = {};
    if (r < m) {
        for (int c = c_lo + ((warp - c_lo) % kResW + kResW) % kResW; c < c_hi; c += kResW) {
            const float ah = Ahi[(size_t)c * m + r], al = Alo[(size_t)c * m + r];
#pragma unroll
            for (int q = 0; q < kAtbQ; ++q)
                if (q < nq) {
                    const float ch = Chi[(size_t)(q0 + q) * n + c], cl = Clo[(size_t)(q0 + q) * n + c];
                    const float p = ah * ch;
                    const float t = fmaf(ah, cl, fmaf(al, ch, fmaf(ah, ch, -p)));  // ah ch - p exact, + cross
                    const float sn = S[q] + p, bb = sn - S[q];
                    E[q] += ((S[q] - (sn - bb)) + (p - bb)) + t;  // TwoSum error + small terms
                    S[q] = sn;
                }
        }
    }
#pragma unroll
    for (int q = 0; q < kAtbQ; ++q) sh[warp][q][lane] = (double)S[q] + (double)E[q];
    __syncthreads();
    if (warp < nq && r < m) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < kResW; ++w) v += sh[w][warp][lane];
        res[(size_t)(q0 + warp) * m + r] = (float)((double)b[(size_t)(q0 + warp) * ldb + r] - v);
    }
}

// FP32 Gram partials of the FP32 copy of A (or of A D; upper 64 x 64 tiles),
// part[chunk][i][j] in float; the chunk sums are added in FP64 by k_syrk_reduce.
// 16 x 16 threads with 4 x 4 outputs each; per step 16 rows of the two column
// blocks in shared memory, stored with the float4 group of column c XORed by
// the row (rr) so that the transposing stores spread over the banks and each
// thread reads its 4 columns as one float4; the next step's rows are loaded
// into registers while this one is multiplied.
__device__ __forceinline__ int gram_sw(int rr, int cc) { return rr * kGT + ((((cc >> 2) ^ rr) & 15) << 2) + (cc & 3); }
__global__ void __launch_bounds__(256) k_syrk32_part(int m, int n, const float *Af, int rows_per, float *part) {
    __shared__ __align__(16) float As[kGR * kGT], Bs[kGR * kGT];
    const int nb = (n + kGT - 1) / kGT;
    int tile = blockIdx.x, bi = 0;
    while (tile >= nb - bi) { tile -= nb - bi; ++bi; }
    const int bj = bi + tile;
    const int chunk = blockIdx.y;
    const int r0 = chunk * rows_per, r1 = min(m, r0 + rows_per);
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    // this thread's 4 elements of each block per step: q = t + 256 e, row q % 16, column q / 16
    float pa[4], pb[4];
    auto fetch = [&](int rs) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int q = t + 256 * e, rr = q % kGR, cc = q / kGR, r = rs + rr;
            const int ci = bi * kGT + cc, cj = bj * kGT + cc;
            pa[e] = (r < r1 && ci < n) ? Af[(size_t)ci * m + r] : 0.f;
            pb[e] = (r < r1 && cj < n) ? Af[(size_t)cj * m + r] : 0.f;
        }
    };
    float acc[4][4] = {};
    if (r0 < r1) fetch(r0);
    for (int rs = r0; rs < r1; rs += kGR) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int q = t + 256 * e;
            As[gram_sw(q % kGR, q / kGR)] = pa[e];
            Bs[gram_sw(q % kGR, q / kGR)] = pb[e];
        }
        __syncthreads();
        if (rs + kGR < r1) fetch(rs + kGR);
#pragma unroll
        for (int rr = 0; rr < kGR; ++rr) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[rr * kGT + (((ty ^ rr) & 15) << 2)]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[rr * kGT + (((tx ^ rr) & 15) << 2)]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
        __syncthreads();
    }
    float *P = part + (size_t)chunk * n * n;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = bi * kGT + ty * 4 + u, j = bj * kGT + tx * 4 + v;
            if (i < n && j < n) P[(size_t)i * n + j] = acc[u][v];
        }
}

// FP32 Cholesky of the (well-conditioned, equilibrated) Gram matrix G = L L^T
// and the triangular inverse X = L^{-1}, in one CTA of kCholT threads, blocked
// by 32.  W (the factor) and X are n x ld floats in shared memory; the row
// stride ld = 4 (mod 8) keeps 16-byte rows and spreads a warp's float4 loads
// of 8 different rows over all banks.
//   per panel p: warp 0 factors the 32 x 32 diagonal block in registers (lane
//   = row, shuffles) and mirrors it into the block's upper triangle, so that
//   column j of L_pp is a contiguous row; the rows below solve against it by
//   right-looking substitution (one thread per row, float4 reads of the
//   mirror); the trailing lower triangle is updated in 4 x 4 register tiles
//   (float4 reads of the two panel rows, 16 FMAs per pair of loads).
//   inverse: warp b inverts diagonal block b (lane = column, right-looking);
//   M[bi][k] = X_bi,bi L[bi][k] goes to X's (unused) upper triangle,
//   transposed; then the off-diagonal blocks by block diagonals d = bi - bj:
//   X[bi][bj] = -sum_{k=bj}^{bi-1} M[bi][k] X[k][bj], both in 4 x 4 tiles.
// Rinv = R^{-1} = X^T is written in FP32 (it only preconditions the FP64
// refinement of every solve, so FP32 suffices for this equilibrated matrix);
// G, the upper triangle of the Gram, is read in FP32.
// Entries of W above the diagonal outside the current diagonal block and of
// the padding columns are scratch (tiles straddling the diagonal write them).
constexpr int kCholT = 384;
__host__ __device__ constexpr int chol_ld(int n) {
    return ((n + 3) & ~3) + ((((n + 3) & ~3) & 7) ? 0 : 4);
}
__host__ __device__ constexpr size_t chol_smem(int n) {
    return sizeof(float) * (2 * (size_t)n * chol_ld(n) + (size_t)n + 3 + 64);
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// (I, K) with 0 <= K <= I from the index I (I + 1) / 2 + K of a lower-triangular tile
__device__ __forceinline__ void tri_decode(int tt, int &I, int &K) {
    int i = (int)((sqrtf(8.f * (float)tt + 1.f) - 1.f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= tt) ++i;
    while (i * (i + 1) / 2 > tt) --i;
    I = i;
    K = tt - i * (i + 1) / 2;
}

// With dscale: G is the Gram of A itself; the kernel equilibrates it first,
// d_j = 1 / sqrt(G_jj) rounded to FP32 (dscale[j] = that value in FP64),
// and factors D G D.
__global__ void __launch_bounds__(kCholT) k_cholesky32(int n, const float *G, float *Rinv, int *status,
                                                       double *dscale) {
    extern __shared__ __align__(16) float sm32[];
    const int ld = chol_ld(n);
    float *W = sm32, *X = sm32 + (size_t)n * ld, *dinv = X + (size_t)n * ld;
    float *colb = dinv + n + ((4 - (n & 3)) & 3);  // 2 x 32 floats, 16-byte aligned
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int NW = kCholT / 32;
    const int nb = (n + 31) >> 5;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // ---- load: G's upper triangle, row j (read coalesced) -> column j of W's
    // lower triangle; the rest of W and all of X zero
    for (int q = t; q < n * ld / 4; q += kCholT) {
        reinterpret_cast<float4 *>(W)[q] = z4;
        reinterpret_cast<float4 *>(X)[q] = z4;
    }
    if (dscale) {
        for (int i = t; i < n; i += kCholT) {
            const float g = G[(size_t)i * n + i];
            const float d = g > 0.f ? 1.f / sqrtf(g) : 1.f;
            dinv[i] = d;  // the factor's reciprocals overwrite it below
            dscale[i] = (double)d;
        }
    }
    __syncthreads();
    // 4 rows of G per warp and pass, all 24 loads of a lane in flight (n <= 192)
    for (int j0 = 4 * warp; j0 < n; j0 += 4 * NW) {
        float v[4][6];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int j = j0 + r, i = 32 * c + lane;
                v[r][c] = (j < n && i < n && i >= j) ? G[(size_t)j * n + i] : 0.f;
            }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int j = j0 + r;
            if (j >= n) break;
            const float dj = dscale ? dinv[j] : 1.f;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int i = 32 * c + lane;
                if (i < n && i >= j) W[i * ld + j] = dscale ? v[r][c] * dinv[i] * dj : v[r][c];
            }
        }
    }
    __syncthreads();
    for (int p = 0; p < nb; ++p) {
        const int c0 = 32 * p, w = min(32, n - c0);
        // ---- diagonal block (warp 0); rows/columns past w are an identity pad.
        // Step j: lane i holds row i of the block (a) and column i of its
        // inverse X_pp (x); l[:, j] goes through colb and is read back as
        // broadcast float4 loads, once for both updates:
        //   a[k] -= l[i][j] l[k][j] (k > j)   and   x[k] -= l[k][j] x[j] (k > j),
        // after x[j] *= 1 / l[j][j].  Entries above the diagonal of a lane's
        // row of a are scratch (updated but never read); x stays zero above.
        if (warp == 0) {
            float a[32], x[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                a[k] = lane < w ? ((k <= lane) ? W[(c0 + lane) * ld + c0 + k] : 0.f) : (k == lane ? 1.f : 0.f);
                x[k] = k == lane ? 1.f : 0.f;
            }
            bool bad = false;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float piv = __shfl_sync(0xffffffffu, a[j], j);
                if (!(piv > 0.f) || !isfinite(piv)) {
                    bad = true;
                    piv = 1.f;
                }
                const float rs = rsqrtf(piv);  // 1 / l[j][j]
                const float lij = a[j] * rs;   // lane j: sqrt(piv)
                a[j] = lij;
                float *cb = colb + 32 * (j & 1);  // two buffers: one __syncwarp per step
                cb[lane] = lij;
                __syncwarp();
                x[j] *= rs;
#pragma unroll
                for (int q = (j + 1) / 4; q < 8; ++q) {
                    const float4 l = ld4(cb + 4 * q);
                    const float lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (4 * q + e > j) {
                            a[4 * q + e] = fmaf(-lij, lv[e], a[4 * q + e]);
                            x[4 * q + e] = fmaf(-lv[e], x[j], x[4 * q + e]);
                        }
                }
            }
            if (bad && lane == 0) status[0] = 1;
            if (lane < w) {
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (k < w) {
                        if (k <= lane) W[(c0 + lane) * ld + c0 + k] = a[k];  // L[lane][k]
                        if (k >= lane) X[(c0 + k) * ld + c0 + lane] = x[k];  // X_pp[k][lane]
                    }
            }
        }
        __syncthreads();
        const int r0 = c0 + w;
        if (r0 >= n) break;  // w == 32 below: the panel is a full block
        // ---- rows below: L[i][c0 + j] = sum_k a[k] X_pp[j][k], a = row i of the
        // panel.  Four threads per row, thread g taking j = g, g + 4, ...; the
        // result goes to PT[j][i] = X[c0 + j][i] (X's upper triangle, free
        // until the inverse) and is copied back into W during the trailing update.
        {
            for (int e = t; e < 4 * (n - r0); e += kCholT) {
                const int i = r0 + (e >> 2), g = e & 3;
                float acc[8] = {};
#pragma unroll 2
                for (int q = 0; q < 8; ++q) {
                    const float4 av = ld4(W + i * ld + c0 + 4 * q);
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        const float4 xv = ld4(X + (c0 + g + 4 * jj) * ld + c0 + 4 * q);
                        acc[jj] = fmaf(av.x, xv.x, fmaf(av.y, xv.y, fmaf(av.z, xv.z, fmaf(av.w, xv.w, acc[jj]))));
                    }
                }
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) X[(c0 + g + 4 * jj) * ld + i] = acc[jj];
            }
        }
        __syncthreads();
        // ---- trailing lower triangle, 4 x 4 tiles: W[i][k] -= sum_j L[i][c0+j] L[k][c0+j],
        // the panel read from PT (rows i0..i0+3 and k0..k0+3 are float4s of a PT row)
        {
            const int nt = (n - r0 + 3) >> 2;
            const float *PT = X + c0 * ld;
            // the panel back into W's lower triangle (columns c0.., not touched below)
            for (int e = t; e < 32 * (n - r0); e += kCholT) {
                const int j = e / (n - r0), i = r0 + e % (n - r0);
                W[i * ld + c0 + j] = PT[j * ld + i];
            }
            for (int tt = t; tt < nt * (nt + 1) / 2; tt += kCholT) {
                int I, K;
                tri_decode(tt, I, K);
                const int i0 = r0 + 4 * I, k0 = r0 + 4 * K;
                float acc[4][4] = {};
#pragma unroll 8
                for (int j = 0; j < 32; ++j) {
                    const float4 li = ld4(PT + j * ld + i0), lk = ld4(PT + j * ld + k0);
                    const float lv[4] = {li.x, li.y, li.z, li.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        acc[u][0] = fmaf(lv[u], lk.x, acc[u][0]);
                        acc[u][1] = fmaf(lv[u], lk.y, acc[u][1]);
                        acc[u][2] = fmaf(lv[u], lk.z, acc[u][2]);
                        acc[u][3] = fmaf(lv[u], lk.w, acc[u][3]);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (i0 + u < n) {
                        float4 *o = reinterpret_cast<float4 *>(W + (i0 + u) * ld + k0);
                        float4 v = *o;
                        v.x -= acc[u][0]; v.y -= acc[u][1]; v.z -= acc[u][2]; v.w -= acc[u][3];
                        *o = v;
                    }
            }
        }
        __syncthreads();
    }
    // ---- M = X_bb L[bi][:bi] for the rows of blocks bi >= 1, stored as
    // M^T in X's upper triangle: X[c][r] = sum_{s in block bi} X[r][s] L[s][c]
    {
        // tiles: per block bi >= 1, (rows of bi)/4 x (32 bi)/4, enumerated by block
        int base = 0;
        for (int bi = 1; bi < nb; ++bi) {
            const int rb = 32 * bi, wb = min(32, n - rb), nrt = (wb + 3) >> 2, nct = 8 * bi;
            const int cnt = nrt * nct;
            for (int tt = t - base; tt < cnt; tt += kCholT) {
                if (tt < 0) continue;
                const int r0 = rb + 4 * (tt / nct), cc = 4 * (tt % nct);
                float acc[4][4] = {};
                for (int q = 0; q < (wb + 3) >> 2; ++q) {
                    const int s0 = rb + 4 * q;
                    float4 xr[4], ls[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        xr[u] = r0 + u < n ? ld4(X + (r0 + u) * ld + s0) : z4;   // X[r][s0..s0+3]
                        ls[u] = s0 + u < n ? ld4(W + (s0 + u) * ld + cc) : z4;   // L[s0+u][cc..cc+3]
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float xs[4] = {xr[u].x, xr[u].y, xr[u].z, xr[u].w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            acc[u][0] = fmaf(xs[e], ls[e].x, acc[u][0]);
                            acc[u][1] = fmaf(xs[e], ls[e].y, acc[u][1]);
                            acc[u][2] = fmaf(xs[e], ls[e].z, acc[u][2]);
                            acc[u][3] = fmaf(xs[e], ls[e].w, acc[u][3]);
                        }
                    }
                }
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    *reinterpret_cast<float4 *>(X + (cc + v) * ld + r0) =
                        make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]);
            }
            base += cnt;
        }
    }
    __syncthreads();
    // ---- off-diagonal blocks of X by block diagonal d:
    // X[r][c] = -sum_{s in [32 bj, 32 bi)} M^T[s][r] X[s][c]
    for (int d = 1; d < nb; ++d) {
        int base = 0;
        for (int bj = 0; bj + d < nb; ++bj) {
            const int bi = bj + d, rb = 32 * bi, wb = min(32, n - rb), nrt = (wb + 3) >> 2;
            const int cnt = nrt * 8;
            for (int tt = t - base; tt < cnt; tt += kCholT) {
                if (tt < 0) continue;
                const int r0 = rb + 4 * (tt >> 3), cc = 32 * bj + 4 * (tt & 7);
                float acc[4][4] = {};
                for (int s = 32 * bj; s < rb; ++s) {
                    const float4 m = ld4(X + s * ld + r0);  // M^T[s][r0..r0+3]
                    const float4 x = ld4(X + s * ld + cc);  // X[s][cc..cc+3]
                    const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        acc[u][0] = fmaf(mv[u], x.x, acc[u][0]);
                        acc[u][1] = fmaf(mv[u], x.y, acc[u][1]);
                        acc[u][2] = fmaf(mv[u], x.z, acc[u][2]);
                        acc[u][3] = fmaf(mv[u], x.w, acc[u][3]);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (r0 + u < n)
                        *reinterpret_cast<float4 *>(X + (r0 + u) * ld + cc) =
                            make_float4(-acc[u][0], -acc[u][1], -acc[u][2], -acc[u][3]);
            }
            base += cnt;
        }
        __syncthreads();
    }
    for (int r = warp; r < n; r += NW)
        for (int c = lane; c < n; c += 32)  // Rinv[r][c] = X[c][r]
            Rinv[(size_t)r * n + c] = c >= r ? X[c * ld + r] : 0.f;
}

// Cholesky G = L L^T (upper triangle of G given) in one CTA; R = L^T row-major.
// Scratch W (n x n) is shared memory when it fits, else global.
__global__ void k_cholesky(int n, const double *G, double *R, double *Wg, int use_smem,
                           int *status) {
    extern __shared__ double Ws[];
    double *W = use_smem ? Ws : Wg;
    const int t = threadIdx.x, T = blockDim.x;
    for (int idx = t; idx < n * n; idx += T) {
        const int i = idx / n, j = idx % n;
        W[idx] = j >= i ? G[(size_t)i * n + j] : G[(size_t)j * n + i];
    }
    __syncthreads();
    __shared__ double dj;
    for (int j = 0; j < n; ++j) {
        if (t == 0) {
            double d = W[(size_t)j * n + j];
            if (!(d > 0.0) || !isfinite(d)) { status[0] = 1; d = 1.0; }
            d = sqrt(d);
            W[(size_t)j * n + j] = d;
            dj = d;
        }
        __syncthreads();
        const double inv = 1.0 / dj;
        for (int i = j + 1 + t; i < n; i += T) W[(size_t)i * n + j] *= inv;
        __syncthreads();
        const int w = n - j - 1;
        for (int idx = t; idx < w * w; idx += T) {
            const int i = j + 1 + idx / w, k = j + 1 + idx % w;
            if (k <= i) W[(size_t)i * n + k] -= W[(size_t)i * n + j] * W[(size_t)k * n + j];
        }
        __syncthreads();
    }
    for (int idx = t; idx < n * n; idx += T) {
        const int i = idx / n, k = idx % n;
        R[idx] = k >= i ? W[(size_t)k * n + i] : 0.0;  // R[i][k] = L[k][i]
    }
}

// Rinv = R^{-1} (upper triangular, row-major): one warp per column j solves
// R x = e_j by back substitution; x lives in shared memory.
__global__ void k_rinv(int n, const double *R, double *Rinv, int *status) {
    extern __shared__ double xs[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + warp;
    if (j >= n) return;
    double *x = xs + (size_t)warp * n;
    for (int i = lane; i < n; i += 32) x[i] = 0.0;
    __syncwarp();
    for (int i = j; i >= 0; --i) {
        double s = 0.0;
        for (int k = i + 1 + lane; k <= j; k += 32) s += R[(size_t)i * n + k] * x[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const double d = R[(size_t)i * n + i];
            if (d == 0.0) status[0] = 1;
            x[i] = ((i == j ? 1.0 : 0.0) - s) / (d == 0.0 ? 1.0 : d);
        }
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) Rinv[(size_t)i * n + j] = i <= j ? x[i] : 0.0;
}

// out[q][i] (+)= sum_k M[i][k] y[q][k] (TRANS = 0) or sum_k M[k][i] y[q][k]
// (TRANS = 1), M upper triangular n x n.  One warp per output element.
// With yparts > 1 (TRANS = 1), y holds the row-slice partial sums of A^T b,
// y[sl][q][k], added here in slice order and scaled by yscale[k] (if given).
template <int TRANS, class MT>
__global__ void k_trimv(int n, const MT *M, const double *y, double *out, int nr,
                        int accumulate, const double *outscale, int yparts = 1,
                        const double *yscale = nullptr) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (gw >= n * nr) return;
    const int q = gw / n, i = gw % n;
    const double *yq = y + (size_t)q * n;
    double s = 0.0;
    if (TRANS == 0) {
        for (int k = i + lane; k < n; k += 32) s += (double)M[(size_t)i * n + k] * yq[k];
    } else {
        for (int k = lane; k <= i; k += 32) {
            double yk = yq[k];
            for (int sl = 1; sl < yparts; ++sl) yk += yq[(size_t)sl * nr * n + k];
            if (yscale) yk *= yscale[k];
            s += (double)M[(size_t)k * n + i] * yk;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        if (outscale) s *= outscale[i];
        double *o2 = out + (size_t)q * n + i;
        *o2 = accumulate ? *o2 + s : s;
    }
}

// The mixed path's two triangular products in one CTA, in FP32 (they apply the
// FP32 preconditioner to a correction that the FP64 residual refines; C
// accumulates in FP64):
//   y[q][k] = yscale[k] sum_sl part[sl][q][k],  z = R^{-T} y,
//   C[q][i] (+)= outscale[i] (R^{-1} z)[q][i],
// with R^{-1} (upper triangular, row-major, FP32) staged in shared memory.
constexpr int kTriT = 1024;
size_t trisolve_smem(int n, int nr) { return sizeof(float) * ((size_t)n * n + 2 * (size_t)nr * n); }
__global__ void __launch_bounds__(kTriT) k_trisolve32(int n, int nr, const float *__restrict__ M,
                                                      const double *__restrict__ part, int S,
                                                      const double *__restrict__ yscale, double *C, int accumulate,
                                                      const double *__restrict__ outscale) {
    extern __shared__ float tsm[];
    float *Ms = tsm, *ys = Ms + (size_t)n * n, *zs = ys + (size_t)nr * n;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nn = n * n;
    for (int e0 = t; e0 < nn; e0 += 8 * kTriT) {  // 8 loads in flight per thread
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = e0 + u * kTriT < nn ? M[e0 + u * kTriT] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (e0 + u * kTriT < nn) Ms[e0 + u * kTriT] = v[u];
    }
    for (int e = t; e < nr * n; e += kTriT) {
        const int q = e / n, k = e - q * n;
        double v = 0.0;
        for (int sl = 0; sl < S; ++sl) v += part[((size_t)sl * nr + q) * n + k];
        if (yscale) v *= yscale[k];
        ys[e] = (float)v;
    }
    __syncthreads();
    for (int o = warp; o < nr * n; o += kTriT / 32) {  // z[q][i] = sum_{k <= i} M[k][i] y[q][k]
        const int q = o / n, i = o - q * n;
        float a = 0.f;
        for (int k = lane; k <= i; k += 32) a = fmaf(Ms[k * n + i], ys[q * n + k], a);
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) zs[o] = a;
    }
    __syncthreads();
    for (int o = warp; o < nr * n; o += kTriT / 32) {  // (R^{-1} z)[q][i] = sum_{k >= i} M[i][k] z[q][k]
        const int q = o / n, i = o - q * n;
        float a = 0.f;
        for (int k = i + lane; k < n; k += 32) a = fmaf(Ms[i * n + k], zs[q * n + k], a);
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) {
            double c = (double)a;
            if (outscale) c *= outscale[i];
            double *dst = C + (size_t)q * n + i;
            *dst = accumulate ? *dst + c : c;
        }
    }
}

}  // namespace

// The dynamic shared-memory limits of the least-squares kernels, raised to the
// per-CTA maximum (less each kernel's static shared memory) once per device.  (Setting each launch's own size before the
// launch raced between host threads that share a device: one thread could
// lower the limit between another's set and its launch.)  The limit bounds a
// launch's request; occupancy follows the size each launch asks for.
static int lsq_configure() {
    static PerDeviceOnce once;
    return once.run([] {
        DPM_RET(raise_dynamic_smem_limit(reinterpret_cast<const void *>(k_cholesky)));
        DPM_RET(raise_dynamic_smem_limit(reinterpret_cast<const void *>(k_cholesky32)));
        DPM_RET(raise_dynamic_smem_limit(reinterpret_cast<const void *>(k_rinv)));
        DPM_RET(raise_dynamic_smem_limit(reinterpret_cast<const void *>(k_trisolve32)));
        return (int)DPM_OK;
    });
}

static int householder_factor(LsqFactor &f, double *A0, double *w, double *rdiag, double *R,
                              int *status, cudaStream_t s) {
    const int m = f.m, n = f.n;
    DPM_RET(f.tau.reserve(sizeof(double) * n));
    double *A = f.A.as<double>();
    DPM_PROF("lsq_householder_qr", s);
    for (int j = 0; j < n; ++j) {
        k_house<<<1, 1024, 0, s>>>(m, n, j, A, f.tau.as<double>(), rdiag, w, status);
        DPM_LAUNCHED();
        int nt = n - j - 1;
        if (nt == 0) break;
        int rows = m - j;
        // enough blocks to cover the GPU when few columns remain
        int chunks = (int)((rows + 4095) / 4096);
        int want = (4 * 152 + nt - 1) / nt;
        if (chunks < want) chunks = want;
        int maxc = (rows + 255) / 256;
        if (chunks > maxc) chunks = maxc;
        if (chunks < 1) chunks = 1;
        int rows_per = (rows + chunks - 1) / chunks;
        dim3 g(nt, chunks);
        k_dot<<<g, kT, 0, s>>>(m, n, j, A, w, rows_per);
        DPM_LAUNCHED();
        k_upd<<<g, kT, 0, s>>>(m, n, j, A, f.tau.as<double>(), w, rows_per);
        DPM_LAUNCHED();
    }
    k_extract_r<<<(n * n + 255) / 256, 256, 0, s>>>(m, n, A, rdiag, R);
    DPM_LAUNCHED();
    (void)A0;
    return DPM_OK;
}

// G[i][j] *= d[i] d[j]: the Gram of A D from the Gram of A, plus `shift` on the
// diagonal (which is 1 after the scaling).
__global__ void k_gscale(int n, double *G, const double *d, double shift) {
    const size_t nn = (size_t)n * n;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x) {
        const size_t i = q / n, j = q % n;
        G[q] = G[q] * (d[i] * d[j]) + (i == j ? shift : 0.0);
    }
}

// Relative diagonal shift of the equilibrated FP64 Gram: directions of A D whose
// singular value is below ~1e-6 of the largest (numerically rank-deficient
// series, e.g. more harmonics than the grid boundary resolves) are damped
// instead of breaking the Cholesky; the FP64 refinement of every solve removes
// the shift's effect on all better-determined directions (contraction
// shift / (sigma_i^2 + shift) per step).
constexpr double kGramShift = 1e-12;

// FP64 Gram G = A^T A (tiles of partial sums reduced in FP64), then, with
// dscale, the column equilibration D G D (R becomes the factor of A D), then
// the FP64 Cholesky.
static int cholesky_factor(LsqFactor &f, const double *A0, double *R, int *status,
                           cudaStream_t s, double *dscale = nullptr) {
    const int m = f.m, n = f.n;
    const int nb = (n + kGT - 1) / kGT;
    const int ntiles = nb * (nb + 1) / 2;
    int chunks = (4 * 152 + ntiles - 1) / ntiles;
    const int maxc = (m + kGR - 1) / kGR;
    if (chunks > maxc) chunks = maxc;
    if (chunks < 1) chunks = 1;
    const int rows_per = ((m + chunks - 1) / chunks + kGR - 1) / kGR * kGR;
    chunks = (m + rows_per - 1) / rows_per;
    // scratch in f.X: partials [chunks][n][n], G [n][n], W [n][n]
    const size_t nn = (size_t)n * n;
    DPM_RET(f.X.reserve(sizeof(double) * (nn * (size_t)chunks + 2 * nn)));
    double *part = f.X.as<double>(), *G = part + nn * chunks, *W = G + nn;
    {
        DPM_PROF("lsq_gram_syrk", s);
        k_syrk_part<<<dim3(ntiles, chunks), 256, 0, s>>>(m, n, A0, rows_per, part);
        DPM_LAUNCHED();
        k_syrk_reduce<double, double><<<(unsigned)((nn + 31) / 32), 32 * kRedW, 0, s>>>(n, chunks, part, G);
        DPM_LAUNCHED();
        if (dscale) {
            k_colscale<<<n, 1024, 0, s>>>(m, A0, dscale);
            DPM_LAUNCHED();
            k_gscale<<<(unsigned)std::min<size_t>((nn + 255) / 256, 4096), 256, 0, s>>>(n, G, dscale, kGramShift);
            DPM_LAUNCHED();
        }
    }
    const size_t smem = nn * sizeof(double);
    const int use_smem = smem <= 200 * 1024 ? 1 : 0;
    if (use_smem) DPM_RET(lsq_configure());
    {
        DPM_PROF("lsq_cholesky", s);
        k_cholesky<<<1, 1024, use_smem ? smem : 0, s>>>(n, G, R, W, use_smem, status);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

// Mixed precision: Gram of an FP32 copy of A with FP32 products (chunk sums
// in FP64), column equilibration d_j = 1 / sqrt(G_jj) and FP32 Cholesky of
// D G D in one CTA; the refinement of every solve is FP64 against the
// original A (the factor only preconditions it).  Past the in-shared-memory
// size the Gram is that of A D (d from FP64 column norms), its Cholesky runs
// in FP64 from global memory and R^-1 is formed separately (*rinv_done = 0).
static int mixed_factor(LsqFactor &f, const double *A0, double *R, double *Rinv, double *dscale,
                        int *status, int *rinv_done, cudaStream_t s) {
    const int m = f.m, n = f.n;
    const int nb = (n + kGT - 1) / kGT;
    const int ntiles = nb * (nb + 1) / 2;
    int chunks = (4 * 152 + ntiles - 1) / ntiles;
    const int maxc = (m + kGR - 1) / kGR;
    if (chunks > maxc) chunks = maxc;
    if (chunks < 1) chunks = 1;
    const int rows_per = ((m + chunks - 1) / chunks + kGR - 1) / kGR * kGR;
    chunks = (m + rows_per - 1) / rows_per;
    const size_t nn = (size_t)n * n;
    const size_t smem = chol_smem(n);
    const bool in_smem = smem <= 227 * 1024;
    // partials [chunks][n][n] floats, then G [n][n] (and W [n][n] for the FP64
    // Cholesky), then Af [n][m] floats
    const size_t gbytes = sizeof(double) * nn * (in_smem ? 1 : 2);
    DPM_RET(f.X.reserve(sizeof(float) * nn * (size_t)chunks + 16 + gbytes + sizeof(float) * (size_t)m * n));
    float *part = f.X.as<float>();
    double *G = reinterpret_cast<double *>(part + nn * chunks + (nn * chunks & 1));
    float *Af = reinterpret_cast<float *>(reinterpret_cast<char *>(G) + gbytes);
    {
        DPM_PROF("lsq_gram_syrk", s);
        if (in_smem) {
            // Gram of float(A); the Cholesky kernel equilibrates it by its diagonal
            k_to_float<<<4 * 152, 256, 0, s>>>((size_t)m * n, A0, Af, nullptr);
            DPM_LAUNCHED();
        } else {
            // the two-float copy of A for the residual, A = hi + lo: its split costs
            // FP64 operations per entry, repaid by the FP32-rate residuals of the
            // many steps a factor of this size serves (n > 168: the decompositions)
            DPM_RET(f.A2.reserve(sizeof(float) * (size_t)m * n * 2));
            k_to_float<<<4 * 152, 256, 0, s>>>((size_t)m * n, A0, f.A2.as<float>(),
                                                f.A2.as<float>() + (size_t)m * n);
            DPM_LAUNCHED();
            f.Ahi = f.A2.as<float>();
            f.Alo = f.Ahi + (size_t)m * n;
            k_colscale<<<n, 1024, 0, s>>>(m, A0, dscale);
            DPM_LAUNCHED();
            k_scale32<<<dim3(8, n), 256, 0, s>>>(m, A0, dscale, Af);
            DPM_LAUNCHED();
        }
        k_syrk32_part<<<dim3(ntiles, chunks), 256, 0, s>>>(m, n, Af, rows_per, part);
        DPM_LAUNCHED();
        if (in_smem)  // the FP32 Cholesky reads the Gram in FP32 (summed in FP64, rounded once)
            k_syrk_reduce<float, float><<<(unsigned)((nn + 31) / 32), 32 * kRedW, 0, s>>>(
                n, chunks, part, reinterpret_cast<float *>(G));
        else
            k_syrk_reduce<float, double><<<(unsigned)((nn + 31) / 32), 32 * kRedW, 0, s>>>(n, chunks, part, G);
        DPM_LAUNCHED();
    }
    if (!in_smem) {
        DPM_PROF("lsq_cholesky", s);
        k_cholesky<<<1, 1024, 0, s>>>(n, G, R, G + nn, 0, status);
        DPM_LAUNCHED();
        *rinv_done = 0;
        f.A32s = Af;  // A D in FP32: the solves' products with A^T
        return DPM_OK;
    }
    *rinv_done = 1;
    f.rinv32 = true;
    f.A32 = Af;
    DPM_RET(lsq_configure());
    {
        DPM_PROF("lsq_cholesky", s);
        k_cholesky32<<<1, kCholT, smem, s>>>(n, reinterpret_cast<const float *>(G),
                                             reinterpret_cast<float *>(Rinv), status, dscale);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

static int lsq_factor_impl(LsqFactor &f, bool sync, cudaStream_t s);

int lsq_factor(LsqFactor &f, const int *cond_flag, cudaStream_t s) {
    (void)cond_flag;
    return lsq_factor_impl(f, true, s);
}

int lsq_factor_async(LsqFactor &f, cudaStream_t s) { return lsq_factor_impl(f, false, s); }

int lsq_set_band(LsqFactor &f, const std::vector<int64_t> &row0, const std::vector<int> &c0,
                 const std::vector<int> &c1, cudaStream_t s) {
    const int m = f.m, n = f.n;
    const size_t nb = c0.size();
    bool ok = m >= 1 && n >= 1 && nb >= 1 && row0.size() == nb + 1 && c1.size() == nb && row0[0] == 0 &&
              row0[nb] == m;
    for (size_t b = 0; ok && b < nb; ++b)
        ok = row0[b] <= row0[b + 1] && 0 <= c0[b] && c0[b] <= c1[b] && c1[b] <= n;
    if (!ok) { set_error("least squares: inconsistent block structure"); return DPM_EINVAL; }
    const int ng = (m + 31) / 32;
    std::vector<int> h(2 * (size_t)n + 2 * (size_t)ng, 0);
    // each column: the rows from its first block's first row to its last block's last
    for (int c = 0; c < n; ++c) {
        int64_t lo = m, hi = 0;
        for (size_t b = 0; b < nb; ++b)
            if (c0[b] <= c && c < c1[b] && row0[b] < row0[b + 1]) {
                lo = std::min(lo, row0[b]);
                hi = std::max(hi, row0[b + 1]);
            }
        if (lo < hi) {
            h[2 * c] = (int)lo;
            h[2 * c + 1] = (int)hi;
        }
    }
    // each 32-row group: the union of the column intervals of the blocks it meets
    for (int g = 0; g < ng; ++g) {
        const int64_t r0 = 32 * (int64_t)g, r1 = std::min<int64_t>(m, r0 + 32);
        int lo = n, hi = 0;
        for (size_t b = 0; b < nb; ++b)
            if (row0[b] < r1 && r0 < row0[b + 1] && c0[b] < c1[b]) {
                lo = std::min(lo, c0[b]);
                hi = std::max(hi, c1[b]);
            }
        if (lo < hi) {
            h[2 * (size_t)n + 2 * g] = lo;
            h[2 * (size_t)n + 2 * g + 1] = hi;
        }
    }
    DPM_RET(f.band.reserve(sizeof(int) * h.size()));
    DPM_CUDA(cudaMemcpyAsync(f.band.p, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice, s));
    DPM_CUDA(cudaStreamSynchronize(s));  // h goes out of scope
    return DPM_OK;
}

int lsq_status(const LsqFactor &f, cudaStream_t s) {
    const int m = f.m, n = f.n;
    if (!f.work.p) return DPM_OK;
    const int *status = reinterpret_cast<const int *>(f.work.as<double>() + (size_t)m * n + 2 * (size_t)n +
                                                      (size_t)n * n);
    int h_status = 0;
    DPM_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    DPM_CUDA(cudaStreamSynchronize(s));
    if (h_status) { set_error("BEP matrix is rank deficient (a zero pivot in the factorisation)"); return DPM_ENUMERIC; }
    return DPM_OK;
}

static int lsq_factor_impl(LsqFactor &f, bool sync, cudaStream_t s) {
    const int m = f.m, n = f.n;
    if (m < n || n < 1) { set_error("least squares: need m >= n >= 1 (m=%d n=%d)", m, n); return DPM_EINVAL; }
    // layout of f.work: [A0 m*n][w n][rdiag n][R n*n][status (64 B)][y R*n][res R*m]
    //                   [z R*n][Rinv n*n][colscale n][A^T b slices kAtbMaxSlices*R*n],
    //                   R = kLsqMaxRhs
    const size_t RR = kLsqMaxRhs;
    size_t need = sizeof(double) * ((size_t)m * n + 2 * (size_t)n + (size_t)n * n) + 64 +
                  sizeof(double) * RR * ((size_t)n + (size_t)m) + sizeof(double) * RR * (size_t)n +
                  sizeof(double) * (size_t)n * n + sizeof(double) * (size_t)n +
                  sizeof(double) * kAtbMaxSlices * RR * (size_t)n;
    DPM_RET(f.work.reserve(need));
    double *A0 = f.work.as<double>();
    double *w = A0 + (size_t)m * n;
    double *rdiag = w + n;
    double *R = rdiag + n;
    int *status = reinterpret_cast<int *>(R + (size_t)n * n);
    if (f.method == LsqFactor::kHouseholder)  // the reflectors overwrite f.A
        DPM_CUDA(cudaMemcpyAsync(A0, f.A.p, sizeof(double) * m * n, cudaMemcpyDeviceToDevice, s));
    else
        A0 = f.A.as<double>();
    DPM_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    double *Rinv = reinterpret_cast<double *>(reinterpret_cast<char *>(R + (size_t)n * n) + 64) +
                   kLsqMaxRhs * ((size_t)n + (size_t)m) + kLsqMaxRhs * (size_t)n;
    double *dscale = Rinv + (size_t)n * n;
    f.equilibrated = false;
    f.rinv32 = false;
    f.A32 = nullptr;
    f.A32s = nullptr;
    f.Ahi = nullptr;
    f.Alo = nullptr;
    int rinv_done = 0;
    if (f.method == LsqFactor::kHouseholder) {
        DPM_RET(householder_factor(f, A0, w, rdiag, R, status, s));
    } else if (f.method == LsqFactor::kCholeskyQR) {
        DPM_RET(cholesky_factor(f, A0, R, status, s));
    } else if (f.method == LsqFactor::kEquilibrated64) {
        DPM_RET(cholesky_factor(f, A0, R, status, s, dscale));
        f.equilibrated = true;
    } else {
        DPM_RET(mixed_factor(f, A0, R, Rinv, dscale, status, &rinv_done, s));
        f.equilibrated = true;
    }
    if (!rinv_done) {
        DPM_PROF("lsq_rinv", s);
        // one warp per column of R^-1, each with an n-vector in shared memory
        const size_t per = sizeof(double) * (size_t)n;
        const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (200 * 1024) / per));
        const size_t smem = per * warps;
        if (smem > 227 * 1024) { set_error("least squares: n = %d too large for R^-1", n); return DPM_EINVAL; }
        if (smem > 48 * 1024) DPM_RET(lsq_configure());
        k_rinv<<<(n + warps - 1) / warps, 32 * warps, smem, s>>>(n, R, Rinv, status);
        DPM_LAUNCHED();
    }
    if (!sync) return DPM_OK;
    int h_status = 0;
    DPM_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    DPM_CUDA(cudaStreamSynchronize(s));
    if (h_status) { set_error("BEP matrix is rank deficient (a zero pivot in the factorisation)"); return DPM_ENUMERIC; }
    return DPM_OK;
}

template <class T>
int lsq_apply(const LsqFactor &f, const T *b, int ldb, double *C, int nr, cudaStream_t s) {
    const int m = f.m, n = f.n;
    const double *R = f.work.as<double>() + (size_t)m * n + 2 * (size_t)n;
    const double *A0 = lsq_matrix(f);
    int *status = reinterpret_cast<int *>(const_cast<double *>(R) + (size_t)n * n);
    if (nr < 1 || nr > kLsqMaxRhs) { set_error("least squares: 1..%d right-hand sides per call", kLsqMaxRhs); return DPM_EINVAL; }
    // scratch after the factor (layout in lsq_factor_impl): the residuals
    // res[nr][m] (FP32 on the mixed path), z[nr][n], then R^{-1}, the column
    // scales and the A^T b slices; the y region is not used by the solve
    size_t base = sizeof(double) * ((size_t)m * n + 2 * (size_t)n + (size_t)n * n) + 64;
    double *y = reinterpret_cast<double *>(static_cast<char *>(f.work.p) + base);
    double *res = y + kLsqMaxRhs * (size_t)n;
    double *z = res + kLsqMaxRhs * (size_t)m;
    const double *Rinv = z + kLsqMaxRhs * (size_t)n;
    (void)status;
    const int mv_blocks = (n * nr * 32 + 255) / 256;
    const double *dsc = f.equilibrated ? Rinv + (size_t)n * n : nullptr;
    // refinement steps (FP64 residual): each contracts the error by
    // ~kappa(AD)^2 eps_32, down to the floor the products with A^T set: none
    // below 1e-10 relative with FP64 products; with FP32 products (the FP32
    // paths with an FP32 copy of A) about kappa eps_32 |r| / (|A| |C|), still
    // far below the FP32 solver's own error.  One step on the FP32 paths, three
    // on the FP64 path.
    const int refine = f.equilibrated ? (sizeof(T) == sizeof(double) ? 3 : 1) : 1;
    DPM_PROF("lsq_solve", s);
    // A^T b by row slices: about six CTAs per SM in all, at most kAtbMaxSlices
    const unsigned qg = (unsigned)((nr + kAtbQ - 1) / kAtbQ);
    int S = (int)std::min<long>(kAtbMaxSlices, std::max<long>(1, (6L * 152 + (long)n * qg - 1) / ((long)n * qg)));
    const int rows_per = (m + S - 1) / S;
    S = (m + rows_per - 1) / rows_per;
    double *ypart = const_cast<double *>(Rinv) + (size_t)n * n + n;
    // FP32 right-hand sides with the factor's FP32 copy of A (or of A D, whose
    // products already carry the column scales): the products with A^T in FP32
    // (FP64 sums), only the residual in FP64; it is stored in FP32 in res's space
    const float *A32 = f.A32 ? f.A32 : (sizeof(T) == sizeof(float) ? f.A32s : nullptr);
    const bool fast32 = sizeof(T) == sizeof(float) && A32 != nullptr;
    const bool y_scaled = fast32 && !f.A32;
    // block-banded A: the column row intervals, then the 32-row column intervals
    const int *cband = f.band.p ? f.band.as<int>() : nullptr;
    const int *rband = cband ? cband + 2 * (size_t)n : nullptr;
    const double *bd = nullptr;
    int ldbd = 0;
    if (!fast32) {
        if constexpr (sizeof(T) == sizeof(float)) {
            // the FP32 right-hand sides in FP64 once (res is free until the refinement)
            k_to_double<<<(unsigned)std::min<size_t>(((size_t)m * nr + 255) / 256, 4 * 152), 256, 0, s>>>(
                m, nr, reinterpret_cast<const float *>(b), ldb, res);
            DPM_LAUNCHED();
            bd = res;
            ldbd = m;
        } else {
            bd = reinterpret_cast<const double *>(b);
            ldbd = ldb;
        }
    }
    float *res32 = reinterpret_cast<float *>(res);
    // out (+)= R^{-1} or R^{-T} times y, R^{-1} in FP32 or FP64
    auto trimv = [&](bool trans, const double *yin, double *out, int accumulate, const double *outscale,
                     int yparts, const double *yscale) -> int {
        const float *M32 = reinterpret_cast<const float *>(Rinv);
        if (trans && f.rinv32)
            k_trimv<1, float><<<mv_blocks, 256, 0, s>>>(n, M32, yin, out, nr, accumulate, outscale, yparts, yscale);
        else if (trans)
            k_trimv<1, double><<<mv_blocks, 256, 0, s>>>(n, Rinv, yin, out, nr, accumulate, outscale, yparts, yscale);
        else if (f.rinv32)
            k_trimv<0, float><<<mv_blocks, 256, 0, s>>>(n, M32, yin, out, nr, accumulate, outscale);
        else
            k_trimv<0, double><<<mv_blocks, 256, 0, s>>>(n, Rinv, yin, out, nr, accumulate, outscale);
        DPM_LAUNCHED();
        return DPM_OK;
    };
    // C = D R^{-1} R^{-T} D A^T b   (D = I unless the factor was equilibrated)
    if (fast32)
        k_atb32<<<dim3(n, S, qg), kAtbT, 0, s>>>(m, n, A32, reinterpret_cast<const float *>(b), ldb, ypart,
                                                 nr, rows_per, cband);
    else
        k_atb<<<dim3(n, S, qg), kAtbT, 0, s>>>(m, n, A0, bd, ldbd, ypart, nr, rows_per, cband);
    DPM_LAUNCHED();
    // z = R^{-T} D y, C (+)= D R^{-1} z
    const size_t tsm = trisolve_smem(n, nr);
    const bool fused = fast32 && !y_scaled && f.rinv32 && tsm <= 227 * 1024;
    if (fused && tsm > 48 * 1024) DPM_RET(lsq_configure());
    auto precondition = [&](int accumulate) -> int {
        if (fused) {
            k_trisolve32<<<1, kTriT, tsm, s>>>(n, nr, reinterpret_cast<const float *>(Rinv), ypart, S, dsc, C,
                                               accumulate, dsc);
            DPM_LAUNCHED();
            return DPM_OK;
        }
        DPM_RET(trimv(true, ypart, z, 0, nullptr, S, y_scaled ? nullptr : dsc));
        return trimv(false, z, C, accumulate, dsc, 1, nullptr);
    };
    DPM_RET(precondition(0));
    // iterative refinement: C += D R^{-1} R^{-T} D A^T (b - A C), the residual in FP64
    // (two-float on the FP32 paths)
    for (int it = 0; it < refine; ++it) {
        if (fast32 && f.Alo) {
            // two-float residual: the coefficients split once per refinement step
            float *chi = reinterpret_cast<float *>(z), *clo = chi + (size_t)nr * n;
            k_split_coef<<<(unsigned)std::min(((size_t)nr * n + 255) / 256, (size_t)152), 256, 0, s>>>(nr * n, C,
                                                                                                   chi, clo);
            DPM_LAUNCHED();
            k_resid2f<<<dim3((m + 31) / 32, qg), 32 * kResW, 0, s>>>(m, n, f.Ahi, f.Alo,
                                                                     reinterpret_cast<const float *>(b), ldb, chi,
                                                                     clo, res32, nr, rband);
            DPM_LAUNCHED();
            k_atb32<<<dim3(n, S, qg), kAtbT, 0, s>>>(m, n, A32, res32, m, ypart, nr, rows_per, cband);
        } else if (fast32) {
            k_resid<T, float><<<dim3((m + 31) / 32, qg), 32 * kResW, 0, s>>>(m, n, A0, b, ldb, C, res32, nr,
                                                                              rband);
            DPM_LAUNCHED();
            k_atb32<<<dim3(n, S, qg), kAtbT, 0, s>>>(m, n, A32, res32, m, ypart, nr, rows_per, cband);
        } else {
            k_resid<T, double><<<dim3((m + 31) / 32, qg), 32 * kResW, 0, s>>>(m, n, A0, b, ldb, C, res, nr,
                                                                               rband);
            DPM_LAUNCHED();
            k_atb<<<dim3(n, S, qg), kAtbT, 0, s>>>(m, n, A0, res, m, ypart, nr, rows_per, cband);
        }
        DPM_LAUNCHED();
        DPM_RET(precondition(1));
    }
    return DPM_OK;
}

template int lsq_apply<float>(const LsqFactor &, const float *, int, double *, int, cudaStream_t);
template int lsq_apply<double>(const LsqFactor &, const double *, int, double *, int, cudaStream_t);

}  // namespace dpm
