// FP64 least squares for the spectral coefficients of the BEP (eq. BEP_recast,
// Steps 2 and 5 of the main algorithm).
//
// Factor (once per BEP, Step 2 / 4b): the R factor of the QR decomposition of
// A (m x n, column-major, m >> n).  Two ways are built:
//   * CholeskyQR (default): R^T R = A^T A with G = A^T A formed by one FP64
//     SYRK over all SMs (fixed-order partial sums, deterministic) and R the
//     Cholesky factor of G (one CTA, in shared memory for n <= 168);
//   * Householder QR, one reflector H_j = I - tau_j v_j v_j^T per column
//     (three dependent launches per column; kept as the reference method).
// Solve (every step): R^T R C = A^T b with the original A (the semi-normal
// equations), then one step of iterative refinement on r = b - A C.  With
// kappa(A)^2 * eps_64 << 1 the refined C agrees with a backward-stable QR
// solve; the FP64 work per step is two GEMVs over all SMs plus n x n
// triangular solves in one CTA, and Q is never formed.
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
template <class T>
__global__ void k_atb(int m, int n, const double *A0, const T *b, int ldb, double *y, int nr,
                      const double *colscale) {
    __shared__ double sh[32];
    int c = blockIdx.x, q = blockIdx.y;
    const double *a = A0 + (size_t)c * m;
    const T *bq = b + (size_t)q * ldb;
    double s = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) s += a[r] * (double)bq[r];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) y[(size_t)q * n + c] = colscale ? s * colscale[c] : s;
}

// res[q][r] = b[q][r] - sum_c A0[r][c] C[q][c]
template <class T>
__global__ void k_resid(int m, int n, const double *A0, const T *b, int ldb, const double *C,
                        double *res, int nr) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    int q = blockIdx.y;
    if (r >= m) return;
    const double *cq = C + (size_t)q * n;
    double s0 = (double)b[(size_t)q * ldb + r], s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int c = 0;
    for (; c + 3 < n; c += 4) {
        s0 -= A0[(size_t)c * m + r] * cq[c];
        s1 -= A0[(size_t)(c + 1) * m + r] * cq[c + 1];
        s2 -= A0[(size_t)(c + 2) * m + r] * cq[c + 2];
        s3 -= A0[(size_t)(c + 3) * m + r] * cq[c + 3];
    }
    for (; c < n; ++c) s0 -= A0[(size_t)c * m + r] * cq[c];
    res[(size_t)q * m + r] = (s0 + s1) + (s2 + s3);
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

// G[i][j] = sum_chunk part[chunk][i][j] in chunk order, for j >= i.
__global__ void k_syrk_reduce(int n, int nchunks, const double *part, double *G) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int i = idx / n, j = idx % n;
    if (j < i) return;
    const int bi = i / kGT, bj = j / kGT;  // only upper tiles were written
    if (bj < bi) return;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * n * n + idx];
    G[idx] = s;
}

// d[j] = 1 / ||A[:, j]||_2 (column equilibration; FP64)
__global__ void k_colscale(int m, const double *A, double *d) {
    __shared__ double sh[32];
    const int j = blockIdx.x;
    const double *a = A + (size_t)j * m;
    double s = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) s += a[r] * a[r];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) d[j] = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
}

// Af = float(A D), column-major like A: the Gram products then read FP32
// operands (FP64 arithmetic runs at a small fraction of the FP32 rate).
__global__ void k_scale32(int m, const double *A, const double *d, float *Af) {
    const int j = blockIdx.y;  // column
    const double dj = d[j];
    const double *a = A + (size_t)j * m;
    float *o = Af + (size_t)j * m;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x)
        o[r] = (float)(a[r] * dj);
}

// FP32 Gram partials of the equilibrated matrix A D (upper 64 x 64 tiles),
// part[chunk][i][j] in float; the chunk sums are added in FP64 by k_syrk_reduce32.
__global__ void k_syrk32_part(int m, int n, const float *Af, int rows_per, float *part) {
    __shared__ float As[kGR][kGT + 1], Bs[kGR][kGT + 1];
    const int nb = (n + kGT - 1) / kGT;
    int tile = blockIdx.x, bi = 0;
    while (tile >= nb - bi) { tile -= nb - bi; ++bi; }
    const int bj = bi + tile;
    const int chunk = blockIdx.y;
    const int r0 = chunk * rows_per, r1 = min(m, r0 + rows_per);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4] = {};
    for (int rs = r0; rs < r1; rs += kGR) {
        for (int q = threadIdx.x; q < kGR * kGT; q += blockDim.x) {
            const int rr = q % kGR, cc = q / kGR;
            const int r = rs + rr;
            const int ci = bi * kGT + cc, cj = bj * kGT + cc;
            As[rr][cc] = (r < r1 && ci < n) ? Af[(size_t)ci * m + r] : 0.f;
            Bs[rr][cc] = (r < r1 && cj < n) ? Af[(size_t)cj * m + r] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < kGR; ++rr) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[rr][ty * 4 + u];
                b[u] = Bs[rr][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
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

__global__ void k_syrk_reduce32(int n, int nchunks, const float *part, double *G) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int i = idx / n, j = idx % n;
    if (j < i) return;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += (double)part[(size_t)c * n * n + idx];
    G[idx] = s;
}

// FP32 Cholesky of the (well-conditioned, equilibrated) Gram matrix G = L L^T
// and the triangular inverse X = L^{-1}, in one CTA, blocked by 32 so that
// the sequential steps stay inside a warp (register rows and shuffles) and
// the CTA meets at ~25 barriers:
//   per panel p: warp 0 factors the diagonal block; one thread per row below
//   solves its panel row against it; all threads apply the trailing update;
//   inverse: warp b inverts diagonal block b; M[bi][k] = X_bi,bi L[bi][k] goes
//   to X's (unused) upper triangle, transposed; then the off-diagonal blocks
//   by block diagonals d = bi - bj: X[bi][bj] = -sum_{k=bj}^{bi-1} M[bi][k] X[k][bj].
// Rinv = R^{-1} = X^T is written in FP64.  It only preconditions the FP64
// refinement of every solve, so FP32 suffices for this equilibrated matrix.
__global__ void __launch_bounds__(1024) k_cholesky32(int n, const double *G, double *Rinv,
                                                     int *status) {
    extern __shared__ float sm32[];
    float *W = sm32, *X = sm32 + (size_t)n * n;
    const int t = threadIdx.x, T = blockDim.x, lane = t & 31, warp = t >> 5, nwarp = T >> 5;
    const int nb = (n + 31) >> 5;
    // G's upper triangle (row-major, read coalesced) -> lower triangle of W
    for (int j = warp; j < n; j += nwarp)
        for (int i = lane; i < n; i += 32) {
            W[i * n + j] = i >= j ? (float)G[(size_t)j * n + i] : 0.f;
            X[j * n + i] = 0.f;
        }
    __syncthreads();
    for (int p = 0; p < nb; ++p) {
        const int c0 = 32 * p, w = min(32, n - c0);
        // ---- diagonal block: lane i owns row c0 + i ----------------------------
        if (warp == 0) {
            float a[32];
#pragma unroll
            for (int k = 0; k < 32; ++k)
                a[k] = (lane < w && k <= lane) ? W[(c0 + lane) * n + c0 + k] : 0.f;
            bool bad = false;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < w) {
                    float piv = __shfl_sync(0xffffffffu, a[j], j);
                    if (!(piv > 0.f) || !isfinite(piv)) {
                        bad = true;
                        piv = 1.f;
                    }
                    const float lij = a[j] * rsqrtf(piv);  // lane j: sqrt(piv)
                    if (lane >= j) a[j] = lij;
#pragma unroll
                    for (int k = j + 1; k < 32; ++k) {
                        const float lkj = __shfl_sync(0xffffffffu, lij, k);
                        if (lane >= k) a[k] -= lij * lkj;
                    }
                }
            }
            if (bad && lane == 0) status[0] = 1;
            if (lane < w) {
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (k <= lane) W[(c0 + lane) * n + c0 + k] = a[k];
            }
        }
        __syncthreads();
        // ---- panel rows below: L[i][c0+j] = (W - sum_k L[i][c0+k] L[c0+j][c0+k]) / L[c0+j][c0+j]
        for (int i = c0 + w + t; i < n; i += T) {
            float x[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) x[j] = j < w ? W[i * n + c0 + j] : 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < w) {
                    float acc = x[j];
#pragma unroll
                    for (int k = 0; k < j; ++k) acc -= x[k] * W[(c0 + j) * n + c0 + k];
                    x[j] = acc / W[(c0 + j) * n + c0 + j];
                }
            }
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (j < w) W[i * n + c0 + j] = x[j];
        }
        __syncthreads();
        // ---- trailing update of the lower triangle ----------------------------------
        const int r0 = c0 + w;
        // rows of the trailing lower triangle round-robin over the warps, columns over lanes
        for (int i = r0 + warp; i < n; i += nwarp)
            for (int k = r0 + lane; k <= i; k += 32) {
            const float *li = W + i * n + c0, *lk = W + k * n + c0;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            int j = 0;
            for (; j + 3 < w; j += 4) {
                a0 += li[j] * lk[j];
                a1 += li[j + 1] * lk[j + 1];
                a2 += li[j + 2] * lk[j + 2];
                a3 += li[j + 3] * lk[j + 3];
            }
            for (; j < w; ++j) a0 += li[j] * lk[j];
            W[i * n + k] -= (a0 + a1) + (a2 + a3);
        }
        __syncthreads();
    }
    // ---- inverse: diagonal blocks, warp b, lane c = column c of X_bb ----------------
    for (int bb = warp; bb < nb; bb += nwarp) {
        const int c0 = 32 * bb, w = min(32, n - c0);
        float x[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            float v = 0.f;
            if (i < w && lane < w && i >= lane) {
                float acc = (i == lane) ? 1.f : 0.f;
#pragma unroll
                for (int k = 0; k < i; ++k)
                    if (k >= lane) acc -= W[(c0 + i) * n + c0 + k] * x[k];
                v = acc / W[(c0 + i) * n + c0 + i];
            }
            x[i] = v;
        }
        if (lane < w) {
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (i < w && i >= lane) X[(c0 + i) * n + c0 + lane] = x[i];
        }
    }
    __syncthreads();
    // ---- M[bi][k] = X_bi,bi L[bi][k] (k < bi), stored transposed in X's upper triangle
    for (int r = 32 + warp; r < n; r += nwarp)
        for (int c = lane; c < (r & ~31); c += 32) {  // (r, c) in the lower off-diagonal blocks
        const int bi = r >> 5;
        const int ri = 32 * bi;
        float a0 = 0.f, a1 = 0.f;
        int s2 = ri;
        for (; s2 + 1 <= r; s2 += 2) {
            a0 += X[r * n + s2] * W[s2 * n + c];
            a1 += X[r * n + s2 + 1] * W[(s2 + 1) * n + c];
        }
        if (s2 <= r) a0 += X[r * n + s2] * W[s2 * n + c];
        X[c * n + r] = a0 + a1;  // M^T
    }
    __syncthreads();
    // ---- off-diagonal blocks of X by block diagonal d ------------------------------
    for (int d = 1; d < nb; ++d) {
        // rows r of block bi >= d, columns c of block bj = bi - d
        for (int r = 32 * d + warp; r < n; r += nwarp) {
            const int bi = r >> 5, bj = bi - d;
            const int c = 32 * bj + lane;
            // sum over k = bj .. bi-1 (block rows), s in block k: M[bi](r, s) X(s, c);
            // the range is a whole number of 32-row blocks
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            const int s_end = 32 * bi;
            for (int s2 = 32 * bj; s2 < s_end; s2 += 4) {
                a0 += X[s2 * n + r] * X[s2 * n + c];
                a1 += X[(s2 + 1) * n + r] * X[(s2 + 1) * n + c];
                a2 += X[(s2 + 2) * n + r] * X[(s2 + 2) * n + c];
                a3 += X[(s2 + 3) * n + r] * X[(s2 + 3) * n + c];
            }
            X[r * n + c] = -((a0 + a1) + (a2 + a3));
        }
        __syncthreads();
    }
    for (int r = warp; r < n; r += nwarp)
        for (int c = lane; c < n; c += 32)  // Rinv[r][c] = X[c][r]
            Rinv[(size_t)r * n + c] = c >= r ? (double)X[c * n + r] : 0.0;
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
template <int TRANS>
__global__ void k_trimv(int n, const double *M, const double *y, double *out, int nr,
                        int accumulate, const double *outscale) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (gw >= n * nr) return;
    const int q = gw / n, i = gw % n;
    const double *yq = y + (size_t)q * n;
    double s = 0.0;
    if (TRANS == 0) {
        for (int k = i + lane; k < n; k += 32) s += M[(size_t)i * n + k] * yq[k];
    } else {
        for (int k = lane; k <= i; k += 32) s += M[(size_t)k * n + i] * yq[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        if (outscale) s *= outscale[i];
        double *o2 = out + (size_t)q * n + i;
        *o2 = accumulate ? *o2 + s : s;
    }
}

}  // namespace

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
        k_syrk_reduce<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(n, chunks, part, G);
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
    if (use_smem) DPM_CUDA(cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        DPM_PROF("lsq_cholesky", s);
        k_cholesky<<<1, 1024, use_smem ? smem : 0, s>>>(n, G, R, W, use_smem, status);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

// Mixed precision: column equilibration d (FP64), Gram of A D with FP32
// products (chunk sums in FP64), FP32 Cholesky; the refinement of every solve
// is FP64 against the original A (the factor only preconditions it).  Past
// the in-shared-memory size (2 n^2 floats) the Cholesky of the same Gram runs
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
    const size_t smem = 2 * nn * sizeof(float);
    const bool in_smem = smem <= 226 * 1024;
    // partials [chunks][n][n] floats, then G [n][n] (and W [n][n] for the FP64
    // Cholesky), then Af [n][m] floats
    const size_t gbytes = sizeof(double) * nn * (in_smem ? 1 : 2);
    DPM_RET(f.X.reserve(sizeof(float) * nn * (size_t)chunks + 16 + gbytes + sizeof(float) * (size_t)m * n));
    float *part = f.X.as<float>();
    double *G = reinterpret_cast<double *>(part + nn * chunks + (nn * chunks & 1));
    float *Af = reinterpret_cast<float *>(reinterpret_cast<char *>(G) + gbytes);
    {
        DPM_PROF("lsq_gram_syrk", s);
        k_colscale<<<n, 1024, 0, s>>>(m, A0, dscale);
        DPM_LAUNCHED();
        k_scale32<<<dim3(8, n), 256, 0, s>>>(m, A0, dscale, Af);
        DPM_LAUNCHED();
        k_syrk32_part<<<dim3(ntiles, chunks), 256, 0, s>>>(m, n, Af, rows_per, part);
        DPM_LAUNCHED();
        k_syrk_reduce32<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(n, chunks, part, G);
        DPM_LAUNCHED();
    }
    if (!in_smem) {
        DPM_PROF("lsq_cholesky", s);
        k_cholesky<<<1, 1024, 0, s>>>(n, G, R, G + nn, 0, status);
        DPM_LAUNCHED();
        *rinv_done = 0;
        return DPM_OK;
    }
    *rinv_done = 1;
    DPM_CUDA(cudaFuncSetAttribute(k_cholesky32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        DPM_PROF("lsq_cholesky", s);
        k_cholesky32<<<1, 1024, smem, s>>>(n, G, Rinv, status);
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
    //                   [z R*n][Rinv n*n][colscale n],  R = kLsqMaxRhs
    const size_t RR = kLsqMaxRhs;
    size_t need = sizeof(double) * ((size_t)m * n + 2 * (size_t)n + (size_t)n * n) + 64 +
                  sizeof(double) * RR * ((size_t)n + (size_t)m) + sizeof(double) * RR * (size_t)n +
                  sizeof(double) * (size_t)n * n + sizeof(double) * (size_t)n;
    DPM_RET(f.work.reserve(need));
    double *A0 = f.work.as<double>();
    double *w = A0 + (size_t)m * n;
    double *rdiag = w + n;
    double *R = rdiag + n;
    int *status = reinterpret_cast<int *>(R + (size_t)n * n);
    DPM_CUDA(cudaMemcpyAsync(A0, f.A.p, sizeof(double) * m * n, cudaMemcpyDeviceToDevice, s));
    DPM_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    double *Rinv = reinterpret_cast<double *>(reinterpret_cast<char *>(R + (size_t)n * n) + 64) +
                   kLsqMaxRhs * ((size_t)n + (size_t)m) + kLsqMaxRhs * (size_t)n;
    double *dscale = Rinv + (size_t)n * n;
    f.equilibrated = false;
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
        if (smem > 48 * 1024)
            DPM_CUDA(cudaFuncSetAttribute(k_rinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
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
    const double *A0 = f.work.as<double>();
    const double *R = A0 + (size_t)m * n + 2 * (size_t)n;
    int *status = reinterpret_cast<int *>(const_cast<double *>(R) + (size_t)n * n);
    if (nr < 1 || nr > kLsqMaxRhs) { set_error("least squares: 1..%d right-hand sides per call", kLsqMaxRhs); return DPM_EINVAL; }
    // scratch after the factor: y[nr][n], res[nr][m]
    size_t base = sizeof(double) * ((size_t)m * n + 2 * (size_t)n + (size_t)n * n) + 64;
    double *y = reinterpret_cast<double *>(static_cast<char *>(f.work.p) + base);
    double *res = y + kLsqMaxRhs * (size_t)n;
    double *z = res + kLsqMaxRhs * (size_t)m;
    const double *Rinv = z + kLsqMaxRhs * (size_t)n;
    (void)status;
    const int mv_blocks = (n * nr * 32 + 255) / 256;
    const double *dsc = f.equilibrated ? Rinv + (size_t)n * n : nullptr;
    // FP64 refinement steps: each contracts the error by ~kappa(AD)^2 eps_32.
    // One leaves C ~1e-11 relative, far below the FP32 solver's error; the
    // FP64 path takes three.
    const int refine = f.equilibrated ? (sizeof(T) == sizeof(double) ? 3 : 1) : 1;
    DPM_PROF("lsq_solve", s);
    // C = D R^{-1} R^{-T} D A^T b   (D = I unless the factor was equilibrated)
    k_atb<T><<<dim3(n, nr), 1024, 0, s>>>(m, n, A0, b, ldb, y, nr, dsc);
    DPM_LAUNCHED();
    k_trimv<1><<<mv_blocks, 256, 0, s>>>(n, Rinv, y, z, nr, 0, nullptr);
    DPM_LAUNCHED();
    k_trimv<0><<<mv_blocks, 256, 0, s>>>(n, Rinv, z, C, nr, 0, dsc);
    DPM_LAUNCHED();
    // iterative refinement: C += D R^{-1} R^{-T} D A^T (b - A C), all in FP64
    for (int it = 0; it < refine; ++it) {
        k_resid<T><<<dim3((m + 255) / 256, nr), 256, 0, s>>>(m, n, A0, b, ldb, C, res, nr);
        DPM_LAUNCHED();
        k_atb<double><<<dim3(n, nr), 1024, 0, s>>>(m, n, A0, res, m, y, nr, dsc);
        DPM_LAUNCHED();
        k_trimv<1><<<mv_blocks, 256, 0, s>>>(n, Rinv, y, z, nr, 0, nullptr);
        DPM_LAUNCHED();
        k_trimv<0><<<mv_blocks, 256, 0, s>>>(n, Rinv, z, C, nr, 1, dsc);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

template int lsq_apply<float>(const LsqFactor &, const float *, int, double *, int, cudaStream_t);
template int lsq_apply<double>(const LsqFactor &, const double *, int, double *, int, cudaStream_t);

}  // namespace dpm
