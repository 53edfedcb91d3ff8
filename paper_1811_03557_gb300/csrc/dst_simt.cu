// SIMT auxiliary-problem solver (Definition 2.4): (sigma - Lap_h) u = q on
// M^0, u = 0 on N^0 \ M^0, by the 3D DST-I,
//   u = (2/(N+1))^3 S_x S_y S_z [ (S_x S_y S_z q) / lambda ],
//   S[a][m] = sin(pi a m/(N+1)),
//   lambda_abc = sigma + (4/h^2)(s_a + s_b + s_c), s_a = sin^2(pi a/(2(N+1))).
//
// Five passes over a [B][N][N][N] workspace, each a per-tile dense transform
// along one axis staged in shared memory:
//   1. k (contiguous) forward, with the right-hand side built in the tile:
//      q = fscale*f on M^+ (eq. rhs:particular_solution) plus L[v_gamma] on
//      the M^- shell (eq. rhs:difference_potentials) from a density on gamma;
//   2. j forward;  3. i forward, times (2/(N+1))^3/lambda, i inverse;
//   4. j inverse;  5. k inverse, with the restriction to N^+ and the trace on
//      gamma_in (Tr operators of Section 2) fused into the store.
//
// Each 1D transform uses the symmetry S[a][N+1-m] = (-1)^(a+1) S[a][m]:
// folding x_m +- x_{N+1-m} first halves the multiply-adds (odd a read the
// sums, even a the differences; for odd N the middle node joins odd a only).
// N+1 = 33, 129, 257 have no radix-2 structure beyond this fold, so the rest
// of each transform is a dense product with the folded sine table.  Tiles
// arrive by asynchronous element copies; the table reaches the product through
// shared memory in double-buffered chunks of rows (see stage_rows).
//
// FP32 grids of N <= 32 take one pass instead (small_body): the whole cube in
// shared memory, the six transforms line by line, 8 N^3 bytes of HBM traffic.
#include <algorithm>
#include <map>
#include <math.h>
#include <mutex>
#include <stdlib.h>
#include <type_traits>
#include <tuple>
#include <utility>
#include <vector>

#include "dpm_internal.cuh"

namespace dpm {

// ---------------------------------------------------------------------------
// Folded sine tables: SE[m'][a'] = S[2a'+1][m'+1] (odd a, sums), with an extra
// row m' = H for the middle node when N is odd; SO[m'][a'] = S[2a'+2][m'+1]
// (even a, differences).  a' padded to a multiple of 4 with zeros.
// ---------------------------------------------------------------------------
struct FoldDims {
    int H, NE, NO, NEp, NOp, rowsE;
    __host__ __device__ FoldDims(int N) {
        H = N / 2;
        NE = (N + 1) / 2;
        NO = N / 2;
        NEp = (NE + 3) & ~3;
        NOp = (NO + 3) & ~3;
        rowsE = H + (N & 1);
    }
    __host__ __device__ size_t offO() const { return (size_t)rowsE * NEp; }
    __host__ __device__ size_t offW() const { return offO() + (size_t)H * NOp; }
    // followed by N weights sin^2(pi (n+1)/(2(N+1)))
    __host__ __device__ size_t total(int N) const { return offW() + (size_t)N; }
};

static double sin_pi_frac(long long num, long long den) {
    // sin(pi num/den) with the argument reduced exactly modulo 2 den
    long long r = num % (2 * den);
    return sin(M_PI * (double)r / (double)den);
}

template <class T> const T *dst_fold_table(int N) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, void *> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, N);
    auto it = cache.find(key);
    if (it != cache.end()) return static_cast<const T *>(it->second);
    FoldDims fd(N);
    std::vector<T> h(fd.total(N), (T)0);
    for (int mp = 0; mp < fd.rowsE; ++mp)
        for (int ap = 0; ap < fd.NE; ++ap)
            h[(size_t)mp * fd.NEp + ap] = (T)sin_pi_frac((long long)(2 * ap + 1) * (mp + 1), N + 1);
    for (int mp = 0; mp < fd.H; ++mp)
        for (int ap = 0; ap < fd.NO; ++ap)
            h[fd.offO() + (size_t)mp * fd.NOp + ap] =
                (T)sin_pi_frac((long long)(2 * ap + 2) * (mp + 1), N + 1);
    for (int n = 0; n < N; ++n) {
        double sn = sin(M_PI * (double)(n + 1) / (2.0 * (N + 1)));
        h[fd.offW() + n] = (T)(sn * sn);
    }
    void *d = nullptr;
    if (cudaMalloc(&d, h.size() * sizeof(T)) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    cache[key] = d;
    return static_cast<const T *>(d);
}
template const float *dst_fold_table<float>(int);
template const double *dst_fold_table<double>(int);

namespace {

constexpr int kThreads = 512;

template <class T> struct V4 { T v[4]; };

__device__ __forceinline__ V4<float> ld4(const float *p) {
    float4 a = *reinterpret_cast<const float4 *>(p);
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ld4(const double *p) {
    double2 a = *reinterpret_cast<const double2 *>(p);
    double2 b = *reinterpret_cast<const double2 *>(p + 2);
    return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float *p, const float *v) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *p, const double *v) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
}

// The folded sine tables reach the transforms through shared memory, KC table
// rows (fold indices m') at a time: both parities' rows [m0, m0 + KC) are one
// contiguous run each in the table, copied with 16-byte cp.async (L2 only)
// into one of two buffers while the other is being read.  Every thread of the
// CTA reads every staged row, so the table crosses the L2 -> SM path once per
// tile and transform instead of once per warp that misses in L1 (the tiles
// leave L1 too small to hold a table of N > 128).
template <class T> __host__ __device__ constexpr int kc_rows() { return sizeof(T) == 4 ? 16 : 8; }
template <class T> __host__ __device__ size_t chunk_elems(int N) {  // one buffer
    const FoldDims fd(N);
    return (size_t)kc_rows<T>() * (fd.NEp + fd.NOp);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// One element global -> shared, asynchronously; valid = false writes zero and
// reads nothing (src must still be a global address).  The tiles' loads are
// issued this way, all of a thread's elements in flight at once, instead of
// one dependent HBM round trip per element.
__device__ __forceinline__ void cp_async_elem(float *dst, const float *src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double *dst, const double *src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copy table rows [m0, m0 + KC) into sb: SE rows (m' < rowsE) at [0, KC NEp),
// SO rows (m' < H) at [KC NEp, KC (NEp + NOp)).  Rows past the end are not copied
// and never read.
template <class T>
__device__ __forceinline__ void stage_rows(T *sb, const T *tab, const FoldDims &fd, int m0) {
    constexpr int KC = kc_rows<T>(), V = 16 / (int)sizeof(T);
    const int nE = max(0, min(KC, fd.rowsE - m0)) * (fd.NEp / V);
    const int nO = max(0, min(KC, fd.H - m0)) * (fd.NOp / V);
    const T *srcE = tab + (size_t)m0 * fd.NEp, *srcO = tab + fd.offO() + (size_t)m0 * fd.NOp;
    T *dO = sb + KC * fd.NEp;
    for (int v = threadIdx.x; v < nE + nO; v += blockDim.x) {
        if (v < nE) cp_async16(sb + v * V, srcE + v * V);
        else cp_async16(dO + (v - nE) * V, srcO + (v - nE) * V);
    }
    cp_async_commit();
}

// 4 x 4 FP32 accumulators of a contraction task, acc[i][j] += s[i] x[j], with the
// pairs of lines (0, 1) and (2, 3) as packed two-lane FMAs, each lane rounding as
// fmaf does (bit-identical to the scalar loop).  Measured on
// GB300: 3.5 % faster in the grouped kernels, 5 % slower in the single-grid ones
// (the register allocation of the surrounding kernel), so only the grouped
// kernels take it.
struct Acc4Packed {
    float2 a[4][2] = {};
    __device__ __forceinline__ void fma(const V4<float> &sv, const float (&xv)[4]) {
        const float2 x01 = make_float2(xv[0], xv[1]), x23 = make_float2(xv[2], xv[3]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 si = make_float2(sv.v[i], sv.v[i]);
            a[i][0] = __ffma2_rn(si, x01, a[i][0]);
            a[i][1] = __ffma2_rn(si, x23, a[i][1]);
        }
    }
    __device__ __forceinline__ void get(float (&o)[4][4]) const {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            o[i][0] = a[i][0].x;
            o[i][1] = a[i][0].y;
            o[i][2] = a[i][1].x;
            o[i][3] = a[i][1].y;
        }
    }
};

// The contraction of a folded tile against the staged table.  A task is 4
// output modes (a' block ab: the sums' modes for ab < NEp/4, the differences'
// after) x 4 tile lines (block lb); xfirst(even) and xstep(even) give the
// first folded operand of the task's lines and the stride between fold indices;
// X(xp, mm) reads the 4 operands of fold index mm; put(abp, even, acc) stores.
// Per output the terms are summed in the order m' = 0, 1, ... (the middle node
// of odd N last among the sums).
template <class T, int C, bool P, class XFirst, class Load, class Put>
__device__ __forceinline__ void tile_contract(const T *tab, T *sb, const FoldDims &fd, XFirst xfirst,
                                              int xstep_e, int xstep_o, Load load, Put put) {
    constexpr int KC = kc_rows<T>();
    const int nabE = fd.NEp / 4, nabO = fd.NOp / 4;
    const int ntask = (nabE + nabO) * (C / 4);
    const int nchunk = (fd.rowsE + KC - 1) / KC;
    const size_t half = (size_t)KC * (fd.NEp + fd.NOp);
    for (int t0 = 0; t0 < ntask; t0 += blockDim.x) {  // rounds: block-uniform
        if (t0 > 0) {
            __syncthreads();  // the previous round has read both buffers
            stage_rows(sb, tab, fd, 0);
        }
        const int t = t0 + (int)threadIdx.x;
        const bool live = t < ntask;
        const int lb = t % (C / 4), ab = t / (C / 4);
        const bool even = ab < nabE;
        const int abp = even ? ab : ab - nabE;
        const int soff = even ? 4 * abp : KC * fd.NEp + 4 * abp;
        const int lds = even ? fd.NEp : fd.NOp;
        const int mend = even ? fd.rowsE : fd.H;
        const int xstep = even ? xstep_e : xstep_o;
        const T *xp = xfirst(even, lb);
        // acc[i][j]: mode i, line j
        constexpr bool kPacked = P && sizeof(T) == 4;
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
        Acc4Packed pk;
        for (int c = 0; c < nchunk; ++c) {
            cp_async_wait_all();
            __syncthreads();  // chunk c has landed; every thread is done with chunk c - 1
            if (c + 1 < nchunk) stage_rows(sb + ((c + 1) & 1) * half, tab, fd, (c + 1) * KC);
            const int m0 = c * KC;
            const int mc = live ? min(KC, mend - m0) : 0;
            const T *sp = sb + (c & 1) * half + soff;
            for (int mm = 0; mm < mc; ++mm, xp += xstep, sp += lds) {
                const V4<T> sv = ld4(sp);
                T xv[4];
                load(xp, xv);
                if constexpr (kPacked) {
                    pk.fma(sv, xv);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fma(sv.v[i], xv[j], acc[i][j]);
                }
            }
        }
        if (live) {
            if constexpr (kPacked) pk.get(acc);
            put(abp, even, lb, acc);
        }
    }
}

// Column-major tile: x[m][c] (m = transform index, C columns, row stride C).
// out[a][c] = sum_m S[a][m] x[m][c].  x is folded in place; sb: two table
// chunks of shared memory.  blockDim.x is a multiple of C.
template <class T, int C = 32, bool P = false>
__device__ void tile_transform_cm(T *x, T *out, int N, const T *tab, T *sb) {
    FoldDims fd(N);
    stage_rows(sb, tab, fd, 0);
    {
        const int c = threadIdx.x % C, R = blockDim.x / C;  // a fixed column per thread
        for (int mp = threadIdx.x / C; mp < fd.H; mp += R) {
            T a = x[mp * C + c], b = x[(N - 1 - mp) * C + c];
            x[mp * C + c] = a + b;
            x[(N - 1 - mp) * C + c] = a - b;
        }
    }
    // (the first barrier of the contraction orders the fold before its reads)
    tile_contract<T, C, P>(
        tab, sb, fd, [&](bool even, int cb) -> const T * { return x + (even ? 0 : (N - 1) * C) + 4 * cb; },
        C, -C,
        [](const T *xp, T *xv) {
            const V4<T> v = ld4(xp);
#pragma unroll
            for (int j = 0; j < 4; ++j) xv[j] = v.v[j];
        },
        [&](int abp, bool even, int cb, T (&acc)[4][4]) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int a0 = even ? 2 * (4 * abp + i) : 2 * (4 * abp + i) + 1;
                if (a0 < N) st4(out + a0 * C + 4 * cb, acc[i]);
            }
        });
    __syncthreads();
}

// Row-major tile: x[r][m] (C rows, row stride ld = N + 1).
// out[r][a] = sum_m S[a][m] x[r][m].  x is folded in place; sb as above.
template <class T, int C = 32, bool P = false>
__device__ void tile_transform_rm(T *x, T *out, int N, int ld, const T *tab, T *sb) {
    FoldDims fd(N);
    stage_rows(sb, tab, fd, 0);
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < C; r += nw) {  // a warp per row: no division by N
        T *xr = x + r * ld;
        for (int mp = lane; mp < fd.H; mp += 32) {
            T a = xr[mp], b = xr[N - 1 - mp];
            xr[mp] = a + b;
            xr[N - 1 - mp] = a - b;
        }
    }
    tile_contract<T, C, P>(
        tab, sb, fd, [&](bool even, int rb) -> const T * { return x + 4 * rb * ld + (even ? 0 : N - 1); },
        1, -1,
        [ld](const T *xp, T *xv) {
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[i] = xp[i * ld];
        },
        [&](int abp, bool even, int rb, T (&acc)[4][4]) {
            // acc[j][i]: mode 4 abp + j of row 4 rb + i
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int a0 = even ? 2 * (4 * abp + j) : 2 * (4 * abp + j) + 1;
                if (a0 < N) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) out[(4 * rb + i) * ld + a0] = acc[j][i];
                }
            }
        });
    __syncthreads();
}

template <class T>
__device__ __forceinline__ bool rhs_skipped(const ApRhs<T> &r, const int *flag) {
    return r.cond && flag && *flag == 0;
}

struct PassArgs {
    int N, B;
    double h, sigma, fscale;
    const double *sigma_dev, *fscale_dev;
    const int *cond_flag;
    int mask_f, mask_out;
    const uint8_t *labels;
    const int *shell, *shell_nb, *rp_shell, *gin, *rp_gin;
};

// Each pass is a device body over one tile of one right-hand side (its cube at
// `cube`), run by a single-problem kernel (every right-hand side on one grid)
// or by a grouped kernel (right-hand sides of grids of different N in one
// launch, each with its own parameters).
// Pass 1: right-hand side + forward transform along k.
template <class T, int C, bool P = false>
__device__ __forceinline__ void body_k_fwd(const PassArgs &a, const ApRhs<T> &r, T *cube, const T *tab,
                                           int tile) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, ld = N + 1;
    if (rhs_skipped(r, a.cond_flag)) return;
    T *x = reinterpret_cast<T *>(smem_raw);
    T *out = x + C * ld;
    T *sb = out + C * ld;
    const int64_t nrows = (int64_t)N * N;
    const int64_t R0 = (int64_t)tile * C;
    const double sig = a.sigma_dev ? *a.sigma_dev : a.sigma;
    const T fs = (T)(a.fscale_dev ? *a.fscale_dev : a.fscale);
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (r.f) {
        // f copied in, then scaled and masked by the thread that copied it
        for (int rr = threadIdx.x >> 5; rr < C; rr += nw) {  // a warp per row: no division by N
            const int64_t R = R0 + rr;
            for (int k = lane; k < N; k += 32)
                cp_async_elem(x + rr * ld + k, R < nrows ? r.f + R * N + k : r.f, R < nrows);
        }
        cp_async_commit();
        cp_async_wait_all();
        for (int rr = threadIdx.x >> 5; rr < C; rr += nw) {
            const int64_t R = R0 + rr;
            if (R >= nrows) break;
            for (int k = lane; k < N; k += 32) {
                const int64_t p = R * N + k;
                T v = fs * x[rr * ld + k];
                if (a.mask_f && !(a.labels[p] & DPM_LBL_MPLUS)) v = (T)0;
                x[rr * ld + k] = v;
            }
        }
    } else {
        for (int rr = threadIdx.x >> 5; rr < C; rr += nw)
            for (int k = lane; k < N; k += 32) x[rr * ld + k] = (T)0;
    }
    __syncthreads();
    if (r.dens) {
        const T cdiag = (T)(sig + 6.0 / (a.h * a.h));
        const T coff = (T)(1.0 / (a.h * a.h));
        int64_t Rend = R0 + C < nrows ? R0 + C : nrows;
        int e0 = a.rp_shell[R0], e1 = a.rp_shell[Rend];
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            int p = a.shell[e];
            const int *nb = a.shell_nb + 8 * (size_t)e;
            T s = (T)0;
#pragma unroll
            for (int t = 1; t < 7; ++t) {
                int g = nb[t];
                if (g >= 0) s += r.dens[g];
            }
            T self = nb[0] >= 0 ? r.dens[nb[0]] : (T)0;
            int rr = (int)(p / N - R0), k = p % N;
            x[rr * ld + k] += cdiag * self - coff * s;
        }
        __syncthreads();
    }
    tile_transform_rm<T, C, P>(x, out, N, ld, tab, sb);
    T *w = cube;
    for (int rr = threadIdx.x >> 5; rr < C; rr += nw) {
        const int64_t R = R0 + rr;
        if (R >= nrows) break;
        for (int k = lane; k < N; k += 32) w[R * N + k] = out[rr * ld + k];
    }
}

// Passes 2 and 4: transform along j for tiles [j][kc..kc+C) at fixed i.
template <class T, int C, bool P = false>
__device__ __forceinline__ void body_j(const PassArgs &a, const ApRhs<T> &r, T *cube, const T *tab, int tile) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N;
    if (rhs_skipped(r, a.cond_flag)) return;
    const int nkc = (N + C - 1) / C;
    const int i = tile / nkc, kc = (tile % nkc) * C;
    T *x = reinterpret_cast<T *>(smem_raw);
    T *out = x + N * C;
    T *sb = out + N * C;
    T *w = cube + (size_t)i * N * N;
    const int c = threadIdx.x % C, R = blockDim.x / C;  // a fixed column per thread
    const bool cv = kc + c < N;
    for (int j = threadIdx.x / C; j < N; j += R)
        cp_async_elem(x + j * C + c, cv ? w + (size_t)j * N + kc + c : w, cv);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    tile_transform_cm<T, C, P>(x, out, N, tab, sb);
    if (cv)
        for (int j = threadIdx.x / C; j < N; j += R) w[(size_t)j * N + kc + c] = out[j * C + c];
}

// Pass 3: along i, forward, scale/lambda, inverse; tiles [i][kc..kc+C) at fixed j.
template <class T, int C, bool P = false>
__device__ __forceinline__ void body_i(const PassArgs &a, const ApRhs<T> &r, T *cube, const T *tab, int tile) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N;
    if (rhs_skipped(r, a.cond_flag)) return;
    const int nkc = (N + C - 1) / C;
    const int j = tile / nkc, kc = (tile % nkc) * C;
    T *x = reinterpret_cast<T *>(smem_raw);
    T *out = x + N * C;
    T *wt = out + N * C;  // N weights (4/h^2) sin^2(pi (n+1)/(2(N+1)))
    T *sb = wt + ((N + 3) & ~3);
    T *w = cube + (size_t)j * N;
    const size_t si = (size_t)N * N;
    const double sig = a.sigma_dev ? *a.sigma_dev : a.sigma;
    const T w4 = (T)(4.0 / (a.h * a.h));
    const T *s2 = tab + FoldDims(N).offW();
    for (int n = threadIdx.x; n < N; n += blockDim.x) wt[n] = w4 * s2[n];
    const int c = threadIdx.x % C, R = blockDim.x / C;  // a fixed column per thread
    const bool cv = kc + c < N;
    for (int i = threadIdx.x / C; i < N; i += R)
        cp_async_elem(x + i * C + c, cv ? w + (size_t)i * si + kc + c : w, cv);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    tile_transform_cm<T, C, P>(x, out, N, tab, sb);
    const double sc = 2.0 / (N + 1);
    const T scale = (T)(sc * sc * sc);
    const T sgT = (T)sig;
    {
        const int kk = cv ? kc + c : N - 1;
        const T wj = wt[j], wk = wt[kk];
        for (int ai = threadIdx.x / C; ai < N; ai += R) {
            T lam = sgT + (wt[ai] + wj + wk);
            x[ai * C + c] = out[ai * C + c] * (scale / lam);
        }
    }
    __syncthreads();
    tile_transform_cm<T, C, P>(x, out, N, tab, sb);
    if (cv)
        for (int i = threadIdx.x / C; i < N; i += R) w[(size_t)i * si + kc + c] = out[i * C + c];
}

// Pass 5: inverse along k, then the dense output (masked to N^+) and/or the
// trace on gamma_in.
template <class T, int C, bool P = false>
__device__ __forceinline__ void body_k_inv(const PassArgs &a, const ApRhs<T> &r, const T *cube, const T *tab,
                                           int tile) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, ld = N + 1;
    if (rhs_skipped(r, a.cond_flag)) return;
    T *x = reinterpret_cast<T *>(smem_raw);
    T *out = x + C * ld;
    T *sb = out + C * ld;
    const int64_t nrows = (int64_t)N * N;
    const int64_t R0 = (int64_t)tile * C;
    const T *w = cube;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int rr = threadIdx.x >> 5; rr < C; rr += nw) {  // a warp per row: no division by N
        const int64_t R = R0 + rr;
        for (int k = lane; k < N; k += 32) cp_async_elem(x + rr * ld + k, R < nrows ? w + R * N + k : w, R < nrows);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    tile_transform_rm<T, C, P>(x, out, N, ld, tab, sb);
    if (r.out_dense) {
        for (int rr = threadIdx.x >> 5; rr < C; rr += nw) {
            const int64_t R = R0 + rr;
            if (R >= nrows) break;
            for (int k = lane; k < N; k += 32) {
                const int64_t p = R * N + k;
                T v = out[rr * ld + k];
                if (a.mask_out && !(a.labels[p] & (DPM_LBL_MPLUS | DPM_LBL_GEX))) v = (T)0;
                r.out_dense[p] = v;
            }
        }
    }
    if (r.out_trace) {
        int64_t Rend = R0 + C < nrows ? R0 + C : nrows;
        int e0 = a.rp_gin[R0], e1 = a.rp_gin[Rend];
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            int p = a.gin[e];
            int rr = (int)(p / N - R0), k = p % N;
            r.out_trace[e] = out[rr * ld + k];
        }
    }
}

template <class T, int C = 32>
__global__ void __launch_bounds__(kThreads) k_pass_k_fwd(PassArgs a, const ApRhs<T> *rhs, T *work,
                                                         const T *tab) {
    const int b = blockIdx.y;
    body_k_fwd<T, C>(a, rhs[b], work + (size_t)b * a.N * a.N * a.N, tab, blockIdx.x);
}
template <class T, int C = 32>
__global__ void __launch_bounds__(kThreads) k_pass_j(PassArgs a, const ApRhs<T> *rhs, T *work, const T *tab) {
    const int b = blockIdx.y;
    body_j<T, C>(a, rhs[b], work + (size_t)b * a.N * a.N * a.N, tab, blockIdx.x);
}
template <class T, int C = 32>
__global__ void __launch_bounds__(kThreads) k_pass_i(PassArgs a, const ApRhs<T> *rhs, T *work, const T *tab) {
    const int b = blockIdx.y;
    body_i<T, C>(a, rhs[b], work + (size_t)b * a.N * a.N * a.N, tab, blockIdx.x);
}
template <class T, int C = 32>
__global__ void __launch_bounds__(kThreads) k_pass_k_inv(PassArgs a, const ApRhs<T> *rhs, const T *work,
                                                         const T *tab) {
    const int b = blockIdx.y;
    body_k_inv<T, C>(a, rhs[b], work + (size_t)b * a.N * a.N * a.N, tab, blockIdx.x);
}

// Grouped launches: item b carries its own grid's parameters, right-hand side,
// cube and sine table; CTAs past the item's tile count return at once.
// Grids of up to kSmallN points per axis solve in one pass in shared memory
// (FP32; see small_body).
constexpr int kSmallN = 32;
template <class T> __host__ __device__ __forceinline__ bool small_item(int N) {
    return sizeof(T) == 4 && N <= kSmallN;
}

template <class T> struct GroupItem {
    PassArgs a;
    ApRhs<T> r;
    T *cube;
    const T *tab;
};
template <int C> __host__ __device__ __forceinline__ int row_tiles(int N) { return (N * N + C - 1) / C; }
template <int C> __host__ __device__ __forceinline__ int col_tiles(int N) { return N * ((N + C - 1) / C); }

template <class T, int C>
__global__ void __launch_bounds__(kThreads) kg_pass_k_fwd(const GroupItem<T> *items) {
    const GroupItem<T> &g = items[blockIdx.y];
    if ((int)blockIdx.x >= row_tiles<C>(g.a.N) || small_item<T>(g.a.N)) return;  // small grids: kg_small
    body_k_fwd<T, C, true>(g.a, g.r, g.cube, g.tab, blockIdx.x);
}
template <class T, int C>
__global__ void __launch_bounds__(kThreads) kg_pass_j(const GroupItem<T> *items) {
    const GroupItem<T> &g = items[blockIdx.y];
    if ((int)blockIdx.x >= col_tiles<C>(g.a.N) || small_item<T>(g.a.N)) return;  // small grids: kg_small
    body_j<T, C, true>(g.a, g.r, g.cube, g.tab, blockIdx.x);
}
template <class T, int C>
__global__ void __launch_bounds__(kThreads) kg_pass_i(const GroupItem<T> *items) {
    const GroupItem<T> &g = items[blockIdx.y];
    if ((int)blockIdx.x >= col_tiles<C>(g.a.N) || small_item<T>(g.a.N)) return;  // small grids: kg_small
    body_i<T, C, true>(g.a, g.r, g.cube, g.tab, blockIdx.x);
}
template <class T, int C>
__global__ void __launch_bounds__(kThreads) kg_pass_k_inv(const GroupItem<T> *items) {
    const GroupItem<T> &g = items[blockIdx.y];
    if ((int)blockIdx.x >= row_tiles<C>(g.a.N) || small_item<T>(g.a.N)) return;  // small grids: kg_small
    body_k_inv<T, C, true>(g.a, g.r, g.cube, g.tab, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Single-pass solve for small grids (FP32, N <= kSmallN): one CTA per
// right-hand side keeps the whole cube in shared memory (row pitch P = N + 1 or
// N + 2, odd, so that the lines of every axis are read without bank
// conflicts), builds q there as pass 1 does, runs the six 1D transforms line
// by line from registers (k and j forward; i forward, times
// (2/(N+1))^3/lambda, i inverse; j and k inverse) and writes u and/or the trace
// as pass 5 does.  The cube crosses HBM once each way: 8 N^3 bytes per
// right-hand side instead of the five passes' 40 N^3.
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 512;
__host__ __device__ __forceinline__ int small_pitch(int N) { return (N & 1) ? N + 2 : N + 1; }
inline size_t small_smem(int N) { return sizeof(float) * ((size_t)N * N * small_pitch(N) + 2 * 256 + 32); }

// Shared-memory layout of the one-pass solve: SE (16 x 16), SO (16 x 16), 32
// weights, then the cube.
constexpr int kSmallCube = 2 * 256 + 32;  // float offset of the cube

// Two lines x[m * st] (m < N) of the cube, starting at float offsets off0 and off1
// (off1 < 0: one line), in place: y[a] = sum_m S[a+1][m+1] x[m] (0-based a), by the
// fold -- sums e against SE (odd modes a+1), differences o against SO (even modes)
// -- with SE, SO 16 x 16 and zero-padded; every output sums over m' in order.  Two
// lines per call make each table load feed eight FMAs.  Out of line (it keeps 512
// threads per CTA within 128 registers); its pointers come from the shared array
// itself, so every access is a shared-memory one.
__device__ __noinline__ void small_line2(int off0, int off1, int st, int N) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const float *SE = reinterpret_cast<const float *>(smem_raw);
    const float *SO = SE + 256;
    float *x0 = reinterpret_cast<float *>(smem_raw) + kSmallCube + off0;
    float *x1 = reinterpret_cast<float *>(smem_raw) + kSmallCube + (off1 < 0 ? off0 : off1);
    const bool two = off1 >= 0;
    const int H = N >> 1;
    float e0[16], o0[16], e1[16], o1[16];
#pragma unroll
    for (int mp = 0; mp < 16; ++mp) {
        float u0 = 0.f, v0 = 0.f, u1 = 0.f, v1 = 0.f;
        if (mp < H) {
            u0 = x0[mp * st];
            v0 = x0[(N - 1 - mp) * st];
            u1 = x1[mp * st];
            v1 = x1[(N - 1 - mp) * st];
        } else if (mp == H && (N & 1)) {
            u0 = x0[mp * st];  // the middle node of an odd line joins the sums only
            u1 = x1[mp * st];
        }
        e0[mp] = u0 + v0;
        o0[mp] = u0 - v0;
        e1[mp] = u1 + v1;
        o1[mp] = u1 - v1;
    }
    // odd modes from the sums, stored, then even modes from the differences (every
    // input is in registers already, so the in-place stores are safe)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const float *T = half ? SO : SE;
        float y0[16], y1[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            y0[q] = 0.f;
            y1[q] = 0.f;
        }
#pragma unroll
        for (int mp = 0; mp < 16; ++mp) {
            const float4 *tr = reinterpret_cast<const float4 *>(T + mp * 16);
            const float a0 = half ? o0[mp] : e0[mp], a1 = half ? o1[mp] : e1[mp];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 s4 = tr[q];
                y0[4 * q] = fmaf(s4.x, a0, y0[4 * q]);
                y0[4 * q + 1] = fmaf(s4.y, a0, y0[4 * q + 1]);
                y0[4 * q + 2] = fmaf(s4.z, a0, y0[4 * q + 2]);
                y0[4 * q + 3] = fmaf(s4.w, a0, y0[4 * q + 3]);
                y1[4 * q] = fmaf(s4.x, a1, y1[4 * q]);
                y1[4 * q + 1] = fmaf(s4.y, a1, y1[4 * q + 1]);
                y1[4 * q + 2] = fmaf(s4.z, a1, y1[4 * q + 2]);
                y1[4 * q + 3] = fmaf(s4.w, a1, y1[4 * q + 3]);
            }
        }
#pragma unroll
        for (int ap = 0; ap < 16; ++ap) {
            const int a = 2 * ap + half;
            if (a < N) {
                x0[a * st] = y0[ap];
                if (two) x1[a * st] = y1[ap];
            }
        }
    }
}

__device__ void small_body(const PassArgs &a, const ApRhs<float> &r, const float *tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (rhs_skipped(r, a.cond_flag)) return;
    const int N = a.N, P = small_pitch(N), L = N * N, Lp = (L + 1) / 2;  // lines, line pairs (l, l + Lp)
    const FoldDims fd(N);
    float *SE = reinterpret_cast<float *>(smem_raw);  // 16 x 16
    float *SO = SE + 256;                              // 16 x 16
    float *w = SO + 256;                               // 32 weights (4/h^2) sin^2(pi (n+1)/(2(N+1)))
    float *x = SE + kSmallCube;                        // the cube, x[(i N + j) P + k]
    const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, warp = t >> 5, nw = nt >> 5;
    const double sig = a.sigma_dev ? *a.sigma_dev : a.sigma;
    const float fs = (float)(a.fscale_dev ? *a.fscale_dev : a.fscale);
    for (int q = t; q < 256; q += nt) {
        const int mp = q >> 4, ap = q & 15;
        SE[q] = (mp < fd.rowsE && ap < fd.NE) ? tab[(size_t)mp * fd.NEp + ap] : 0.f;
        SO[q] = (mp < fd.H && ap < fd.NO) ? tab[fd.offO() + (size_t)mp * fd.NOp + ap] : 0.f;
    }
    const float w4 = (float)(4.0 / (a.h * a.h));
    for (int n = t; n < 32; n += nt) w[n] = n < N ? w4 * tab[fd.offW() + n] : 0.f;
    // q = fscale f on M^+ (everywhere without the mask), as pass 1 builds it
    for (int row = warp; row < L; row += nw)
        for (int k = lane; k < N; k += 32) {
            float v = 0.f;
            if (r.f) {
                const int p = row * N + k;
                v = fs * r.f[p];
                if (a.mask_f && !(a.labels[p] & DPM_LBL_MPLUS)) v = 0.f;
            }
            x[row * P + k] = v;
        }
    __syncthreads();
    if (r.dens) {  // + L[v_gamma] on the M^- shell
        const float cdiag = (float)(sig + 6.0 / (a.h * a.h));
        const float coff = (float)(1.0 / (a.h * a.h));
        const int e0 = a.rp_shell[0], e1 = a.rp_shell[L];
        for (int e = e0 + t; e < e1; e += nt) {
            const int p = a.shell[e];
            const int *nb = a.shell_nb + 8 * (size_t)e;
            float sum = 0.f;
#pragma unroll
            for (int u = 1; u < 7; ++u) {
                const int g = nb[u];
                if (g >= 0) sum += r.dens[g];
            }
            const float self = nb[0] >= 0 ? r.dens[nb[0]] : 0.f;
            x[(p / N) * P + p % N] += cdiag * self - coff * sum;
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int l = t; l < Lp; l += nt) small_line2(l * P, l + Lp < L ? (l + Lp) * P : -1, 1, N);  // k
    __syncthreads();
#pragma unroll 1
    for (int l = t; l < Lp; l += nt) {  // j
        const int l1 = l + Lp;
        small_line2((l / N) * N * P + l % N, l1 < L ? (l1 / N) * N * P + l1 % N : -1, P, N);
    }
    __syncthreads();
    {
        const double sc = 2.0 / (N + 1);
        const float scale = (float)(sc * sc * sc);
        const float sgT = (float)sig;
#pragma unroll 1
        for (int l = t; l < Lp; l += nt) {  // i: forward, / lambda, inverse
            const int st = N * P, l1 = l + Lp;
            const int b0 = l / N, c0 = l % N, b1 = l1 / N, c1 = l1 % N;
            const int off1 = l1 < L ? b1 * P + c1 : -1;
            small_line2(b0 * P + c0, off1, st, N);
            for (int ai = 0; ai < N; ++ai) {
                x[b0 * P + c0 + ai * st] *= scale / (sgT + (w[ai] + w[b0] + w[c0]));
                if (off1 >= 0) x[off1 + ai * st] *= scale / (sgT + (w[ai] + w[b1] + w[c1]));
            }
            small_line2(b0 * P + c0, off1, st, N);
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int l = t; l < Lp; l += nt) {  // j
        const int l1 = l + Lp;
        small_line2((l / N) * N * P + l % N, l1 < L ? (l1 / N) * N * P + l1 % N : -1, P, N);
    }
    __syncthreads();
#pragma unroll 1
    for (int l = t; l < Lp; l += nt) small_line2(l * P, l + Lp < L ? (l + Lp) * P : -1, 1, N);  // k
    __syncthreads();
    if (r.out_dense)
        for (int row = warp; row < L; row += nw)
            for (int k = lane; k < N; k += 32) {
                const int p = row * N + k;
                float v = x[row * P + k];
                if (a.mask_out && !(a.labels[p] & (DPM_LBL_MPLUS | DPM_LBL_GEX))) v = 0.f;
                r.out_dense[p] = v;
            }
    if (r.out_trace) {
        const int e0 = a.rp_gin[0], e1 = a.rp_gin[L];
        for (int e = e0 + t; e < e1; e += nt) {
            const int p = a.gin[e];
            r.out_trace[e] = x[(p / N) * P + p % N];
        }
    }
}

__global__ void __launch_bounds__(kSmallThreads) k_small(PassArgs a, const ApRhs<float> *rhs, const float *tab) {
    small_body(a, rhs[blockIdx.x], tab);
}

__global__ void __launch_bounds__(kSmallThreads) kg_small(const GroupItem<float> *items) {
    const GroupItem<float> &g = items[blockIdx.x];
    if (!small_item<float>(g.a.N)) return;
    small_body(g.a, g.r, g.tab);
}

int small_configure() {
    static PerDeviceOnce once;
    return once.run([] {
        DPM_RET(raise_dynamic_smem_limit(reinterpret_cast<const void *>(k_small)));
        return raise_dynamic_smem_limit(reinterpret_cast<const void *>(kg_small));
    });
}

int small_launch(const PassArgs &a, const ApRhs<float> *rhs_dev, const float *tab, cudaStream_t s) {
    DPM_RET(small_configure());
    DPM_PROF("ap_simt32_small", s);
    k_small<<<a.B, kSmallThreads, small_smem(a.N), s>>>(a, rhs_dev, tab);
    DPM_LAUNCHED();
    return DPM_OK;
}

int small_group_launch(const GroupItem<float> *items, int B, cudaStream_t s) {
    DPM_RET(small_configure());
    DPM_PROF("ap_simt32_small", s);
    kg_small<<<B, kSmallThreads, small_smem(kSmallN), s>>>(items);
    DPM_LAUNCHED();
    return DPM_OK;
}

// tile regions, then two table chunks (16-byte aligned)
template <class T, int C = 32> size_t smem_rows(int N) {
    return (2 * (size_t)C * (N + 1) + 2 * chunk_elems<T>(N)) * sizeof(T);
}
template <class T, int C = 32> size_t smem_cols(int N) {
    return (2 * (size_t)N * C + ((N + 3) & ~3) + 2 * chunk_elems<T>(N)) * sizeof(T);
}

template <class T, int C = 32> int set_smem_limits(int) {
    static PerDeviceOnce once;
    return once.run([] {
        const int v = 227 * 1024;
        DPM_CUDA(cudaFuncSetAttribute(k_pass_k_fwd<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
        DPM_CUDA(cudaFuncSetAttribute(k_pass_j<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
        DPM_CUDA(cudaFuncSetAttribute(k_pass_i<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
        DPM_CUDA(cudaFuncSetAttribute(k_pass_k_inv<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
        return (int)DPM_OK;
    });
}

// Threads per CTA: one per task of the tile transform (4 output modes x 4 of the
// C columns), at most 512, so that every task of a tile runs in one sweep over the
// staged table.
template <int C> int tile_threads(int N) {
    const FoldDims fd(N);
    const int tasks = (fd.NEp / 4 + fd.NOp / 4) * (C / 4);
    const int q = C > 32 ? C : 32;  // a multiple of C: the column loops keep one column per thread
    return std::min(kThreads, std::max(q, (tasks + q - 1) / q * q));
}

template <class T, int C> bool tile_fits(int N) {
    return smem_rows<T, C>(N) <= 227 * 1024 && smem_cols<T, C>(N) <= 227 * 1024;
}

// The five passes with tile width C (columns or rows per CTA).
template <class T, int C>
int simt_passes(const PassArgs &a, const ApRhs<T> *rhs_dev, T *work, const T *tab, cudaStream_t s) {
    const int N = a.N;
    DPM_RET((set_smem_limits<T, C>(N)));
    const int64_t nrows = (int64_t)N * N;
    dim3 grow((unsigned)((nrows + C - 1) / C), a.B);
    dim3 gcol((unsigned)(N * ((N + C - 1) / C)), a.B);
    const bool f64 = sizeof(T) == 8;
    const int nt = tile_threads<C>(N);
    {
        DPM_PROF(f64 ? "ap_simt64_pass_k_fwd" : "ap_simt32_pass_k_fwd", s);
        k_pass_k_fwd<T, C><<<grow, nt, smem_rows<T, C>(N), s>>>(a, rhs_dev, work, tab);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF(f64 ? "ap_simt64_pass_j" : "ap_simt32_pass_j", s);
        k_pass_j<T, C><<<gcol, nt, smem_cols<T, C>(N), s>>>(a, rhs_dev, work, tab);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF(f64 ? "ap_simt64_pass_i" : "ap_simt32_pass_i", s);
        k_pass_i<T, C><<<gcol, nt, smem_cols<T, C>(N), s>>>(a, rhs_dev, work, tab);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF(f64 ? "ap_simt64_pass_j" : "ap_simt32_pass_j", s);
        k_pass_j<T, C><<<gcol, nt, smem_cols<T, C>(N), s>>>(a, rhs_dev, work, tab);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF(f64 ? "ap_simt64_pass_k_inv" : "ap_simt32_pass_k_inv", s);
        k_pass_k_inv<T, C><<<grow, nt, smem_rows<T, C>(N), s>>>(a, rhs_dev, work, tab);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

template <class T>
int simt_dispatch(int C, const PassArgs &a, const ApRhs<T> *rhs_dev, T *work, const T *tab, cudaStream_t s) {
    if (C == 16) return simt_passes<T, 16>(a, rhs_dev, work, tab, s);
    if (C == 64) return simt_passes<T, 64>(a, rhs_dev, work, tab, s);
    return simt_passes<T, 32>(a, rhs_dev, work, tab, s);
}

// ---- autotuner of the tile width ---------------------------------------------------
// The first solve of each (N, precision, batch class) on a device times the
// candidate widths on a workspace-only problem (every right-hand side zero, no
// outputs: the passes do the same work as for real data) and keeps the fastest.
// The per-output sums run in the same order for every width, so the choice
// changes the time, not the result.  DPM_SIMT_TILE=16|32|64 forces a width;
// DPM_AUTOTUNE=0 keeps 32.  A solve issued while its stream is being captured
// uses the tuned width if there is one, else 32.
struct TuneKey {
    int dev, N, f64, bclass;
    bool operator<(const TuneKey &o) const {
        return std::tie(dev, N, f64, bclass) < std::tie(o.dev, o.N, o.f64, o.bclass);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

int batch_class(int B) { return B <= 2 ? 0 : (B <= 16 ? 1 : 2); }

template <class T>
int tuned_tile(const PassArgs &a0, T *work, const T *tab, cudaStream_t s, int *out) {
    const char *force = getenv("DPM_SIMT_TILE");
    if (force) {
        const int c = atoi(force);
        if ((c == 16 || c == 32 || c == 64) &&
            (c == 16 ? tile_fits<T, 16>(a0.N) : c == 32 ? tile_fits<T, 32>(a0.N) : tile_fits<T, 64>(a0.N))) {
            *out = c;
            return DPM_OK;
        }
    }
    *out = 32;
    const char *en = getenv("DPM_AUTOTUNE");
    if (en && en[0] == '0') return DPM_OK;
    int dev = 0;
    DPM_CUDA(cudaGetDevice(&dev));
    const TuneKey key{dev, a0.N, (int)(sizeof(T) == 8), batch_class(a0.B)};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) { *out = it->second; return DPM_OK; }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return DPM_OK;
    // One tuning at a time: the zero descriptors below are shared.
    static std::mutex run_mu;
    static std::map<int, std::pair<void *, size_t>> zdesc;  // device -> (descriptors, bytes)
    std::lock_guard<std::mutex> run_lk(run_mu);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) { *out = it->second; return DPM_OK; }
    }
    auto &zb = zdesc[dev];
    const size_t need = sizeof(ApRhs<T>) * (size_t)a0.B;
    if (zb.second < need) {
        if (zb.first) DPM_CUDA(cudaFree(zb.first));
        zb.first = nullptr;
        zb.second = 0;
        DPM_CUDA(cudaMalloc(&zb.first, need));
        zb.second = need;
    }
    ApRhs<T> *zd = static_cast<ApRhs<T> *>(zb.first);
    DPM_CUDA(cudaMemsetAsync(zd, 0, need, s));
    PassArgs a = a0;
    a.cond_flag = nullptr;
    a.mask_f = a.mask_out = 0;
    cudaEvent_t e0, e1;
    DPM_CUDA(cudaEventCreate(&e0));
    DPM_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bestC = 32;
    const int cands[3] = {16, 32, 64};
    int rc = DPM_OK;
    for (int c : cands) {
        const bool fits = c == 16 ? tile_fits<T, 16>(a.N) : c == 32 ? tile_fits<T, 32>(a.N) : tile_fits<T, 64>(a.N);
        if (!fits) continue;
        rc = simt_dispatch<T>(c, a, zd, work, tab, s);  // warm-up
        if (rc == DPM_OK && cudaEventRecord(e0, s) != cudaSuccess) rc = DPM_ECUDA;
        for (int r = 0; r < 2 && rc == DPM_OK; ++r) rc = simt_dispatch<T>(c, a, zd, work, tab, s);
        if (rc == DPM_OK && cudaEventRecord(e1, s) != cudaSuccess) rc = DPM_ECUDA;
        if (rc == DPM_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = DPM_ECUDA;
        float ms = 0.f;
        if (rc == DPM_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = DPM_ECUDA;
        if (rc != DPM_OK) break;
        if (ms < best) { best = ms; bestC = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != DPM_OK) { set_error("SIMT tile tuning failed"); return rc; }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = bestC;
    }
    *out = bestC;
    return DPM_OK;
}

}  // namespace

void ap_params_from_index(ApParams &p, const GridIndex &gi) {
    p.labels = gi.labels.as<uint8_t>();
    p.shell = gi.shell.as<int>();
    p.shell_nb = gi.shell_nb.as<int>();
    p.rp_shell = gi.rp_shell.as<int>();
    p.gin = gi.gin.as<int>();
    p.rp_gin = gi.rp_gin.as<int>();
    p.n_shell = gi.n_shell;
}

template <class T>
int ap_solve_simt(const ApParams &p, const ApRhs<T> *rhs_dev, T *work, cudaStream_t s) {
    const int N = p.N;
    if (N < 2 || N > 256) { set_error("AP solve: N=%d outside [2, 256]", N); return DPM_EINVAL; }
    if (p.B < 1 || p.B > 65535) { set_error("AP solve: B=%d outside [1, 65535]", p.B); return DPM_EINVAL; }
    const T *tab = dst_fold_table<T>(N);
    if (!tab) { set_error("AP solve: could not create the DST table"); return DPM_ENOMEM; }
    PassArgs a{N, p.B, p.h, p.sigma, p.fscale, p.sigma_dev, p.fscale_dev, p.cond_flag, p.mask_f,
               p.mask_out, p.labels, p.shell, p.shell_nb, p.rp_shell, p.gin, p.rp_gin};
    if constexpr (sizeof(T) == 4) {
        if (small_item<T>(N)) return small_launch(a, rhs_dev, tab, s);  // one pass, no workspace
    }
    int C = 32;
    DPM_RET(tuned_tile<T>(a, work, tab, s, &C));
    return simt_dispatch<T>(C, a, rhs_dev, work, tab, s);
}

namespace {
// Tile width of a grouped launch, set by its largest grid: 32 while two
// 32-wide CTAs fit on an SM, else 16 (FP64 above N ~ 150).
template <class T> int group_width(int maxN) { return 2 * smem_cols<T, 32>(maxN) <= 227 * 1024 ? 32 : 16; }

template <class T, int C> int set_group_smem_limits() {
    static PerDeviceOnce once;
    return once.run([] {
        const int v = 227 * 1024;
        DPM_CUDA(cudaFuncSetAttribute(kg_pass_k_fwd<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
        DPM_CUDA(cudaFuncSetAttribute(kg_pass_j<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
        DPM_CUDA(cudaFuncSetAttribute(kg_pass_i<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
        DPM_CUDA(cudaFuncSetAttribute(kg_pass_k_inv<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
        return (int)DPM_OK;
    });
}

template <class T, int C>
int simt_group_passes(const GroupItem<T> *items, int B, int maxN, cudaStream_t s) {
    if (!tile_fits<T, C>(maxN)) { set_error("grouped AP solve: N=%d tiles exceed shared memory", maxN); return DPM_EINVAL; }
    DPM_RET((set_group_smem_limits<T, C>()));
    const bool f64 = sizeof(T) == 8;
    const dim3 grow((unsigned)row_tiles<C>(maxN), B), gcol((unsigned)col_tiles<C>(maxN), B);
    const size_t sr = smem_rows<T, C>(maxN), sc = smem_cols<T, C>(maxN);
    const int nt = tile_threads<C>(maxN);
    {
        DPM_PROF(f64 ? "ap_simt64_pass_k_fwd" : "ap_simt32_pass_k_fwd", s);
        kg_pass_k_fwd<T, C><<<grow, nt, sr, s>>>(items);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF(f64 ? "ap_simt64_pass_j" : "ap_simt32_pass_j", s);
        kg_pass_j<T, C><<<gcol, nt, sc, s>>>(items);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF(f64 ? "ap_simt64_pass_i" : "ap_simt32_pass_i", s);
        kg_pass_i<T, C><<<gcol, nt, sc, s>>>(items);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF(f64 ? "ap_simt64_pass_j" : "ap_simt32_pass_j", s);
        kg_pass_j<T, C><<<gcol, nt, sc, s>>>(items);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF(f64 ? "ap_simt64_pass_k_inv" : "ap_simt32_pass_k_inv", s);
        kg_pass_k_inv<T, C><<<grow, nt, sr, s>>>(items);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

}  // namespace

template <class T>
int ap_solve_simt_group(const std::vector<ApParams> &probs, const std::vector<ApRhs<T>> &rhs,
                        const std::vector<int> &prob_of, DevBuf &work, DevBuf &items_dev, cudaStream_t s) {
    const size_t B = rhs.size();
    if (B == 0) return DPM_OK;
    if (prob_of.size() != B) { set_error("grouped AP solve: one problem index per right-hand side"); return DPM_EINVAL; }
    int maxN = 0;
    for (const ApParams &p : probs) {
        if (p.N < 2 || p.N > 256) { set_error("grouped AP solve: N=%d outside [2, 256]", p.N); return DPM_EINVAL; }
        maxN = std::max(maxN, p.N);
    }
    std::vector<const T *> tabs(probs.size());
    for (size_t q = 0; q < probs.size(); ++q) {
        tabs[q] = dst_fold_table<T>(probs[q].N);
        if (!tabs[q]) { set_error("grouped AP solve: could not create the DST table"); return DPM_ENOMEM; }
    }
    // one launch set per chunk of right-hand sides whose cubes fit the workspace cap
    constexpr size_t kCap = size_t(8) << 30;
    std::vector<GroupItem<T>> items(B);
    size_t b0 = 0;
    while (b0 < B) {
        size_t bytes = 0, b1 = b0;
        while (b1 < B && b1 - b0 < 65535) {
            const int pi = prob_of[b1];
            if (pi < 0 || pi >= (int)probs.size()) { set_error("grouped AP solve: bad problem index"); return DPM_EINVAL; }
            const size_t cube = (size_t)probs[pi].N * probs[pi].N * probs[pi].N * sizeof(T);
            if (b1 > b0 && bytes + cube > kCap) break;
            bytes += cube;
            ++b1;
        }
        DPM_RET(work.reserve(bytes));
        DPM_RET(items_dev.reserve(sizeof(GroupItem<T>) * (b1 - b0)));
        size_t off = 0;
        for (size_t b = b0; b < b1; ++b) {
            const ApParams &p = probs[prob_of[b]];
            GroupItem<T> &g = items[b - b0];
            g.a = PassArgs{p.N, 1, p.h, p.sigma, p.fscale, p.sigma_dev, p.fscale_dev, p.cond_flag, p.mask_f,
                           p.mask_out, p.labels, p.shell, p.shell_nb, p.rp_shell, p.gin, p.rp_gin};
            g.r = rhs[b];
            g.cube = reinterpret_cast<T *>(static_cast<char *>(work.p) + off);
            g.tab = tabs[prob_of[b]];
            off += (size_t)p.N * p.N * p.N * sizeof(T);
        }
        // pageable source: staged before the call returns, so `items` may be reused
        DPM_CUDA(cudaMemcpyAsync(items_dev.p, items.data(), sizeof(GroupItem<T>) * (b1 - b0),
                                 cudaMemcpyHostToDevice, s));
        const auto *d = static_cast<const GroupItem<T> *>(items_dev.p);
        bool any_small = false, any_large = false;
        for (size_t b = b0; b < b1; ++b) {
            const bool sm = small_item<T>(probs[prob_of[b]].N);
            any_small |= sm;
            any_large |= !sm;
        }
        if constexpr (sizeof(T) == 4) {
            if (any_small) DPM_RET(small_group_launch(d, (int)(b1 - b0), s));
        }
        if (any_large && group_width<T>(maxN) == 16) DPM_RET((simt_group_passes<T, 16>(d, (int)(b1 - b0), maxN, s)));
        else if (any_large) DPM_RET((simt_group_passes<T, 32>(d, (int)(b1 - b0), maxN, s)));
        if (b1 < B) DPM_CUDA(cudaStreamSynchronize(s));  // the items / workspace are reused
        b0 = b1;
    }
    return DPM_OK;
}
template <class T>
size_t ap_group_bytes(const std::vector<ApParams> &probs, const std::vector<int> &prob_of) {
    size_t bytes = 0;
    for (int pi : prob_of)
        if (pi >= 0 && pi < (int)probs.size()) bytes += (size_t)probs[pi].N * probs[pi].N * probs[pi].N * sizeof(T);
    return bytes;
}

template <class T>
int ap_group_build(const std::vector<ApParams> &probs, const std::vector<ApRhs<T>> &rhs,
                   const std::vector<int> &prob_of, void *work, DevBuf &items_dev, int *maxN, int *minN,
                   cudaStream_t s) {
    const size_t B = rhs.size();
    *maxN = 0;
    *minN = 0;
    if (B == 0) return DPM_OK;
    if (prob_of.size() != B || B > 65535) {
        set_error("grouped AP solve: one problem index per right-hand side, at most 65535");
        return DPM_EINVAL;
    }
    std::vector<GroupItem<T>> items(B);
    size_t off = 0;
    for (size_t b = 0; b < B; ++b) {
        const int pi = prob_of[b];
        if (pi < 0 || pi >= (int)probs.size()) { set_error("grouped AP solve: bad problem index"); return DPM_EINVAL; }
        const ApParams &p = probs[pi];
        if (p.N < 2 || p.N > 256) { set_error("grouped AP solve: N=%d outside [2, 256]", p.N); return DPM_EINVAL; }
        const T *tab = dst_fold_table<T>(p.N);
        if (!tab) { set_error("grouped AP solve: could not create the DST table"); return DPM_ENOMEM; }
        GroupItem<T> &g = items[b];
        g.a = PassArgs{p.N, 1, p.h, p.sigma, p.fscale, p.sigma_dev, p.fscale_dev, p.cond_flag, p.mask_f,
                       p.mask_out, p.labels, p.shell, p.shell_nb, p.rp_shell, p.gin, p.rp_gin};
        g.r = rhs[b];
        g.cube = reinterpret_cast<T *>(static_cast<char *>(work) + off);
        g.tab = tab;
        off += (size_t)p.N * p.N * p.N * sizeof(T);
        *maxN = std::max(*maxN, p.N);
        *minN = b == 0 ? p.N : std::min(*minN, p.N);
    }
    DPM_RET(items_dev.reserve(sizeof(GroupItem<T>) * B));
    DPM_CUDA(cudaMemcpyAsync(items_dev.p, items.data(), sizeof(GroupItem<T>) * B, cudaMemcpyHostToDevice, s));
    DPM_CUDA(cudaStreamSynchronize(s));  // `items` goes out of scope
    return DPM_OK;
}

template <class T>
int ap_group_launch(const void *items_dev, int B, int maxN, int minN, cudaStream_t s) {
    if (B == 0) return DPM_OK;
    const auto *d = static_cast<const GroupItem<T> *>(items_dev);
    if constexpr (sizeof(T) == 4) {
        if (small_item<T>(minN)) DPM_RET(small_group_launch(d, B, s));
    }
    if (small_item<T>(maxN)) return DPM_OK;  // every grid solved in one pass
    if (group_width<T>(maxN) == 16) return simt_group_passes<T, 16>(d, B, maxN, s);
    return simt_group_passes<T, 32>(d, B, maxN, s);
}

#define DPM_GROUP_INST(T)                                                                                         \
    template size_t ap_group_bytes<T>(const std::vector<ApParams> &, const std::vector<int> &);                 \
    template int ap_group_build<T>(const std::vector<ApParams> &, const std::vector<ApRhs<T>> &,                \
                                   const std::vector<int> &, void *, DevBuf &, int *, int *, cudaStream_t);     \
    template int ap_group_launch<T>(const void *, int, int, int, cudaStream_t);
DPM_GROUP_INST(float)
DPM_GROUP_INST(double)
#undef DPM_GROUP_INST

template int ap_solve_simt_group<float>(const std::vector<ApParams> &, const std::vector<ApRhs<float>> &,
                                        const std::vector<int> &, DevBuf &, DevBuf &, cudaStream_t);
template int ap_solve_simt_group<double>(const std::vector<ApParams> &, const std::vector<ApRhs<double>> &,
                                         const std::vector<int> &, DevBuf &, DevBuf &, cudaStream_t);

int simt_tile_choice(int N, int f64, int B) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(TuneKey{dev, N, f64, batch_class(B)});
    return it == g_tuned.end() ? 0 : it->second;
}

template int ap_solve_simt<float>(const ApParams &, const ApRhs<float> *, float *, cudaStream_t);
template int ap_solve_simt<double>(const ApParams &, const ApRhs<double> *, double *, cudaStream_t);

}  // namespace dpm

// ===========================================================================
// Allocation-free variant of the batched FP32 auxiliary solve.
//
// Some callers cannot let a library allocate device memory: an application
// whose memory allocator owns every byte of the GPU (so a cudaMalloc behind
// its back would break its accounting or fail against its reservation), or a
// latency-critical loop where cudaMalloc/cudaFree -- which may synchronise the
// device and take an unbounded time -- are not acceptable.  For them,
// dpm_aux_solve_batched_noalloc runs the same five SIMT passes as the FP32
// path of dpm_aux_solve_batched, but every piece of scratch (the B*N^3
// workspace, the folded sine table and the right-hand-side descriptors) lives
// in one file-scope device array compiled into the library.  Nothing is
// allocated on any call.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call writes every byte it later reads (the table and the
// descriptors are rebuilt, the workspace is filled by the first pass), so
// nothing has to start at zero.  Calls that overlap on the GPU (e.g. issued
// to two streams without ordering) race on the array.
// ===========================================================================
namespace dpm {
namespace {

constexpr size_t kStaticWorkElems = size_t(16) << 20;     // 16 Mi floats = 64 MiB
constexpr size_t kStaticTableElems = 34816;               // >= folded table + weights for N <= 256
constexpr int kStaticMaxB = 1024;
constexpr size_t kStaticDescBytes = sizeof(ApRhs<float>) * kStaticMaxB;
constexpr size_t kStaticBytes =
    kStaticWorkElems * sizeof(float) + kStaticTableElems * sizeof(float) + kStaticDescBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {nullptr};

// Device address of g_static_scratch for the current device (looked up once
// per device with that device current).
int static_scratch_address(void **out) {
    int dev = 0;
    DPM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d beyond the %d devices this entry point tracks", dev, kMaxDevices);
        return DPM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            return DPM_ECUDA;
        }
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return DPM_OK;
}

// Folded sine table of dst_fold_table, generated on the device.
__global__ void k_static_table(int N, float *tab) {
    FoldDims fd(N);
    const size_t total = fd.total(N);
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        long long den = N + 1;
        if (idx < fd.offO()) {
            int mp = (int)(idx / fd.NEp), ap = (int)(idx % fd.NEp);
            if (ap < fd.NE) v = sin(M_PI * (double)(((long long)(2 * ap + 1) * (mp + 1)) % (2 * den)) / (double)den);
        } else if (idx < fd.offW()) {
            size_t r = idx - fd.offO();
            int mp = (int)(r / fd.NOp), ap = (int)(r % fd.NOp);
            if (ap < fd.NO) v = sin(M_PI * (double)(((long long)(2 * ap + 2) * (mp + 1)) % (2 * den)) / (double)den);
        } else {
            int n = (int)(idx - fd.offW());
            double sn = sin(M_PI * (double)(n + 1) / (2.0 * (double)den));
            v = sn * sn;
        }
        tab[idx] = (float)v;
    }
}

__global__ void k_static_desc(int B, size_t n3, const float *q, float *u, ApRhs<float> *d) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) d[b] = ApRhs<float>{q + (size_t)b * n3, nullptr, u + (size_t)b * n3, nullptr, 0, 0};
}

}  // namespace
}  // namespace dpm

extern "C" int dpm_aux_solve_batched_noalloc(int N, double h, double sigma, int B, const float *q,
                                             float *u, cudaStream_t s) {
    using namespace dpm;
    if (!q || !u) { set_error("q/u is NULL"); return DPM_EINVAL; }
    if (N < 2 || N > 256 || B < 1 || !(h > 0) || !(sigma >= 0)) {
        set_error("aux solve (no-alloc): need 2<=N<=256, B>=1, h>0, sigma>=0 (N=%d B=%d h=%g sigma=%g)",
                  N, B, h, sigma);
        return DPM_EINVAL;
    }
    const size_t n3 = (size_t)N * N * N;
    if (B > kStaticMaxB || (size_t)B * n3 > kStaticWorkElems) {
        set_error("aux solve (no-alloc): B*N^3 = %zu exceeds the static workspace of %zu floats "
                  "(and B <= %d); split the batch or use dpm_aux_solve_batched",
                  (size_t)B * n3, kStaticWorkElems, kStaticMaxB);
        return DPM_EINVAL;
    }
    if (FoldDims(N).total(N) > kStaticTableElems) { set_error("internal: table too large"); return DPM_EINVAL; }
    void *base = nullptr;
    DPM_RET(static_scratch_address(&base));
    float *work = static_cast<float *>(base);
    float *tab = work + kStaticWorkElems;
    ApRhs<float> *desc = reinterpret_cast<ApRhs<float> *>(tab + kStaticTableElems);
    k_static_table<<<64, 256, 0, s>>>(N, tab);
    DPM_LAUNCHED();
    k_static_desc<<<(B + 127) / 128, 128, 0, s>>>(B, n3, q, u, desc);
    DPM_LAUNCHED();
    PassArgs a{N, B, h, sigma, 1.0, nullptr, nullptr, nullptr, 0, 0,
               nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    return simt_passes<float, 32>(a, desc, work, tab, s);
}

extern "C" int dpm_simt_tile(int N, int precision, int B, int *tile) {
    using namespace dpm;
    if (!tile) { set_error("tile is NULL"); return DPM_EINVAL; }
    if (precision != DPM_PREC_FP32 && precision != DPM_PREC_FP64) {
        set_error("dpm_simt_tile: precision must be DPM_PREC_FP32 or DPM_PREC_FP64");
        return DPM_EINVAL;
    }
    *tile = simt_tile_choice(N, precision == DPM_PREC_FP64, B < 1 ? 1 : B);
    return DPM_OK;
}
