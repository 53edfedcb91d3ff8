// Tensor-core (tcgen05) auxiliary-problem solver for N = 128 (Definition 2.4).
//
// Same mathematics as the SIMT solver -- u = (2/(N+1))^3 S S S [(S S S q)/lambda]
// with S[a][m] = sin(pi a m/(N+1)) and the even/odd fold
// S[a][N+1-m] = (-1)^(a+1) S[a][m] -- arranged as three passes over HBM:
//
//   plane pass (per x-plane i): fold+contract along k, then along j;
//   pencil pass (per j-mode b): along i forward, times (2/(N+1))^3/lambda,
//                               along i inverse;
//   inverse plane pass: along k, then j; restriction to N^+ / trace on gamma_in.
//
// Each 1D transform of 128 points is the fold (64 sums, 64 differences) and two
// 128 x 64 x 64 contractions with the folded sine blocks SE[a'][m'] =
// S[2a'+1][m'+1] (sums) and SO[a'][m'] = S[2a'+2][m'+1] (differences), issued
// as tcgen05.mma kind::f16 with FP32 accumulation in TMEM.  FP32 accuracy comes
// from a 3-term split: every operand v (scaled by a power of two into
// [2^13, 2^14)) is hi = f16(v), lo = f16(v - hi), and the product is
// hi*hi' + hi*lo' + lo*hi' (the dropped lo*lo' is ~2^-22 relative).  Sine
// blocks are pre-split on the host, scaled by 2^12.
//
// CTA = 128 threads (4 warps = the 128 TMEM lanes), 2 CTAs per SM, persistent
// over work items.  Every wait on the MMA-completion mbarrier is bounded; on
// expiry the kernel records an error in g_tc_status and stops.
#include <algorithm>
#include <map>
#include <math.h>
#include <mutex>
#include <utility>
#include <vector>

#include "dpm_internal.cuh"
#include "tc_ptx.cuh"

namespace dpm {

namespace {

constexpr int kN = 128;             // grid points per axis handled by these kernels
constexpr int kH = 64;              // fold length
constexpr int kThreads = 128;
constexpr uint32_t kTmemCols = 128; // D_E in columns [0,64), D_O in [64,128)
constexpr float kSScale = 4096.f;   // sine blocks are stored times 2^12
constexpr uint32_t kWaitIters = 1u << 26;

// shared-memory layout (offsets from a 1024-aligned base)
constexpr int kATile = kN * 128;                   // 128 rows x 64 f16 = 16 KB
constexpr int kBTile = kH * 128;                   // 64 rows x 64 f16 = 8 KB
constexpr int kOffA = 0;                           // E_hi, E_lo, O_hi, O_lo
constexpr int kOffB = 4 * kATile;                  // SE_hi, SE_lo, SO_hi, SO_lo
constexpr int kOffScale = kOffB + 4 * kBTile;      // float sE[128], sO[128]
constexpr int kOffW = kOffScale + 2 * kN * 4;      // float weights[128]
constexpr int kOffRed = kOffW + kN * 4;            // float red[8]
constexpr int kOffBar = kOffRed + 64;              // mbarrier
constexpr int kOffTmem = kOffBar + 16;             // TMEM base address
constexpr int kSmemUsed = kOffTmem + 16;
constexpr int kSmemBytes = kSmemUsed + 1024;       // slack for 1024-byte alignment

__device__ int g_tc_status;  // 0 ok; 1 = an MMA wait expired

struct TcArgs {
    int B;
    double h, sigma, fscale;
    int mask_f, mask_out;
    const uint8_t *labels;
    const int *shell, *shell_nb, *rp_shell, *gin, *rp_gin;
    const uint4 *bops;   // 32 KB pre-split, pre-swizzled sine blocks
    const float *s2;     // sin^2(pi (n+1)/(2(N+1))), n < 128
};

__device__ __forceinline__ float pow2_scale(float m, float *inv) {
    // s = 2^(14 - e) with m = f 2^e, f in [0.5, 1): m*s in [2^13, 2^14)
    if (!(m > 0.f) || !isfinite(m)) { *inv = 1.f; return 1.f; }
    int e;
    frexpf(m, &e);
    if (e < -100) e = -100;
    *inv = ldexpf(1.f, e - 14);
    return ldexpf(1.f, 14 - e);
}

__device__ __forceinline__ void split2(float v, __half &hi, __half &lo) {
    hi = __float2half_rn(v);
    lo = __float2half_rn(v - __half2float(hi));
}

struct Smem {
    unsigned char *base;
    __device__ unsigned char *A(int t) const { return base + kOffA + t * kATile; }
    __device__ unsigned char *Bt(int t) const { return base + kOffB + t * kBTile; }
    __device__ float *sE() const { return reinterpret_cast<float *>(base + kOffScale); }
    __device__ float *sO() const { return reinterpret_cast<float *>(base + kOffScale) + kN; }
    __device__ float *w() const { return reinterpret_cast<float *>(base + kOffW); }
    __device__ float *red() const { return reinterpret_cast<float *>(base + kOffRed); }
    __device__ uint64_t *bar() const { return reinterpret_cast<uint64_t *>(base + kOffBar); }
    __device__ uint32_t *tslot() const { return reinterpret_cast<uint32_t *>(base + kOffTmem); }
};

__device__ __forceinline__ Smem smem_base() {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    uint32_t a = tc::smem_u32(sm_raw);
    return Smem{sm_raw + ((1024u - (a & 1023u)) & 1023u)};
}

// Prologue shared by the kernels: sine blocks into smem, mbarrier, TMEM.
__device__ void tc_prologue(const Smem &S, const TcArgs &a) {
    const int t = threadIdx.x;
    uint4 *dst = reinterpret_cast<uint4 *>(S.Bt(0));
    for (int i = t; i < 4 * kBTile / 16; i += kThreads) dst[i] = a.bops[i];
    if (t == 0) {
        tc::mbar_init(S.bar(), 1);
        tc::fence_mbar_init();
    }
    if ((t >> 5) == 0) {
        tc::tmem_alloc(S.tslot(), kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
}

__device__ void tc_epilogue(const Smem &S) {
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(*S.tslot(), kTmemCols);
}

// One folded 128-point transform: D[:,0:64) = E * SE^T, D[:,64:128) = O * SO^T,
// each as hi*hi + hi*lo + lo*hi (issued by one thread), then commit.
__device__ __forceinline__ void issue_transform(const Smem &S, uint32_t tm) {
    const uint32_t id = tc::idesc_f16_f32(kN, kH);
    const uint32_t a0 = tc::smem_u32(S.A(0)), b0 = tc::smem_u32(S.Bt(0));
#pragma unroll
    for (int part = 0; part < 2; ++part) {  // 0: sums (E), 1: differences (O)
        const uint32_t ahi = a0 + (2 * part) * kATile, alo = ahi + kATile;
        const uint32_t bhi = b0 + (2 * part) * kBTile, blo = bhi + kBTile;
        const uint32_t d = tm + part * kH;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            tc::mma_f16(d, tc::sdesc_k128(ahi + kk * 32), tc::sdesc_k128(bhi + kk * 32), id, kk > 0);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            tc::mma_f16(d, tc::sdesc_k128(ahi + kk * 32), tc::sdesc_k128(blo + kk * 32), id, 1);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            tc::mma_f16(d, tc::sdesc_k128(alo + kk * 32), tc::sdesc_k128(bhi + kk * 32), id, 1);
    }
    tc::mma_commit(S.bar());
}

// Operands written -> MMA issued -> completion observed by every thread.
__device__ __forceinline__ bool run_transform(const Smem &S, uint32_t tm, uint32_t &phase) {
    tc::fence_async_smem();
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    if (threadIdx.x == 0) issue_transform(S, tm);
    bool ok = tc::mbar_wait(S.bar(), phase, kWaitIters);
    phase ^= 1u;
    tc::tc_fence_after_sync();
    if (!ok) atomicExch(&g_tc_status, 1);
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// Store 4 consecutive K values (hi and lo) of row `row` starting at K = k0
// (k0 % 4 == 0) into the pair of tiles (hi, lo).
__device__ __forceinline__ void put4(unsigned char *thi, unsigned char *tlo, int row, int k0,
                                     const float *v, float s) {
    __half h[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) split2(v[u] * s, h[u], l[u]);
    uint32_t off = tc::sw128_chunk(row, k0 >> 3) + (k0 & 7) * 2;
    uint2 ph, pl;
    ph.x = (uint32_t)__half_as_ushort(h[0]) | ((uint32_t)__half_as_ushort(h[1]) << 16);
    ph.y = (uint32_t)__half_as_ushort(h[2]) | ((uint32_t)__half_as_ushort(h[3]) << 16);
    pl.x = (uint32_t)__half_as_ushort(l[0]) | ((uint32_t)__half_as_ushort(l[1]) << 16);
    pl.y = (uint32_t)__half_as_ushort(l[2]) | ((uint32_t)__half_as_ushort(l[3]) << 16);
    *reinterpret_cast<uint2 *>(thi + off) = ph;
    *reinterpret_cast<uint2 *>(tlo + off) = pl;
}

// Store 8 consecutive K values of row `row` starting at K = k0 (k0 % 8 == 0).
__device__ __forceinline__ void put8(unsigned char *thi, unsigned char *tlo, int row, int k0,
                                     const float *v, float s) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        __half h0, l0, h1, l1;
        split2(v[2 * u] * s, h0, l0);
        split2(v[2 * u + 1] * s, h1, l1);
        hw[u] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
        lw[u] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
    }
    uint32_t off = tc::sw128_chunk(row, k0 >> 3);
    *reinterpret_cast<uint4 *>(thi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4 *>(tlo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

__device__ __forceinline__ float half_max(float v) {  // max over a 16-lane half of the warp
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------------------
// Plane pass.  INV = false: q built from f / the gamma density, forward k then
// j, result Z[i][b][c] back to the workspace.  INV = true: reads Z, inverse
// along c -> k then b -> j, writes u (masked) and/or the gamma_in trace.
// ---------------------------------------------------------------------------
template <bool INV>
__global__ void __launch_bounds__(kThreads, 2)
k_tc_plane(TcArgs a, const ApRhs<float> *rhs, float *work) {
    const Smem S = smem_base();
    tc_prologue(S, a);
    const uint32_t tm = *S.tslot();
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    uint32_t phase = 0;
    const int nitems = a.B * kN;
    const float fs = (float)a.fscale;
    const float cdiag = (float)(a.sigma + 6.0 / (a.h * a.h)), coff = (float)(1.0 / (a.h * a.h));
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int b = item / kN, i = item % kN;
        const ApRhs<float> r = rhs[b];
        float *wplane = work + ((size_t)b * kN + i) * kN * kN;
        // ---- phase A: rows of the plane -> folded, split operands ----------
        // The difference-potential part of q lives on the sparse M^- shell:
        // stage it as an fp32 plane in the operand region first.
        const bool has_dens = !INV && r.dens != nullptr;
        float *stage = reinterpret_cast<float *>(S.A(0));  // 128 x 128 fp32 = 64 KB
        if (has_dens) {
            float4 *st4 = reinterpret_cast<float4 *>(stage);
            for (int q = t; q < kN * kN / 4; q += kThreads) st4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            __syncthreads();
            const int e0 = a.rp_shell[(int64_t)i * kN], e1 = a.rp_shell[(int64_t)(i + 1) * kN];
            for (int e = e0 + t; e < e1; e += kThreads) {
                const int pnode = a.shell[e];
                const int* nb = a.shell_nb + 8 * (size_t)e;
                float sacc = 0.f;
#pragma unroll
                for (int q = 1; q < 7; ++q)
                    if (nb[q] >= 0) sacc += r.dens[nb[q]];
                const float self = nb[0] >= 0 ? r.dens[nb[0]] : 0.f;
                stage[pnode - i * kN * kN] = cdiag * self - coff * sacc;
            }
            __syncthreads();
        }
        // all 32 rows of this warp in flight at once (lane owns k = 4 lane .. 4 lane + 3)
        float x[32][4];
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) {
            const int row = warp * 32 + rr;
            if (INV) {
                const float4 v = *reinterpret_cast<const float4 *>(wplane + row * kN + 4 * lane);
                x[rr][0] = v.x; x[rr][1] = v.y; x[rr][2] = v.z; x[rr][3] = v.w;
            } else {
                x[rr][0] = x[rr][1] = x[rr][2] = x[rr][3] = 0.f;
                const int64_t p0 = ((int64_t)i * kN + row) * kN + 4 * lane;
                if (r.f) {
                    const float4 v = *reinterpret_cast<const float4 *>(r.f + p0);
                    x[rr][0] = fs * v.x; x[rr][1] = fs * v.y; x[rr][2] = fs * v.z; x[rr][3] = fs * v.w;
                    if (a.mask_f) {
                        const uint32_t lb = *reinterpret_cast<const uint32_t *>(a.labels + p0);
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (!((lb >> (8 * u)) & DPM_LBL_MPLUS)) x[rr][u] = 0.f;
                    }
                }
                if (has_dens) {
                    const float4 v = *reinterpret_cast<const float4 *>(stage + row * kN + 4 * lane);
                    x[rr][0] += v.x; x[rr][1] += v.y; x[rr][2] += v.z; x[rr][3] += v.w;
                }
            }
        }
        if (has_dens) __syncthreads();  // staged plane fully read before operands overwrite it
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) {
            const int row = warp * 32 + rr;
            float y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) y[u] = __shfl_xor_sync(0xffffffffu, x[rr][u], 31);
            float v[4];
            if (lane < 16) {
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = x[rr][u] + y[3 - u];     // m' = 4 lane + u
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = y[u] - x[rr][3 - u];     // m' = 4 (31-lane) + u
            }
            float m = fmaxf(fmaxf(fabsf(v[0]), fabsf(v[1])), fmaxf(fabsf(v[2]), fabsf(v[3])));
            m = half_max(m);
            float inv;
            const float sc = pow2_scale(m, &inv);
            const int L = row < kH ? 2 * row : 2 * (kN - 1 - row) + 1;
            if (lane < 16) {
                put4(S.A(0), S.A(1), L, 4 * lane, v, sc);
                if (lane == 0) S.sE()[L] = inv;
            } else {
                put4(S.A(2), S.A(3), L, 4 * (31 - lane), v, sc);
                if (lane == 16) S.sO()[L] = inv;
            }
        }
        if (!run_transform(S, tm, phase)) break;
        // ---- phase C: D1 (row L = plane row r(L)) -> fold over rows -> A2 ---
        const int L = t;
        const uint32_t lane_addr = tm + ((uint32_t)(warp * 32) << 16);
        const float iE = S.sE()[L] * (1.f / kSScale), iO = S.sO()[L] * (1.f / kSScale);
        // tile maximum of the folded values
        float mx = 0.f;
#pragma unroll
        for (int c0 = 0; c0 < 2 * kH; c0 += 16) {
            float d[16];
            tc::tmem_ld16(lane_addr + c0, d);
            tc::tmem_wait_ld();
            const float sc = c0 < kH ? iE : iO;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const float own = d[u] * sc;
                const float par = __shfl_xor_sync(0xffffffffu, own, 1);
                const float f2 = (L & 1) ? (par - own) : (own + par);
                mx = fmaxf(mx, fabsf(f2));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) S.red()[warp] = mx;
        __syncthreads();
        mx = fmaxf(fmaxf(S.red()[0], S.red()[1]), fmaxf(S.red()[2], S.red()[3]));
        float inv2;
        const float s2 = pow2_scale(mx, &inv2);
        {
            const int p = L >> 1;
            unsigned char *thi = S.A((L & 1) ? 2 : 0), *tlo = S.A((L & 1) ? 3 : 1);
            const uint32_t koff = (uint32_t)(p & 7) * 2;
#pragma unroll
            for (int c0 = 0; c0 < 2 * kH; c0 += 16) {
                float d[16];
                tc::tmem_ld16(lane_addr + c0, d);
                tc::tmem_wait_ld();
                const float sc = c0 < kH ? iE : iO;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const float own = d[u] * sc;
                    const float par = __shfl_xor_sync(0xffffffffu, own, 1);
                    const float f2 = ((L & 1) ? (par - own) : (own + par)) * s2;
                    // output index of the first transform: c = 2(c0+u) (sums), 2(c0+u-64)+1 (diffs)
                    const int c = c0 < kH ? 2 * (c0 + u) : 2 * (c0 + u - kH) + 1;
                    __half hi, lo;
                    split2(f2, hi, lo);
                    const uint32_t off = tc::sw128_chunk(c, p >> 3) + koff;
                    *reinterpret_cast<__half *>(thi + off) = hi;
                    *reinterpret_cast<__half *>(tlo + off) = lo;
                }
            }
        }
        if (!run_transform(S, tm, phase)) break;
        // ---- phase E: D2 (row = c, columns = second-transform output) --------
        const float iout = inv2 * (1.f / kSScale);
        if (!INV) {
            // Z[i][bmode][c], bmode = 2 col (sums) or 2 col + 1 (diffs)
#pragma unroll
            for (int c0 = 0; c0 < 2 * kH; c0 += 16) {
                float d[16];
                tc::tmem_ld16(lane_addr + c0, d);
                tc::tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int bm = c0 < kH ? 2 * (c0 + u) : 2 * (c0 + u - kH) + 1;
                    wplane[bm * kN + t] = d[u] * iout;
                }
            }
        } else {
            // u[i][j][k]: thread = k, column -> j
            float *stage = reinterpret_cast<float *>(S.A(0));  // 128 x 128 fp32 = 64 KB
            const int64_t pbase = (int64_t)i * kN * kN;
#pragma unroll
            for (int c0 = 0; c0 < 2 * kH; c0 += 16) {
                float d[16];
                tc::tmem_ld16(lane_addr + c0, d);
                tc::tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int j = c0 < kH ? 2 * (c0 + u) : 2 * (c0 + u - kH) + 1;
                    float val = d[u] * iout;
                    if (r.out_dense) {
                        const int64_t p = pbase + (int64_t)j * kN + t;
                        float o = val;
                        if (a.mask_out && !(a.labels[p] & (DPM_LBL_MPLUS | DPM_LBL_GEX))) o = 0.f;
                        r.out_dense[p] = o;
                    }
                    if (r.out_trace) stage[j * kN + t] = val;
                }
            }
            if (r.out_trace) {
                __syncthreads();
                const int e0 = a.rp_gin[(int64_t)i * kN], e1 = a.rp_gin[(int64_t)(i + 1) * kN];
                for (int e = e0 + t; e < e1; e += kThreads) {
                    const int p = a.gin[e];
                    const int j = (p / kN) % kN, k = p % kN;
                    r.out_trace[e] = stage[j * kN + k];
                }
            }
        }
        // everyone is done with TMEM and the operand/staging smem of this item
        tc::tc_fence_before_sync();
        __syncthreads();
        tc::tc_fence_after_sync();
    }
    tc_epilogue(S);
}

// ---------------------------------------------------------------------------
// Pencil pass along i for a fixed j-mode jb: forward, scale/lambda, inverse.
// Thread t = c (the contiguous index), A rows = c, K = fold index over i / a.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 2)
k_tc_pencil(TcArgs a, const ApRhs<float> *rhs, float *work) {
    const Smem S = smem_base();
    tc_prologue(S, a);
    const uint32_t tm = *S.tslot();
    const int t = threadIdx.x, warp = t >> 5;
    uint32_t phase = 0;
    const float w4 = (float)(4.0 / (a.h * a.h));
    for (int n = t; n < kN; n += kThreads) S.w()[n] = w4 * a.s2[n];
    __syncthreads();
    const float sig = (float)a.sigma;
    const double sc = 2.0 / (kN + 1);
    const float nscale = (float)(sc * sc * sc);
    const int nitems = a.B * kN;
    const size_t sN2 = (size_t)kN * kN;
    const uint32_t lane_addr = tm + ((uint32_t)(warp * 32) << 16);
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int b = item / kN, jb = item % kN;
        (void)rhs;
        float *base = work + (size_t)b * kN * sN2 + (size_t)jb * kN + t;
        // ---- phase A: fold along i, split, per-row (per-c) scale -----------
        float e[kH], o[kH];
#pragma unroll
        for (int mp = 0; mp < kH; ++mp) {
            const float x1 = base[(size_t)mp * sN2], x2 = base[(size_t)(kN - 1 - mp) * sN2];
            e[mp] = x1 + x2;
            o[mp] = x1 - x2;
        }
        float me = 0.f, mo = 0.f;
#pragma unroll
        for (int mp = 0; mp < kH; ++mp) {
            me = fmaxf(me, fabsf(e[mp]));
            mo = fmaxf(mo, fabsf(o[mp]));
        }
        float ie, io;
        const float se = pow2_scale(me, &ie), so = pow2_scale(mo, &io);
#pragma unroll
        for (int k0 = 0; k0 < kH; k0 += 8) {
            put8(S.A(0), S.A(1), t, k0, e + k0, se);
            put8(S.A(2), S.A(3), t, k0, o + k0, so);
        }
        if (!run_transform(S, tm, phase)) break;
        // ---- phase C: z[a] = D / lambda, fold over a, split -------------------
        float z[kN];  // z[a], a = 0..127 (a = 2a' from sums, 2a'+1 from differences)
#pragma unroll
        for (int c0 = 0; c0 < 2 * kH; c0 += 16) {
            float d[16];
            tc::tmem_ld16(lane_addr + c0, d);
            tc::tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int am = c0 < kH ? 2 * (c0 + u) : 2 * (c0 + u - kH) + 1;
                z[am] = d[u] * ((c0 < kH ? ie : io) * (1.f / kSScale));
            }
        }
        const float wjc = S.w()[jb] + S.w()[t] + sig;
#pragma unroll
        for (int am = 0; am < kN; ++am) z[am] *= __fdividef(nscale, wjc + S.w()[am]);
#pragma unroll
        for (int mp = 0; mp < kH; ++mp) {
            const float lo_ = z[mp], hi_ = z[kN - 1 - mp];
            e[mp] = lo_ + hi_;
            o[mp] = lo_ - hi_;
        }
        me = 0.f;
        mo = 0.f;
#pragma unroll
        for (int mp = 0; mp < kH; ++mp) {
            me = fmaxf(me, fabsf(e[mp]));
            mo = fmaxf(mo, fabsf(o[mp]));
        }
        const float se2 = pow2_scale(me, &ie), so2 = pow2_scale(mo, &io);
#pragma unroll
        for (int k0 = 0; k0 < kH; k0 += 8) {
            put8(S.A(0), S.A(1), t, k0, e + k0, se2);
            put8(S.A(2), S.A(3), t, k0, o + k0, so2);
        }
        if (!run_transform(S, tm, phase)) break;
        // ---- phase E: D3[c][i'] -> Z[i][jb][c] ---------------------------------
#pragma unroll
        for (int c0 = 0; c0 < 2 * kH; c0 += 16) {
            float d[16];
            tc::tmem_ld16(lane_addr + c0, d);
            tc::tmem_wait_ld();
            const float sc2 = (c0 < kH ? ie : io) * (1.f / kSScale);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int ii = c0 < kH ? 2 * (c0 + u) : 2 * (c0 + u - kH) + 1;
                base[(size_t)ii * sN2] = d[u] * sc2;
            }
        }
        tc::tc_fence_before_sync();
        __syncthreads();
        tc::tc_fence_after_sync();
    }
    tc_epilogue(S);
}

// Host: pre-split, pre-swizzled sine blocks (per device), 4 tiles of 64 x 64 f16.
const uint4 *tc_sine_blocks() {
    static std::mutex mu;
    static std::map<int, void *> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return static_cast<const uint4 *>(it->second);
    std::vector<unsigned char> img(4 * kBTile, 0);
    auto put = [&](int tile, int row, int k, __half v) {
        size_t off = (size_t)tile * kBTile + (row >> 3) * 1024 + (row & 7) * 128 +
                     (((k >> 3) ^ (row & 7)) << 4) + (k & 7) * 2;
        *reinterpret_cast<__half *>(&img[off]) = v;
    };
    for (int part = 0; part < 2; ++part)
        for (int ap = 0; ap < kH; ++ap)
            for (int mp = 0; mp < kH; ++mp) {
                long long num = (long long)(2 * ap + 1 + part) * (mp + 1) % (2 * (kN + 1));
                double v = sin(M_PI * (double)num / (double)(kN + 1)) * (double)kSScale;
                __half hi = __double2half(v);
                __half lo = __float2half((float)(v - (double)__half2float(hi)));
                put(2 * part, ap, mp, hi);
                put(2 * part + 1, ap, mp, lo);
            }
    void *d = nullptr;
    if (cudaMalloc(&d, img.size()) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    cache[dev] = d;
    return static_cast<const uint4 *>(d);
}

int tc_configure() {
    static bool done = false;
    if (done) return DPM_OK;
    DPM_CUDA(cudaFuncSetAttribute(k_tc_plane<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    DPM_CUDA(cudaFuncSetAttribute(k_tc_plane<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    DPM_CUDA(cudaFuncSetAttribute(k_tc_pencil, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    done = true;
    return DPM_OK;
}

}  // namespace

bool tc_supported(int N) { return N == kN; }

int tc_status_check() {
    int st = 0;
    DPM_CUDA(cudaMemcpyFromSymbol(&st, g_tc_status, sizeof(int)));
    if (st) {
        int z = 0;
        cudaMemcpyToSymbol(g_tc_status, &z, sizeof(int));
        set_error("a tensor-core MMA wait expired (bounded wait)");
        return DPM_ETIMEOUT;
    }
    return DPM_OK;
}

int ap_solve_tc(const ApParams &p, const ApRhs<float> *rhs_dev, float *work, cudaStream_t s) {
    if (!tc_supported(p.N)) {
        set_error("tensor-core AP solve supports N = %d only (got %d)", kN, p.N);
        return DPM_EUNSUPPORTED;
    }
    if (p.sigma_dev || p.fscale_dev || p.cond_flag) {
        set_error("tensor-core AP solve takes sigma/fscale by value");
        return DPM_EINVAL;
    }
    DPM_RET(tc_configure());
    const uint4 *bops = tc_sine_blocks();
    const float *tab = dst_fold_table<float>(kN);
    if (!bops || !tab) { set_error("tensor-core AP solve: table allocation failed"); return DPM_ENOMEM; }
    int dev = 0, sms = 0;
    DPM_CUDA(cudaGetDevice(&dev));
    DPM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // offset of the sin^2 weights inside the fold table (see dst_simt.cu)
    const int H = kN / 2, NEp = (H + 3) & ~3;
    const size_t offW = (size_t)H * NEp + (size_t)H * NEp;
    TcArgs a{p.B, p.h, p.sigma, p.fscale, p.mask_f, p.mask_out, p.labels, p.shell, p.shell_nb,
             p.rp_shell, p.gin, p.rp_gin, bops, tab + offW};
    const int nitems = p.B * kN;
    const int grid = std::min(nitems, 2 * sms);
    {
        DPM_PROF("tc_plane_fwd", s);
        k_tc_plane<false><<<grid, kThreads, kSmemBytes, s>>>(a, rhs_dev, work);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF("tc_pencil", s);
        k_tc_pencil<<<grid, kThreads, kSmemBytes, s>>>(a, rhs_dev, work);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF("tc_plane_inv", s);
        k_tc_plane<true><<<grid, kThreads, kSmemBytes, s>>>(a, rhs_dev, work);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

}  // namespace dpm
