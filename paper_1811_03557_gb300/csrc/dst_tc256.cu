// Tensor-core (tcgen05) auxiliary-problem solver for N = 256 (Definition 2.4).
//
// The same mathematics as the N = 128 solver -- u = (2/(N+1))^3 S S S [(S S S q)
// / lambda] with the even/odd fold S[a][N+1-m] = (-1)^(a+1) S[a][m] -- but a
// 256 x 256 FP32 plane (256 KB) does not fit in shared memory, so every axis
// is its own pass over HBM, out of place between two workspace halves X and Y:
//
//   assemble q (f on M^+ times fscale, plus L[v_gamma] on the shell) -> X
//   k forward X -> Y;  j forward Y -> X;  i forward, times (2/(N+1))^3/lambda, X -> Y
//   i inverse Y -> X;  j inverse X -> Y;  k inverse Y -> the outputs (restriction
//   to N^+ and/or the trace on gamma_in, written from the pass's staged rows)
//
// A 256-point transform folds to 128 sums (odd 1-based modes) and 128
// differences (even modes); each is a 128 x 128 x 128 contraction with the
// folded sine block of its parity.  One CTA computes one parity for a tile of
// 128 lines (the A operand: 128 lines x 128 fold indices, 64 KB as hi/lo f16;
// the B operand: that parity's sine block, 64 KB, resident for the CTA's
// lifetime), so the CTAs of even and odd index split the two parities of the
// same tiles and read the same input lines at about the same time (the second
// read hits L2).  FP32 accuracy from the 3-term split hi*hi + hi*lo + lo*hi with
// one power-of-two scale per A row (line), undone per TMEM lane.
//
//   k pass (contiguous axis): lines are rows; loads by half-warps (float4 from
//     both ends of the row); the 128 x 128 result goes through shared memory
//     (XOR-swizzled) to rows of the output, each parity writing every second
//     element.
//   j / i passes (strided axes): lines are columns; thread c owns the line at
//     the contiguous index c, so loads and stores are coalesced across c.
//
// 256 threads, one CTA per SM (~130 KB shared memory), persistent over tiles.
// Every wait on an mbarrier is bounded; on expiry the kernel records an error
// in g_tc256_status and stops.
#include <algorithm>
#include <map>
#include <math.h>
#include <mutex>
#include <vector>

#include "dpm_internal.cuh"
#include "tc_ptx.cuh"

namespace dpm {

namespace {

constexpr int kN = 256;             // grid points per axis handled here
constexpr int kH = 128;             // fold length = modes per parity
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 128;
constexpr float kSScale = 4096.f;   // sine blocks are stored times 2^12
constexpr uint32_t kWaitIters = 1u << 26;
constexpr int kTile = 128 * 128;    // bytes: 128 rows x 64 f16 (one K half), 128-byte swizzle
constexpr int kOffA = 0;            // A tiles [hi/lo][K half]
constexpr int kOffB = 4 * kTile;    // B tiles [hi/lo][K half] of the CTA's parity
constexpr int kOffX = 8 * kTile;    // float[2][128]: row maxima (j/i) or inverse scales (k)
constexpr int kOffW = kOffX + 2 * kH * 4;  // float[256] lambda weights (4/h^2) sin^2
constexpr int kOffBar = kOffW + kN * 4;    // mbarrier
constexpr int kOffTmem = kOffBar + 16;     // TMEM base address
constexpr int kSmemUsed = kOffTmem + 16;
constexpr int kSmemBytes = kSmemUsed + 1024;  // slack for 1024-byte alignment

__device__ int g_tc256_status;  // 0 ok; 1 = an MMA wait expired

struct Sm {
    unsigned char *base;
    __device__ unsigned char *A(int t) const { return base + kOffA + t * kTile; }
    __device__ unsigned char *Bt(int t) const { return base + kOffB + t * kTile; }
    __device__ float *x() const { return reinterpret_cast<float *>(base + kOffX); }
    __device__ float *w() const { return reinterpret_cast<float *>(base + kOffW); }
    __device__ uint64_t *bar() const { return reinterpret_cast<uint64_t *>(base + kOffBar); }
    __device__ uint32_t *tslot() const { return reinterpret_cast<uint32_t *>(base + kOffTmem); }
};

__device__ __forceinline__ Sm sm_base() {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    const uint32_t a = tc::smem_u32(sm_raw);
    return Sm{sm_raw + ((1024u - (a & 1023u)) & 1023u)};
}

struct LineArgs {
    int B;
    int lam;  // strided passes: times (2/(N+1))^3 / lambda before the store
    double h, sigma;
    const double *sigma_dev;
    const float *in;
    float *out;
    const uint4 *bops;  // [parity][hi/lo][K half] tiles, pre-split and pre-swizzled
    const float *s2;    // sin^2(pi (n+1)/(2(N+1))), n < 256
    // last k pass: write each right-hand side's result (dense, masked to N^+
    // when asked, and/or its trace on gamma_in) instead of `out`
    int final_out, mask_out;
    const ApRhs<float> *rhs;
    const uint8_t *labels;
    const int *rp_gin, *gin;
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

__device__ __forceinline__ void split_pack(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// 4 consecutive K values of A row `row` at K = k0 (k0 % 4 == 0) within one K half.
__device__ __forceinline__ void put4(unsigned char *thi, unsigned char *tlo, int row, int k0,
                                     const float *v, float s) {
    uint2 ph, pl;
    split_pack(v[0] * s, v[1] * s, ph.x, pl.x);
    split_pack(v[2] * s, v[3] * s, ph.y, pl.y);
    const uint32_t off = tc::sw128_chunk(row, k0 >> 3) + (k0 & 7) * 2;
    *reinterpret_cast<uint2 *>(thi + off) = ph;
    *reinterpret_cast<uint2 *>(tlo + off) = pl;
}

// 8 consecutive K values of A row `row` at K = k0 (k0 % 8 == 0) within one K half.
__device__ __forceinline__ void put8(unsigned char *thi, unsigned char *tlo, int row, int k0,
                                     const float *v, float s) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) split_pack(v[2 * u] * s, v[2 * u + 1] * s, hw[u], lw[u]);
    const uint32_t off = tc::sw128_chunk(row, k0 >> 3);
    *reinterpret_cast<uint4 *>(thi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4 *>(tlo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

__device__ __forceinline__ float half_max(float v) {  // max over a 16-lane half of the warp
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// D[128 x 128] = A (128 x 128) * B^T as hi*lo + lo*hi + hi*hi, 8 K steps of 16.
// The small cross terms go first: every accumulation step of the tensor core
// rounds the running sum toward zero, so the terms added while D is still small
// cost nothing, and only the 8 steps of the main term shrink the full-size sum
// (24 steps at full size left u about 5e-6 too small at N = 256).
__device__ __forceinline__ void issue_part(const Sm &S, uint32_t tm) {
    const uint32_t id = tc::idesc_f16_f32(128, kH, false);
    const uint32_t a0 = tc::smem_u32(S.A(0)), b0 = tc::smem_u32(S.Bt(0));
    auto desc = [](uint32_t base, int lohi, int kk) {
        return tc::sdesc_k128(base + (2 * lohi + (kk >> 2)) * kTile + (kk & 3) * 32);
    };
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) tc::mma_f16(tm, desc(a0, 0, kk), desc(b0, 1, kk), id, kk > 0);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) tc::mma_f16(tm, desc(a0, 1, kk), desc(b0, 0, kk), id, 1);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) tc::mma_f16(tm, desc(a0, 0, kk), desc(b0, 0, kk), id, 1);
    tc::mma_commit(S.bar());
}

__device__ __forceinline__ bool run_part(const Sm &S, uint32_t tm, uint32_t &phase) {
    tc::fence_async_smem();
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    if (threadIdx.x == 0) issue_part(S, tm);
    const bool ok = tc::mbar_wait(S.bar(), phase, kWaitIters);
    phase ^= 1u;
    tc::tc_fence_after_sync();
    if (!ok) atomicExch(&g_tc256_status, 1);
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// Prologue: the CTA's parity blocks and the lambda weights into shared memory,
// the mbarrier, 128 TMEM columns.
__device__ void prologue(const Sm &S, const LineArgs &a, int parity) {
    const int t = threadIdx.x;
    const uint4 *src = a.bops + (size_t)parity * (4 * kTile / 16);
    uint4 *dst = reinterpret_cast<uint4 *>(S.Bt(0));
    for (int i = t; i < 4 * kTile / 16; i += kThreads) dst[i] = src[i];
    const float w4 = (float)(4.0 / (a.h * a.h));
    for (int n = t; n < kN; n += kThreads) S.w()[n] = w4 * a.s2[n];
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

__device__ void epilogue(const Sm &S) {
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(*S.tslot(), kTmemCols);
}

// ---------------------------------------------------------------------------
// k pass: tiles of 128 rows (j = 128 jb + r) of plane i; CTA parity = blockIdx.x & 1.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1) k256_rows(LineArgs a) {
    const Sm S = sm_base();
    const int parity = blockIdx.x & 1;
    prologue(S, a, parity);
    const uint32_t tm = *S.tslot();
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int hw = t >> 4, lp = t & 15;
    const int L = 32 * (warp & 3) + lane, hc = warp >> 2;
    const uint32_t lane_addr = tm + ((uint32_t)(32 * (warp & 3)) << 16);
    float *rowinv = S.x();
    uint32_t phase = 0;
    const int per = gridDim.x >> 1;
    const int nitems = a.B * kN * 2;
    const size_t n3 = (size_t)kN * kN * kN;
    for (int it = blockIdx.x >> 1; it < nitems; it += per) {
        const int b = it / (2 * kN), rem = it % (2 * kN);
        const int i = rem >> 1, jb = rem & 1;
        const size_t tile0 = (size_t)b * n3 + ((size_t)i * kN + 128 * jb) * kN;
        // ---- A: half-warp hw folds rows 8 hw .. 8 hw + 7 ------------------------------
#pragma unroll 2
        for (int q = 0; q < 8; ++q) {
            const int r = 8 * hw + q;
            const float4 *row = reinterpret_cast<const float4 *>(a.in + tile0 + (size_t)r * kN);
            float v[2][4];
            float rm = 0.f;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const float4 f = row[16 * s + lp], g = row[63 - 16 * s - lp];
                const float fx[4] = {f.x, f.y, f.z, f.w}, gx[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    v[s][u] = parity ? fx[u] - gx[3 - u] : fx[u] + gx[3 - u];
                    rm = fmaxf(rm, fmaxf(fabsf(fx[u]), fabsf(gx[u])));
                }
            }
            rm = half_max(rm);
            float rinv;
            const float sr = pow2_scale(2.f * rm, &rinv);
#pragma unroll
            for (int s = 0; s < 2; ++s) put4(S.A(s), S.A(2 + s), r, 4 * lp, v[s], sr);
            if (lp == 0) rowinv[r] = rinv;
        }
        if (!run_part(S, tm, phase)) break;
        // ---- D (row L, modes 2a' + parity) -> shared memory, XOR-swizzled -----------
        float *stage = reinterpret_cast<float *>(S.A(0));
        const float iD = rowinv[L] * (1.f / kSScale);
#pragma unroll
        for (int c0 = 64 * hc; c0 < 64 * hc + 64; c0 += 32) {
            float d0[16], d1[16];
            tc::tmem_ld16(lane_addr + c0, d0);
            tc::tmem_ld16(lane_addr + c0 + 16, d1);
            tc::tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int a0 = c0 + u, a1 = c0 + 16 + u;
                stage[L * 128 + ((a0 & ~31) | ((a0 ^ L) & 31))] = d0[u] * iD;
                stage[L * 128 + ((a1 & ~31) | ((a1 ^ L) & 31))] = d1[u] * iD;
            }
        }
        __syncthreads();
        // ---- rows of the output: warp w writes rows w, w + 8, ... ------------------
        if (!a.final_out) {
            for (int r = warp; r < 128; r += kThreads / 32) {
                float *orow = a.out + tile0 + (size_t)r * kN;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int ap = 32 * q + lane;
                    orow[2 * ap + parity] = stage[r * 128 + 32 * q + ((lane ^ r) & 31)];
                }
            }
        } else {
            // the solve's result: this CTA's parity of every row, masked to N^+,
            // and the gamma_in nodes of the tile whose k has this parity (the
            // tile's rows are consecutive, so its nodes are one run of the
            // sorted gamma_in list, taken in parallel)
            const ApRhs<float> rb = a.rhs[b];
            const uint8_t keep = DPM_LBL_MPLUS | DPM_LBL_GEX;
            const int row0 = i * kN + 128 * jb;  // grid row (i, j) of the tile's first line
            if (rb.out_dense) {
                for (int r = warp; r < 128; r += kThreads / 32) {
                    const size_t prow = (size_t)(row0 + r) * kN;  // linear index of node (i, j, 0)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ap = 32 * q + lane, k = 2 * ap + parity;
                        float v = stage[r * 128 + 32 * q + ((lane ^ r) & 31)];
                        if (a.mask_out && !(a.labels[prow + k] & keep)) v = 0.f;
                        rb.out_dense[prow + k] = v;
                    }
                }
            }
            if (rb.out_trace && a.rp_gin) {
                const int e0 = a.rp_gin[row0], e1 = a.rp_gin[row0 + 128];
                for (int e = e0 + t; e < e1; e += kThreads) {
                    const int rel = a.gin[e] - row0 * kN;  // r * 256 + k
                    const int r = rel >> 8, k = rel & (kN - 1);
                    if ((k & 1) != parity) continue;
                    const int ap = k >> 1;
                    rb.out_trace[e] = stage[r * 128 + ((ap & ~31) | ((ap ^ r) & 31))];
                }
            }
        }
        tc::tc_fence_before_sync();
        __syncthreads();
        tc::tc_fence_after_sync();
    }
    epilogue(S);
}

// ---------------------------------------------------------------------------
// j pass (stride N, outer = i) and i pass (stride N^2, outer = j): tiles of 128
// columns c = 128 cb + t mod 128; thread half h = t / 128 folds m' in [64h, 64h+64).
// ---------------------------------------------------------------------------
template <int AXIS>  // 1: j, 2: i
__global__ void __launch_bounds__(kThreads, 1) k256_cols(LineArgs a) {
    const Sm S = sm_base();
    const int parity = blockIdx.x & 1;
    prologue(S, a, parity);
    const uint32_t tm = *S.tslot();
    const int t = threadIdx.x, warp = t >> 5;
    const int c = t & 127, h = t >> 7;
    const uint32_t lane_addr = tm + ((uint32_t)(32 * (warp & 3)) << 16);
    float *xmax = S.x();
    uint32_t phase = 0;
    const int per = gridDim.x >> 1;
    const int nitems = a.B * kN * 2;
    const size_t n3 = (size_t)kN * kN * kN;
    const size_t stride = AXIS == 1 ? (size_t)kN : (size_t)kN * kN;
    // (2/(N+1))^3, times 1 + the expected relative loss of the solve to the tensor
    // cores' round-toward-zero accumulation (tc_rz_bias: kH/16 = 8 main-term steps per
    // transform, 6 transforms, 1.16e-6; measured means -1.1e-6 to -1.55e-6 on
    // dense random and Gaussian data), so that long time loops do not drift
    const double sc = 2.0 / (kN + 1);
    const float nscale = (float)(sc * sc * sc * (1.0 + tc_rz_bias(kH / 16)));
    const float sig = (float)(a.sigma_dev ? *a.sigma_dev : a.sigma);
    for (int it = blockIdx.x >> 1; it < nitems; it += per) {
        const int b = it / (2 * kN), rem = it % (2 * kN);
        const int outer = rem >> 1, cb = rem & 1;
        const int cg = 128 * cb + c;  // contiguous index (k)
        const size_t base = (size_t)b * n3 + (AXIS == 1 ? (size_t)outer * kN * kN : (size_t)outer * kN) + cg;
        // ---- A: fold along the strided axis -----------------------------------------
        float v[64];
        float rm = 0.f;
#pragma unroll
        for (int q = 0; q < 64; ++q) {
            const int mp = 64 * h + q;
            const float x1 = a.in[base + (size_t)mp * stride];
            const float x2 = a.in[base + (size_t)(kN - 1 - mp) * stride];
            v[q] = parity ? x1 - x2 : x1 + x2;
            rm = fmaxf(rm, fmaxf(fabsf(x1), fabsf(x2)));
        }
        xmax[h * 128 + c] = rm;
        __syncthreads();
        rm = fmaxf(xmax[c], xmax[128 + c]);
        float rinv;
        const float sr = pow2_scale(2.f * rm, &rinv);
#pragma unroll
        for (int k0 = 0; k0 < 64; k0 += 8) put8(S.A(h), S.A(2 + h), c, k0, v + k0, sr);
        if (!run_part(S, tm, phase)) break;
        // ---- D (row c, modes 2a' + parity), columns [64h, 64h + 64) -> out ----------
        const float iD = rinv * (1.f / kSScale);
        const float wjk = S.w()[outer] + S.w()[cg] + sig;
#pragma unroll
        for (int c0 = 64 * h; c0 < 64 * h + 64; c0 += 32) {
            float d0[16], d1[16];
            tc::tmem_ld16(lane_addr + c0, d0);
            tc::tmem_ld16(lane_addr + c0 + 16, d1);
            tc::tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int am = 2 * (c0 + u) + parity;  // mode along the transformed axis
                float val = (u < 16 ? d0[u] : d1[u - 16]) * iD;
                if (a.lam) val *= __fdividef(nscale, wjk + S.w()[am]);
                a.out[base + (size_t)am * stride] = val;
            }
        }
        tc::tc_fence_before_sync();
        __syncthreads();
        tc::tc_fence_after_sync();
    }
    epilogue(S);
}

// ---------------------------------------------------------------------------
// Right-hand side and output (plain memory-bound kernels)
// ---------------------------------------------------------------------------
// X[b] = fscale f (on M^+ when masked), or 0 without f.
__global__ void k256_q(const ApRhs<float> *rhs, int mask_f, double fscale, const double *fscale_dev,
                       const uint8_t *lab, float *X) {
    const int b = blockIdx.y;
    const ApRhs<float> r = rhs[b];
    const float fs = (float)(fscale_dev ? *fscale_dev : fscale);
    const size_t n4 = (size_t)kN * kN * kN / 4;
    float4 *x = reinterpret_cast<float4 *>(X + (size_t)b * kN * kN * kN);
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n4; q += (size_t)gridDim.x * blockDim.x) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r.f) {
            v = reinterpret_cast<const float4 *>(r.f)[q];
            v.x *= fs; v.y *= fs; v.z *= fs; v.w *= fs;
            if (mask_f) {
                const uint32_t lb = reinterpret_cast<const uint32_t *>(lab)[q];
                if (!(lb & DPM_LBL_MPLUS)) v.x = 0.f;
                if (!((lb >> 8) & DPM_LBL_MPLUS)) v.y = 0.f;
                if (!((lb >> 16) & DPM_LBL_MPLUS)) v.z = 0.f;
                if (!((lb >> 24) & DPM_LBL_MPLUS)) v.w = 0.f;
            }
        }
        x[q] = v;
    }
}

// X[b] += L[v_gamma] on the shell: (sigma + 6/h^2) v(self) - (1/h^2) sum of v over
// the 6 neighbours, for every right-hand side with a density.
__global__ void k256_shell(int n_shell, double c6, float coff, double sigma, const double *sigma_dev,
                           const ApRhs<float> *rhs, const int *shell, const int *shell_nb, float *X) {
    __shared__ float cd;
    if (threadIdx.x == 0) cd = (float)((sigma_dev ? *sigma_dev : sigma) + c6);
    __syncthreads();
    const int b = blockIdx.y;
    const ApRhs<float> r = rhs[b];
    if (!r.dens) return;
    float *x = X + (size_t)b * kN * kN * kN;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_shell; e += gridDim.x * blockDim.x) {
        const int *nb = shell_nb + 8 * (size_t)e;
        float sacc = 0.f;
#pragma unroll
        for (int q = 1; q < 7; ++q)
            if (nb[q] >= 0) sacc += r.dens[nb[q]];
        const float self = nb[0] >= 0 ? r.dens[nb[0]] : 0.f;
        x[shell[e]] += cd * self - coff * sacc;
    }
}

// Host: pre-split, pre-swizzled folded sine blocks, [parity][hi/lo][K half] x 16 KB.
const uint4 *tc256_sine_blocks() {
    static std::mutex mu;
    static std::map<int, void *> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return static_cast<const uint4 *>(it->second);
    std::vector<unsigned char> img((size_t)2 * 4 * kTile, 0);
    auto put = [&](int parity, int lohi, int row, int k, __half v) {
        const int kh = k >> 6, kk = k & 63;
        const size_t off = (size_t)(parity * 4 + 2 * lohi + kh) * kTile + (row >> 3) * 1024 +
                           (row & 7) * 128 + (((kk >> 3) ^ (row & 7)) << 4) + (kk & 7) * 2;
        *reinterpret_cast<__half *>(&img[off]) = v;
    };
    for (int parity = 0; parity < 2; ++parity)
        for (int ap = 0; ap < kH; ++ap)
            for (int mp = 0; mp < kH; ++mp) {
                const long long num = (long long)(2 * ap + 1 + parity) * (mp + 1) % (2 * (kN + 1));
                const double v = sin(M_PI * (double)num / (double)(kN + 1)) * (double)kSScale;
                const __half hi = __double2half(v);
                const __half lo = __float2half((float)(v - (double)__half2float(hi)));
                put(parity, 0, ap, mp, hi);
                put(parity, 1, ap, mp, lo);
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

int configure256() {
    static PerDeviceOnce once;
    return once.run([] {
        DPM_CUDA(cudaFuncSetAttribute(k256_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        DPM_CUDA(cudaFuncSetAttribute(k256_cols<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        DPM_CUDA(cudaFuncSetAttribute(k256_cols<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        return (int)DPM_OK;
    });
}

}  // namespace

int tc256_status_check() {
    int st = 0;
    DPM_CUDA(cudaMemcpyFromSymbol(&st, g_tc256_status, sizeof(int)));
    if (st) {
        int z = 0;
        cudaMemcpyToSymbol(g_tc256_status, &z, sizeof(int));
        set_error("a tensor-core MMA wait expired (bounded wait, N = 256)");
        return DPM_ETIMEOUT;
    }
    return DPM_OK;
}

// work: 2 * B * N^3 floats (X then Y).
int ap_solve_tc256(const ApParams &p, const ApRhs<float> *rhs_dev, float *work, cudaStream_t s) {
    if (p.N != kN) { set_error("ap_solve_tc256: N = %d", p.N); return DPM_EINVAL; }
    DPM_RET(configure256());
    const uint4 *bops = tc256_sine_blocks();
    const float *tab = dst_fold_table<float>(kN);
    if (!bops || !tab) { set_error("tensor-core AP solve: table allocation failed"); return DPM_ENOMEM; }
    int dev = 0, sms = 0;
    DPM_CUDA(cudaGetDevice(&dev));
    DPM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int H = kN / 2, NEp = (H + 3) & ~3;
    const float *s2 = tab + (size_t)H * NEp + (size_t)H * NEp;  // weights after the two fold tables
    const size_t n3 = (size_t)kN * kN * kN;
    float *X = work, *Y = work + (size_t)p.B * n3;
    const int grid = std::max(2, (sms / 2) * 2);
    const dim3 ge(4 * sms, p.B);
    {
        DPM_PROF("tc256_rhs", s);
        k256_q<<<ge, 256, 0, s>>>(rhs_dev, p.mask_f, p.fscale, p.fscale_dev, p.labels, X);
        DPM_LAUNCHED();
        if (p.n_shell > 0 && p.shell_nb) {
            const dim3 gs((unsigned)std::min<int64_t>((p.n_shell + 255) / 256, 256), p.B);
            k256_shell<<<gs, 256, 0, s>>>((int)p.n_shell, 6.0 / (p.h * p.h), (float)(1.0 / (p.h * p.h)),
                                          p.sigma, p.sigma_dev, rhs_dev, p.shell, p.shell_nb, X);
            DPM_LAUNCHED();
        }
    }
    LineArgs a{p.B, 0, p.h, p.sigma, p.sigma_dev, nullptr, nullptr, bops, s2,
               0, p.mask_out, rhs_dev, p.labels, p.rp_gin, p.gin};
    auto rows = [&](const float *in, float *out, int final_out) -> int {
        a.in = in, a.out = out, a.lam = 0, a.final_out = final_out;
        DPM_PROF(final_out ? "tc256_k_out" : "tc256_k", s);
        k256_rows<<<grid, kThreads, kSmemBytes, s>>>(a);
        DPM_LAUNCHED();
        return DPM_OK;
    };
    auto cols = [&](int axis, int lam, const float *in, float *out) -> int {
        a.in = in, a.out = out, a.lam = lam;
        DPM_PROF(axis == 1 ? "tc256_j" : "tc256_i", s);
        if (axis == 1) k256_cols<1><<<grid, kThreads, kSmemBytes, s>>>(a);
        else k256_cols<2><<<grid, kThreads, kSmemBytes, s>>>(a);
        DPM_LAUNCHED();
        return DPM_OK;
    };
    DPM_RET(rows(X, Y, 0));
    DPM_RET(cols(1, 0, Y, X));
    DPM_RET(cols(2, 1, X, Y));
    DPM_RET(cols(2, 0, Y, X));
    DPM_RET(cols(1, 0, X, Y));
    DPM_RET(rows(Y, nullptr, 1));  // k inverse straight into the outputs
    return DPM_OK;
}

}  // namespace dpm
