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
// Plane passes: 256 threads (8 warps; warps w and w+4 share the TMEM lanes
// 32(w%4).. and split the columns) at 128 registers; pencil: 128 threads (one
// column per thread).  Two CTAs per SM, persistent over work items; each item's
// input is staged by TMA into the operand tiles while the previous item writes
// its output.  Every wait on the MMA-completion mbarrier is bounded; on
// expiry the kernel records an error in g_tc_status and stops.
#include <cuda.h>

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
constexpr uint32_t kTmemCols = 128; // D_E in columns [0,64), D_O in [64,128)
constexpr float kSScale = 4096.f;   // sine blocks are stored times 2^12
constexpr uint32_t kWaitIters = 1u << 26;
constexpr double kRzBias = tc_rz_bias(kH / 16);  // see the pencil pass's spectral scale

// shared-memory layout (offsets from a 1024-aligned base)
constexpr int kATile = kN * 128;                   // 128 rows x 64 f16 = 16 KB
constexpr int kBTile = kH * 128;                   // 64 rows x 64 f16 = 8 KB
constexpr int kOffA = 0;                           // E_hi, E_lo, O_hi, O_lo
constexpr int kOffB = 4 * kATile;                  // SE_hi, SE_lo, SO_hi, SO_lo
constexpr int kOffScale = kOffB + 4 * kBTile;      // float sE[128], sO[128]
constexpr int kOffW = kOffScale + 2 * kN * 4;      // float weights[128]
constexpr int kOffXch = kOffW + kN * 4;            // float xch[4][128] (pencil row maxima)
constexpr int kOffRed = kOffXch + 4 * kN * 4;      // float red[16]
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
    const float *qsh;    // staged L[v] on the shell, [B][n_shell]
    int64_t n_shell;
    const double *sigma_dev, *fscale_dev;  // override sigma / fscale when set
};

__device__ __forceinline__ float pow2_scale(float m, float *inv) {
    // s = 2^(14 - e) with m = f 2^e, f in [0.5, 1): m*s in [2^13, 2^14); e is
    // read from the exponent field (a normal m has e = biased exponent - 126),
    // clamped below at -100 (which also covers subnormal m), and both powers of
    // two are assembled as exponent fields.  m = 0, inf or NaN: s = 1.
    const uint32_t be = __float_as_uint(m) >> 23;  // m >= 0: no sign bit
    const int e = max((int)be - 126, -100);
    const bool ok = m > 0.f && be < 255u;
    *inv = ok ? __uint_as_float((uint32_t)(113 + e) << 23) : 1.f;
    return ok ? __uint_as_float((uint32_t)(141 - e) << 23) : 1.f;
}

// hi/lo split of two values at once, packed as f16x2 (first value in the low half).
__device__ __forceinline__ void split_pack(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

struct Smem {
    unsigned char *base;
    __device__ unsigned char *A(int t) const { return base + kOffA + t * kATile; }
    __device__ unsigned char *Bt(int t) const { return base + kOffB + t * kBTile; }
    __device__ float *sE() const { return reinterpret_cast<float *>(base + kOffScale); }
    __device__ float *w() const { return reinterpret_cast<float *>(base + kOffW); }
    __device__ float *xch() const { return reinterpret_cast<float *>(base + kOffXch); }
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
    for (int i = t; i < 4 * kBTile / 16; i += (int)blockDim.x) dst[i] = a.bops[i];
    if (t == 0) {
        tc::mbar_init(S.bar(), 1);      // MMA completion
        tc::mbar_init(S.bar() + 1, 1);  // input bulk copies
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
// each as hi*lo + lo*hi + hi*hi (issued by one thread), then commit.  The A
// tiles are K-major (rows of 64 K) or, with MN = true, MN-major (atoms of
// 64 rows x 8 K placed at (kgroup * 2 + matom) * 1024 B).
template <bool MN>
__device__ __forceinline__ void issue_transform(const Smem &S, uint32_t tm) {
    const uint32_t id = tc::idesc_f16_f32(kN, kH, MN);
    const uint32_t a0 = tc::smem_u32(S.A(0)), b0 = tc::smem_u32(S.Bt(0));
#pragma unroll
    for (int part = 0; part < 2; ++part) {  // 0: sums (E), 1: differences (O)
        const uint32_t ahi = a0 + (2 * part) * kATile, alo = ahi + kATile;
        const uint32_t bhi = b0 + (2 * part) * kBTile, blo = bhi + kBTile;
        const uint32_t d = tm + part * kH;
        auto ad = [](uint32_t base, int kk) {
            return MN ? tc::sdesc_mn128(base + kk * 4096, 1024, 2048) : tc::sdesc_k128(base + kk * 32);
        };
        // cross terms first: each accumulation step rounds the running sum toward
        // zero, so only the main term's 4 steps act on the full-size sum (12 such
        // steps left u about 2e-6 too small)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            tc::mma_f16(d, ad(ahi, kk), tc::sdesc_k128(blo + kk * 32), id, kk > 0);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            tc::mma_f16(d, ad(alo, kk), tc::sdesc_k128(bhi + kk * 32), id, 1);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            tc::mma_f16(d, ad(ahi, kk), tc::sdesc_k128(bhi + kk * 32), id, 1);
    }
    tc::mma_commit(S.bar());
}

// Byte offset of element (m, k) in an MN-major 128-row tile (see issue_transform).
__device__ __forceinline__ uint32_t mn_off(int m, int k) {
    const int row = k & 7;
    return (uint32_t)((((k >> 3) * 2 + (m >> 6)) << 10) + row * 128 + ((((m & 63) >> 3) ^ row) << 4) +
                      (m & 7) * 2);
}

struct NoWork {
    __device__ void operator()() const {}
};

// Operands written -> MMA issued -> completion observed by every thread.
// `during` runs on every thread while the MMAs execute (it must not touch the
// operand tiles or TMEM).
template <bool MN = false, class F = NoWork>
__device__ __forceinline__ bool run_transform(const Smem &S, uint32_t tm, uint32_t &phase,
                                              F during = F()) {
    tc::fence_async_smem();
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    if (threadIdx.x == 0) issue_transform<MN>(S, tm);
    during();
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
    uint2 ph, pl;
    split_pack(v[0] * s, v[1] * s, ph.x, pl.x);
    split_pack(v[2] * s, v[3] * s, ph.y, pl.y);
    const uint32_t off = tc::sw128_chunk(row, k0 >> 3) + (k0 & 7) * 2;
    *reinterpret_cast<uint2 *>(thi + off) = ph;
    *reinterpret_cast<uint2 *>(tlo + off) = pl;
}

// Store 8 consecutive K values of row `row` starting at K = k0 (k0 % 8 == 0).
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

// ---------------------------------------------------------------------------
// Plane pass.  256 threads (warps w and w+4 share TMEM lanes 32(w%4)..+31 and
// split the columns), two CTAs per SM,
// persistent over items (rhs b, plane i).  The FP32 input plane (64 KB) is
// staged in the operand region itself: it is read into registers before the
// first operand tiles are written, and the bulk copy (TMA) of the next item's
// plane is issued as soon as this item's second MMA has completed, so it
// streams in during this item's output phase.  The other CTA on the SM runs
// its MMAs and memory waits while this one computes, and the reverse.
// INV = false: q = fscale f (on M^+ when masked) + L[v_gamma] on the shell
//   (staged values from k_shell_rhs), forward along k then j, Z[i][b][c] out.
// INV = true: reads Z, along c -> k then b -> j, writes u (masked to N^+)
//   and/or the trace on gamma_in.
// Operand scaling: the first transform's A rows (grid lines) get one
// power-of-two scale each; the second transform's operand gets one scale from
// the bound |A2| <= 256 max|x| (a 64-term fold of |x| <= max|x| with |S| <= 1,
// then a sum of two rows), which keeps every f16 value below 2^14 without a
// reduction over the tile.
// ---------------------------------------------------------------------------
constexpr int kPlaneThreads = 256;
constexpr int kRawBytes = kN * kN * 4;                   // one fp32 plane = the four A tiles
static_assert(kRawBytes == 4 * kATile, "the input plane is staged in the operand tiles");

// q on the shell for every right-hand side that has a density:
// qsh[b][e] = (sigma + 6/h^2) v(self) - (1/h^2) sum of v over the 6 neighbours.
__global__ void k_shell_rhs(int n_shell, double c6, float coff, double sigma,
                            const double *sigma_dev, const ApRhs<float> *rhs, const int *shell_nb,
                            float *qsh) {
    // cdiag = sigma + 6/h^2 in FP64, rounded once (FP64 work kept out of the per-thread path)
    __shared__ float cd;
    if (threadIdx.x == 0) cd = (float)((sigma_dev ? *sigma_dev : sigma) + c6);
    __syncthreads();
    const float cdiag = cd;
    const int b = blockIdx.y;
    const ApRhs<float> r = rhs[b];
    if (!r.dens) return;
    if (r.pre) {  // the density's shell pairs are precomputed: a streaming pass
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_shell; e += gridDim.x * blockDim.x) {
            const float2 v = r.pre[e];
            qsh[(size_t)b * n_shell + e] = cdiag * v.x - coff * v.y;
        }
        return;
    }
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_shell; e += gridDim.x * blockDim.x) {
        const int *nb = shell_nb + 8 * (size_t)e;
        float sacc = 0.f;
#pragma unroll
        for (int q = 1; q < 7; ++q)
            if (nb[q] >= 0) sacc += r.dens[nb[q]];
        const float self = nb[0] >= 0 ? r.dens[nb[0]] : 0.f;
        qsh[(size_t)b * n_shell + e] = cdiag * self - coff * sacc;
    }
}

// pre[c][e] = {v_c(self), sum of v_c over the 6 neighbours} on the shell: the
// sigma-independent parts of q for densities that stay fixed between solves
// (the same neighbour order and FP32 sum as k_shell_rhs)
__global__ void k_shell_pre(int n_shell, const int *shell_nb, const float *dens, int64_t ng, float2 *pre) {
    const int c = blockIdx.y;
    const float *d = dens + (size_t)c * ng;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_shell; e += gridDim.x * blockDim.x) {
        const int *nb = shell_nb + 8 * (size_t)e;
        float sacc = 0.f;
#pragma unroll
        for (int q = 1; q < 7; ++q)
            if (nb[q] >= 0) sacc += d[nb[q]];
        const float self = nb[0] >= 0 ? d[nb[0]] : 0.f;
        pre[(size_t)c * n_shell + e] = make_float2(self, sacc);
    }
}

template <bool INV>
__device__ __forceinline__ const float *plane_src(const ApRhs<float> &r, const float *work, int b,
                                                  int i) {
    if (INV) return work + ((size_t)b * kN + i) * kN * kN;
    return r.f ? r.f + (size_t)i * kN * kN : nullptr;
}

template <bool INV>
__global__ void __launch_bounds__(kPlaneThreads, 2)
k_tc_plane(TcArgs a, const ApRhs<float> *rhs, float *work) {
    const Smem S = smem_base();
    tc_prologue(S, a);
    float *raw = reinterpret_cast<float *>(S.A(0));
    uint64_t *bar_ld = S.bar() + 1;
    float *rowinv = S.sE();  // inverse scale of each A row of the first transform
    float *wmax = S.red();   // max |x| per warp
    const uint32_t tm = *S.tslot();
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int q4 = warp & 3, hc = warp >> 2;  // TMEM lane quarter, column half
    const int L = 32 * q4 + lane;             // TMEM lane = row of D owned by this thread
    const uint32_t lane_addr = tm + ((uint32_t)(32 * q4) << 16);
    uint32_t phase = 0, ld_phase = 0;
    const int nitems = a.B * kN;
    const float fs = (float)(a.fscale_dev ? *a.fscale_dev : a.fscale);
    // An item whose plane needs no transform: forward without f and without shell
    // nodes in plane i (the transform of zero is zero: the output plane is zeroed),
    // inverse without dense output and without gamma_in nodes in plane i.
    auto skippable = [&](int it) -> bool {
        const ApRhs<float> &rr = rhs[it / kN];
        const int ii = it % kN;
        if (!INV) {
            if (rr.f) return false;
            if (!rr.dens) return true;
            return a.rp_shell[(int64_t)ii * kN] == a.rp_shell[(int64_t)(ii + 1) * kN];
        }
        if (rr.out_dense) return false;
        if (!rr.out_trace) return true;
        return a.rp_gin[(int64_t)ii * kN] == a.rp_gin[(int64_t)(ii + 1) * kN];
    };
    int item = blockIdx.x;
    bool inflight = false;  // a bulk copy into raw completes on bar_ld
    if (item < nitems && !skippable(item)) {
        const float *src = plane_src<INV>(rhs[item / kN], work, item / kN, item % kN);
        if (src) {
            if (t == 0) {
                tc::mbar_arrive_expect_tx(bar_ld, kRawBytes);
                tc::bulk_g2s(raw, src, kRawBytes, bar_ld);
            }
            inflight = true;
        }
    }
    bool ok = true;
    bool pre = false;  // raw was zeroed for this shell-only item during the last item
    // forward pass: the next item's shell values (linear node index within the
    // plane, value) are loaded into registers during this item's output phase, up
    // to kPre per thread, so their global-memory latency is hidden
    constexpr int kPre = 4;
    int pidx[kPre], pcnt = 0, pe0 = 0, pe1 = 0;  // pe0, pe1: the prefetched item's shell range
    float pval[kPre];
    bool pref = false;  // pidx / pval hold this item's first kPre * kPlaneThreads entries
    for (; item < nitems && ok; item += gridDim.x) {
        const int b = item / kN, i = item % kN;
        const ApRhs<float> r = rhs[b];
        const int nx = item + gridDim.x;
        const float *nsrc = nullptr;
        bool nsparse = false;  // next item: shell-only right-hand side (a BEP column)
        int n_e0 = 0, n_e1 = 0;
        const float *n_qs = nullptr;
        if (nx < nitems && !skippable(nx)) {
            const ApRhs<float> &rn = rhs[nx / kN];
            nsrc = plane_src<INV>(rn, work, nx / kN, nx % kN);
            nsparse = !INV && !rn.f && rn.dens;
            if (!INV && rn.dens) {
                n_e0 = a.rp_shell[(int64_t)(nx % kN) * kN];
                n_e1 = a.rp_shell[(int64_t)(nx % kN + 1) * kN];
                n_qs = a.qsh + (size_t)(nx / kN) * a.n_shell;
            }
        }
        const bool have_pref = pref;
        pref = false;
        auto prefetch_next = [&]() {
            if (INV || !n_qs) return;
            const int off = (nx % kN) * kN * kN;
            pcnt = 0;
            pe0 = n_e0;
            pe1 = n_e1;
#pragma unroll
            for (int q = 0; q < kPre; ++q) {
                const int e = n_e0 + t + q * kPlaneThreads;
                if (e < n_e1) {
                    pidx[q] = a.shell[e] - off;
                    pval[q] = n_qs[e];
                    pcnt = q + 1;
                }
            }
            pref = true;
        };
        // stage the next item's input in raw (free whenever this is called)
        auto stage_next = [&]() {
            prefetch_next();
            if (nsrc) {
                if (t == 0) {
                    tc::mbar_arrive_expect_tx(bar_ld, kRawBytes);
                    tc::bulk_g2s(raw, nsrc, kRawBytes, bar_ld);
                }
                inflight = true;
            } else if (nsparse) {
                float4 *r4 = reinterpret_cast<float4 *>(raw);
                for (int q = t; q < kN * kN / 4; q += kPlaneThreads) r4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        if (skippable(item)) {
            if (!INV) {
                float4 *w4 = reinterpret_cast<float4 *>(work + ((size_t)b * kN + i) * kN * kN);
                for (int q = t; q < kN * kN / 4; q += kPlaneThreads) w4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            tc::fence_async_smem();
            __syncthreads();
            stage_next();
            tc::tc_fence_before_sync();
            __syncthreads();
            tc::tc_fence_after_sync();
            pre = nsparse;
            continue;
        }
        int ge0 = 0, ge1 = 0;  // gamma_in nodes of this plane (trace output)
        if (INV && r.out_trace) {
            ge0 = a.rp_gin[(int64_t)i * kN];
            ge1 = a.rp_gin[(int64_t)(i + 1) * kN];
        }
        // ---- input plane in smem ----------------------------------------------
        if (inflight) {
            const bool got = tc::mbar_wait(bar_ld, ld_phase, kWaitIters);
            if (got) {
                ld_phase ^= 1u;
                inflight = false;
            }
            if (!got) atomicExch(&g_tc_status, 1);
            if (!__syncthreads_and(got ? 1 : 0)) { ok = false; break; }
            if (!INV && (a.mask_f || fs != 1.f)) {
                // scale f and keep it on M^+ only
                const uint8_t *lab = a.labels + (size_t)i * kN * kN;
                for (int q = t; q < kN * kN / 4; q += kPlaneThreads) {
                    float4 v = reinterpret_cast<float4 *>(raw)[q];
                    v.x *= fs; v.y *= fs; v.z *= fs; v.w *= fs;
                    if (a.mask_f) {
                        const uint32_t lb = reinterpret_cast<const uint32_t *>(lab)[q];
                        if (!(lb & DPM_LBL_MPLUS)) v.x = 0.f;
                        if (!((lb >> 8) & DPM_LBL_MPLUS)) v.y = 0.f;
                        if (!((lb >> 16) & DPM_LBL_MPLUS)) v.z = 0.f;
                        if (!((lb >> 24) & DPM_LBL_MPLUS)) v.w = 0.f;
                    }
                    reinterpret_cast<float4 *>(raw)[q] = v;
                }
                __syncthreads();
            }
        } else if (!INV && !pre) {
            float4 *r4 = reinterpret_cast<float4 *>(raw);
            for (int q = t; q < kN * kN / 4; q += kPlaneThreads) r4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            __syncthreads();
        }
        if (!INV && r.dens) {
            const int e0 = have_pref ? pe0 : a.rp_shell[(int64_t)i * kN];
            const int e1 = have_pref ? pe1 : a.rp_shell[(int64_t)(i + 1) * kN];
            const float *qs = a.qsh + (size_t)b * a.n_shell;
            const int off = i * kN * kN;
            int e = e0 + t;
            if (have_pref) {
#pragma unroll
                for (int q = 0; q < kPre; ++q)
                    if (q < pcnt) raw[pidx[q]] += pval[q];
                e += kPre * kPlaneThreads;
            }
            for (; e < e1; e += kPlaneThreads) raw[a.shell[e] - off] += qs[e];
            __syncthreads();
        }
        // ---- phase A: rows -> folded, split operands ---------------------------
        // warp: 16 rows, two per step; lanes 0-15 take row 2s, lanes 16-31 row
        // 2s+1, lane l' = l mod 16 holding x[4l'..4l'+3] and x[124-4l'..127-4l'],
        // so the fold (sums e, differences o at m' = 4l'+u) is thread-local.
        // Rows p and 127-p (p < 64) go to A rows 16(p/8) + p%8 and that + 8, so
        // the fold over rows in phase C pairs TMEM lanes L and L^8, and the 8
        // lanes of a quarter-warp hold 8 consecutive p (conflict-free stores of
        // the MN-major second operand).
        const int lp = lane & 15, rsel = lane >> 4;
        float xa[8][4], xb[8][4];
#pragma unroll
        for (int st = 0; st < 8; ++st) {
            const int row = warp * 16 + 2 * st + rsel;
            const float4 v1 = reinterpret_cast<const float4 *>(raw)[row * (kN / 4) + lp];
            const float4 v2 = reinterpret_cast<const float4 *>(raw)[row * (kN / 4) + 31 - lp];
            xa[st][0] = v1.x; xa[st][1] = v1.y; xa[st][2] = v1.z; xa[st][3] = v1.w;
            xb[st][0] = v2.x; xb[st][1] = v2.y; xb[st][2] = v2.z; xb[st][3] = v2.w;
        }
        __syncthreads();  // the plane is in registers: the tiles may overwrite it
        float wm = 0.f;
#pragma unroll
        for (int st = 0; st < 8; ++st) {
            const int row = warp * 16 + 2 * st + rsel;
            const int pr = row < kH ? row : kN - 1 - row;
            const int LL = 16 * (pr >> 3) + (row < kH ? 0 : 8) + (pr & 7);
            float rm = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) rm = fmaxf(rm, fmaxf(fabsf(xa[st][u]), fabsf(xb[st][u])));
            rm = half_max(rm);
            float rinv;
            const float sr = pow2_scale(2.f * rm, &rinv);  // |e|, |o| <= 2 max|x| of the row
            float e[4], o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                e[u] = xa[st][u] + xb[st][3 - u];
                o[u] = xa[st][u] - xb[st][3 - u];
            }
            put4(S.A(0), S.A(1), LL, 4 * lp, e, sr);
            put4(S.A(2), S.A(3), LL, 4 * lp, o, sr);
            if (lp == 0) rowinv[LL] = rinv;
            wm = fmaxf(wm, rm);
        }
#pragma unroll
        for (int q = 16; q > 0; q >>= 1) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, q));
        if (lane == 0) wmax[warp] = wm;
        if (!run_transform(S, tm, phase)) { ok = false; break; }
        // ---- phase C: fold over rows (lanes L, L^8), A2 in MN-major layout --------
        // Columns [32 hc, 32 hc + 32) of the sums (modes 2c') and of the
        // differences (modes 2c'+1) of this thread's row, 16 at a time.
        float amax = 0.f;
#pragma unroll
        for (int w = 0; w < kPlaneThreads / 32; ++w) amax = fmaxf(amax, wmax[w]);
        float inv2;
        const float s2 = pow2_scale(256.f * amax, &inv2);
        {
            // row scale, sine-block scale and the second operand's scale in one
            // factor (powers of two: the products are exact)
            const float iD = rowinv[L] * (1.f / kSScale) * s2;
            const int sd = (L >> 3) & 1;            // 0: row p (sums), 1: row 127-p (differences)
            const float sgn = sd ? -1.f : 1.f;
            const int p = 8 * (L >> 4) + (L & 7);
            unsigned char *thi = S.A(sd ? 2 : 0), *tlo = S.A(sd ? 3 : 1);
#pragma unroll
            for (int c0 = 32 * hc; c0 < 32 * hc + 32; c0 += 16) {
                float de[16], dd[16];
                tc::tmem_ld16(lane_addr + c0, de);
                tc::tmem_ld16(lane_addr + kH + c0, dd);
                tc::tmem_wait_ld();
                float f2[32];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const float oe = de[u] * iD, od = dd[u] * iD;
                    const float pe = __shfl_xor_sync(0xffffffffu, oe, 8);
                    const float pd = __shfl_xor_sync(0xffffffffu, od, 8);
                    f2[2 * u] = fmaf(oe, sgn, pe);  // oe + pe, or pe - oe on row 127-p
                    f2[2 * u + 1] = fmaf(od, sgn, pd);
                }
#pragma unroll
                for (int q8 = 0; q8 < 4; ++q8) {
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        split_pack(f2[8 * q8 + 2 * u], f2[8 * q8 + 2 * u + 1], hw[u], lw[u]);
                    const uint32_t off = mn_off(2 * c0 + 8 * q8, p);
                    *reinterpret_cast<uint4 *>(thi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4 *>(tlo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
            }
        }
        if (!run_transform<true>(S, tm, phase)) { ok = false; break; }
        // ---- the operand region is free: stage the next item's input -------------
        const bool stage_trace = INV && r.out_trace;
        if (!stage_trace) stage_next();
        // ---- phase E: D2 (row = c = L); columns [0,64) even j-modes, [64,128) odd --
        const float iout = inv2 * (1.f / kSScale);
        if (!INV) {
            // j = 2c' + hc for column c = 64 hc + c' (even modes from the sums, odd
            // ones from the differences); four TMEM loads in flight per wait
            float *wrow = work + ((size_t)b * kN + i) * kN * kN + hc * kN + L;
#pragma unroll
            for (int c0 = 0; c0 < kH; c0 += 64) {
                float d[4][16];
#pragma unroll
                for (int q = 0; q < 4; ++q) tc::tmem_ld16(lane_addr + kH * hc + c0 + 16 * q, d[q]);
                tc::tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int u = 0; u < 16; ++u) wrow[2 * (c0 + 16 * q + u) * kN] = d[q][u] * iout;
            }
        } else {
            float *stage = raw;  // 128 x 128 fp32 (the operand region, free again)
            const int64_t pbase = (int64_t)i * kN * kN;
            // the first kPre * kPlaneThreads gamma_in nodes of the plane: their
            // positions are loaded now, so the gather below does not wait on them
            if (r.out_trace) {
#pragma unroll
                for (int q = 0; q < kPre; ++q) {
                    const int e = ge0 + t + q * kPlaneThreads;
                    if (e < ge1) pidx[q] = a.gin[e];
                }
            }
            if (r.out_dense) {
#pragma unroll
                for (int c0 = kH * hc; c0 < kH * hc + kH; c0 += 32) {
                    float d[2][16];  // two TMEM loads in flight per wait
                    tc::tmem_ld16(lane_addr + c0, d[0]);
                    tc::tmem_ld16(lane_addr + c0 + 16, d[1]);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 2; ++q)
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const int c = c0 + 16 * q + u;
                            const int j = c < kH ? 2 * c : 2 * (c - kH) + 1;
                            const float val = d[q][u] * iout;
                            const int64_t pp = pbase + (int64_t)j * kN + L;
                            float o = val;
                            if (a.mask_out && !(a.labels[pp] & (DPM_LBL_MPLUS | DPM_LBL_GEX))) o = 0.f;
                            r.out_dense[pp] = o;
                            if (r.out_trace) stage[j * kN + L] = val;
                        }
                }
            } else if (r.out_trace) {
                // trace only (every BEP column): the plane goes to the staging area
                // (j = 2c' + hc: the even modes from the sums, the odd ones from the
                // differences), four TMEM loads in flight per wait
                float *srow = stage + hc * kN + L;
#pragma unroll
                for (int c0 = 0; c0 < kH; c0 += 64) {
                    float d[4][16];
#pragma unroll
                    for (int q = 0; q < 4; ++q) tc::tmem_ld16(lane_addr + kH * hc + c0 + 16 * q, d[q]);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int u = 0; u < 16; ++u) srow[2 * (c0 + 16 * q + u) * kN] = d[q][u] * iout;
                }
            }
            if (r.out_trace) {
                __syncthreads();
#pragma unroll
                for (int q = 0; q < kPre; ++q) {
                    const int e = ge0 + t + q * kPlaneThreads;
                    if (e < ge1) r.out_trace[e] = stage[((pidx[q] / kN) % kN) * kN + pidx[q] % kN];
                }
                for (int e = ge0 + t + kPre * kPlaneThreads; e < ge1; e += kPlaneThreads) {
                    const int pg = a.gin[e];
                    r.out_trace[e] = stage[((pg / kN) % kN) * kN + pg % kN];
                }
                // the staging writes precede the next bulk copy into the same bytes
                tc::fence_async_smem();
                __syncthreads();
                stage_next();
            }
        }
        tc::tc_fence_before_sync();
        __syncthreads();
        tc::tc_fence_after_sync();
        pre = nsparse;
    }
    // a bulk copy issued for an item this CTA did not reach must land before exit
    if (inflight) tc::mbar_wait(bar_ld, ld_phase, kWaitIters);
    tc_epilogue(S);
}


// ---------------------------------------------------------------------------
// Pencil pass along i for a fixed j-mode jb: forward, scale/lambda, inverse.
// Thread t = c (the contiguous index), A rows = c, K = fold index over i / a.
// ---------------------------------------------------------------------------
constexpr int kPencilThreads = 128;

__global__ void __launch_bounds__(kPencilThreads, 2)
k_tc_pencil(TcArgs a, const ApRhs<float> *rhs, float *work, const __grid_constant__ CUtensorMap zmap) {
    const Smem S = smem_base();
    tc_prologue(S, a);
    const uint32_t tm = *S.tslot();
    const int t = threadIdx.x, warp = t >> 5;
    uint32_t phase = 0;
    const float w4 = (float)(4.0 / (a.h * a.h));
    for (int n = t; n < kN; n += kPencilThreads) S.w()[n] = w4 * a.s2[n];
    __syncthreads();
    const float sig = (float)(a.sigma_dev ? *a.sigma_dev : a.sigma);
    // (2/(N+1))^3, times 1 + kRzBias: the expected relative loss of the solve to
    // the tensor cores' round-toward-zero accumulation (tc_rz_bias: 4 main-term
    // steps per transform, 6 transforms, 6.45e-7; measured means -4e-7 to -6e-7
    // on dense random and Gaussian data), so that long time loops do not drift
    const double sc = 2.0 / (kN + 1);
    const float nscale = (float)(sc * sc * sc * (1.0 + kRzBias));
    const int nitems = a.B * kN;
    const size_t sN2 = (size_t)kN * kN;
    const uint32_t lane_addr = tm + ((uint32_t)(warp * 32) << 16);
    // The item's column block Z[b][0..128)[jb][0..128) (128 rows of 512 B) is
    // staged in the operand region by one tensor copy (box 128 x 1 x 128 x 1 of
    // the [b][i][j][c] workspace) once the previous item's second MMA has completed.
    float *raw = reinterpret_cast<float *>(S.A(0));
    uint64_t *bar_ld = S.bar() + 1;
    uint32_t ld_phase = 0;
    const int lane = t & 31;
    auto stage_block = [&](int it) {
        if (lane == 0) {
            tc::mbar_arrive_expect_tx(bar_ld, kN * kN * 4);
            tc::tma_load_4d(raw, &zmap, 0, it % kN, 0, it / kN, bar_ld);
        }
    };
    bool inflight = false;
    if (blockIdx.x < nitems) {
        if (warp == 0) stage_block(blockIdx.x);
        inflight = true;
    }
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int b = item / kN, jb = item % kN;
        (void)rhs;
        float *base = work + (size_t)b * kN * sN2 + (size_t)jb * kN + t;
        {
            const bool got = tc::mbar_wait(bar_ld, ld_phase, kWaitIters);
            if (got) {
                ld_phase ^= 1u;
                inflight = false;
            }
            if (!got) atomicExch(&g_tc_status, 1);
            if (!__syncthreads_and(got ? 1 : 0)) break;
        }
        // ---- phase A: fold along i, split, per-row (per-c) scale -----------
        float e[kH], o[kH];
#pragma unroll
        for (int mp = 0; mp < kH; ++mp) {
            const float x1 = raw[mp * kN + t], x2 = raw[(kN - 1 - mp) * kN + t];
            e[mp] = x1 + x2;
            o[mp] = x1 - x2;
        }
        __syncthreads();  // the block is in registers: the tiles may overwrite it
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
        // 64 columns per TMEM round trip (four loads in flight, one wait)
#pragma unroll
        for (int c0 = 0; c0 < 2 * kH; c0 += 64) {
            float d[4][16];
#pragma unroll
            for (int q = 0; q < 4; ++q) tc::tmem_ld16(lane_addr + c0 + 16 * q, d[q]);
            tc::tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int c = c0 + 16 * q + u;
                    const int am = c < kH ? 2 * c : 2 * (c - kH) + 1;
                    z[am] = d[q][u] * ((c0 < kH ? ie : io) * (1.f / kSScale));
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
        if (item + (int)gridDim.x < nitems) {
            if (warp == 0) stage_block(item + gridDim.x);
            inflight = true;
        }
        // ---- phase E: D3[c][i'] -> Z[i][jb][c] ---------------------------------
#pragma unroll
        for (int c0 = 0; c0 < 2 * kH; c0 += 64) {
            float d[4][16];
#pragma unroll
            for (int q = 0; q < 4; ++q) tc::tmem_ld16(lane_addr + c0 + 16 * q, d[q]);
            tc::tmem_wait_ld();
            const float sc2 = (c0 < kH ? ie : io) * (1.f / kSScale);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int c = c0 + 16 * q + u;
                    const int ii = c < kH ? 2 * c : 2 * (c - kH) + 1;
                    base[(size_t)ii * sN2] = d[q][u] * sc2;
                }
        }
        tc::tc_fence_before_sync();
        __syncthreads();
        tc::tc_fence_after_sync();
    }
    // copies issued for an item this CTA did not reach must land before exit
    if (inflight) tc::mbar_wait(bar_ld, ld_phase, kWaitIters);
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

// Tensor map of the workspace [B][i][j][c] (FP32, 128^3 per right-hand side)
// with a box of one (b, j) column block: 128 c x 1 j x 128 i x 1 b.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_work_map(CUtensorMap *map, float *work, int B) {
    static std::mutex mu;
    static EncodeTiledFn fn = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!fn) {
            void *f = nullptr;
            cudaDriverEntryPointQueryResult q{};
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                                 &q) != cudaSuccess ||
                q != cudaDriverEntryPointSuccess || !f) {
                set_error("tensor-core AP solve: cuTensorMapEncodeTiled is unavailable");
                return DPM_ECUDA;
            }
            fn = reinterpret_cast<EncodeTiledFn>(f);
        }
    }
    const cuuint64_t dims[4] = {(cuuint64_t)kN, (cuuint64_t)kN, (cuuint64_t)kN, (cuuint64_t)B};
    const cuuint64_t strides[3] = {(cuuint64_t)kN * 4, (cuuint64_t)kN * kN * 4,
                                   (cuuint64_t)kN * kN * kN * 4};
    const cuuint32_t box[4] = {(cuuint32_t)kN, 1, (cuuint32_t)kN, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, work, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("tensor-core AP solve: tensor map encoding failed (%d)", (int)r);
        return DPM_ECUDA;
    }
    return DPM_OK;
}

int tc_configure() {
    static PerDeviceOnce once;
    return once.run([] {
        DPM_CUDA(cudaFuncSetAttribute(k_tc_plane<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        DPM_CUDA(cudaFuncSetAttribute(k_tc_plane<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        DPM_CUDA(cudaFuncSetAttribute(k_tc_pencil, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        return (int)DPM_OK;
    });
}

}  // namespace

bool tc_supported(int N) { return N == kN || N == 256; }

size_t tc_scratch_elems(const ApParams &p, int B) {
    return p.N == kN ? (size_t)B * (size_t)p.n_shell : 0;  // the N = 256 solver scatters in place
}

int tc_status_check() {
    DPM_RET(tc256_status_check());
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

int tc_shell_pre(int64_t n_shell, const int *shell_nb, const float *dens, int64_t ng, int ncol, float2 *pre,
                 cudaStream_t s) {
    if (n_shell <= 0 || ncol <= 0) return DPM_OK;
    dim3 g((unsigned)std::min<int64_t>((n_shell + 255) / 256, 256), (unsigned)ncol);
    k_shell_pre<<<g, 256, 0, s>>>((int)n_shell, shell_nb, dens, ng, pre);
    DPM_LAUNCHED();
    return DPM_OK;
}

int ap_solve_tc(const ApParams &p, const ApRhs<float> *rhs_dev, float *work, cudaStream_t s) {
    if (!tc_supported(p.N)) {
        set_error("tensor-core AP solve supports N = 128 and 256 only (got %d)", p.N);
        return DPM_EUNSUPPORTED;
    }
    if (p.cond_flag) {
        set_error("tensor-core AP solve has no conditional right-hand sides");
        return DPM_EINVAL;
    }
    if (p.N == 256) return ap_solve_tc256(p, rhs_dev, work, s);
    if (p.cond_flag) {
        set_error("tensor-core AP solve has no conditional right-hand sides");
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
             p.rp_shell, p.gin, p.rp_gin, bops, tab + offW, p.scratch, p.n_shell,
             p.sigma_dev, p.fscale_dev};
    const int nitems = p.B * kN;
    if (p.n_shell > 0 && p.shell_nb) {
        if (!p.scratch) { set_error("tensor-core AP solve: shell scratch missing"); return DPM_EINVAL; }
        DPM_PROF("tc_shell_rhs", s);
        dim3 g((unsigned)std::min<int64_t>((p.n_shell + 255) / 256, 256), p.B);
        k_shell_rhs<<<g, 256, 0, s>>>((int)p.n_shell, 6.0 / (p.h * p.h), (float)(1.0 / (p.h * p.h)),
                                      p.sigma, p.sigma_dev, rhs_dev, p.shell_nb, p.scratch);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF("tc_plane_fwd", s);
        k_tc_plane<false><<<std::min(nitems, 2 * sms), kPlaneThreads, kSmemBytes, s>>>(a, rhs_dev, work);
        DPM_LAUNCHED();
    }
    CUtensorMap zmap;
    DPM_RET(encode_work_map(&zmap, work, p.B));
    {
        DPM_PROF("tc_pencil", s);
        k_tc_pencil<<<std::min(nitems, 2 * sms), kPencilThreads, kSmemBytes, s>>>(a, rhs_dev, work, zmap);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF("tc_plane_inv", s);
        k_tc_plane<true><<<std::min(nitems, 2 * sms), kPlaneThreads, kSmemBytes, s>>>(a, rhs_dev, work);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

}  // namespace dpm
