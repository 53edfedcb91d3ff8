// FFT-style auxiliary-problem solver for N = 256 (Definition 2.4), FP32 SIMT.
//
// The AP is diagonalised by the 3D DST-I: u = (2/p)^3 S S S [(S S S q) / lambda]
// with p = N + 1 = 257 and lambda_abc = sigma + (4/h^2) sum sin^2(pi a/(2p)).
// Here each 256-point DST-I costs O(log N) per point instead of the O(N) of a
// dense product, through two exact identities:
//
//  * the even/odd fold.  With x_{p-m} the mirror of x_m (m = 1..128),
//      y_{2b}   = sum_m sin(2 pi b m / p) (x_m - x_{p-m})
//      y_{p-2b} = sum_m sin(2 pi b m / p) (-1)^(m+1) (x_m + x_{p-m}),  b = 1..128,
//    so one real line is one "Z transform" Z(b) = sum_m sin(2 pi b m / p) e_m of
//    the complex sequence e = d + i s' (real part -> even modes, imaginary part
//    -> odd modes).  The inverse transform of a line whose modes are stored in
//    that packed form is again one Z transform, of U + i V with U = Y_{2b} +
//    Y_{p-2b}, V = Y_{2b} - Y_{p-2b}, followed by the mirror unfold.
//  * Rader's algorithm (p is prime; 3 generates the multiplicative group mod
//    257).  With m = 3^j and b = 3^-k the sine kernel depends only on j - k, and
//    since 3^128 = -1 (mod 257) the sequences are anti-periodic: Z is a
//    negacyclic convolution of length 128 with the fixed sequence
//    h_n = sin(2 pi 3^-n / p).  It is computed exactly as
//      twist by zeta^j (zeta = e^{i pi/128}) -> DFT_128 -> times DFT_128(h zeta^n)
//      -> inverse DFT_128 -> untwist.
//
// One convolution runs on a group of 16 threads holding 8 complex values each
// (position j = t + 16 n): an 8-point DFT in registers, twiddles, a transpose
// through 1 KB of shared memory (XOR-swizzled, conflict-free), a second 8-point
// DFT and a radix-2 step across thread pairs by shuffles; the product with the
// kernel's spectrum is taken in that (digit-reversed) order and the inverse
// DFT retraces the stages, so no reordering pass is needed.
//
// Three passes over HBM, 24 bytes per grid point for a dense solve:
//   P1 plane (k then j forward, plane i): a 2-CTA cluster holds the 256 x 256
//      FP32 plane (256 KB, more than one CTA's shared memory): CTA r the rows
//      j in [128 r, 128 r + 128).  The k transform is local; the j fold pairs
//      row j with row 255 - j, i.e. the two CTAs, and is done with plain
//      distributed-shared-memory loads (CTA 0 keeps the differences -> even j
//      modes, CTA 1 the signed sums -> odd j modes).
//   P2 pencil (i forward, times (2/p)^3 / lambda, i inverse) on tiles of 256 x
//      32 complex slots; the forward output feeds the inverse through a fixed
//      re-indexing inside the thread group.
//   P3 plane (j then k inverse) mirrors P1: the j unfold is the cluster
//      exchange (CTA 0 U, CTA 1 V), after which CTA r owns the rows of parity r.
// The workspace between passes holds plane i as [r][k-pair b][j-mode] of
// complex slots (re: k mode 2b, im: k mode p - 2b).  Every array is updated in
// place; the shared-memory views are XOR-swizzled so that lines and columns
// are both bank-conflict-free and each transform's scratch is its own line.
//
// The right-hand side is read by P1 directly (fscale f, masked to M^+) unless
// some right-hand side carries a density on gamma: then q is assembled in the
// workspace first (f part, plus L[v_gamma] on the shell).  P3 writes u
// (restricted to N^+ when asked) and/or the trace on gamma_in.
//
// No wait here spins: the cluster barriers are hardware barriers that both
// CTAs of a cluster reach the same number of times (the item loop is
// cluster-uniform and has no early exit).
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>
#include <complex>
#include <map>
#include <mutex>
#include <vector>

#include "dpm_internal.cuh"

namespace cg = cooperative_groups;

namespace dpm {

namespace {

constexpr int kN = 256, kP = 257, kM = 128;
constexpr int kThreads = 512;        // 32 groups of 16 threads
constexpr int kGroups = kThreads / 16;
constexpr int kPlaneF2 = kM * kM;    // complex slots of one CTA's half plane (128 KB)
constexpr int kPenSlots = 32;        // complex slots per pencil tile
constexpr int kPenThreads = 256;     // pencil pass: two CTAs per SM (one loads while one computes)
constexpr int kPenGroups = kPenThreads / 16;

// Constants of the length-128 convolution, laid out [register][thread t of the
// group] (a warp's two groups read the same words: broadcast, conflict-free).
struct FftTab {
    float2 twist[8][16];   // zeta^(t + 16 n)
    float2 w128[8][16];    // W128^(t k1)  (first-stage twiddles, forward)
    float2 w128i[8][16];   // conj W128^((2 s + (t & 1)) (t >> 1))  (inverse)
    float2 cs[8][16];      // the 2 x 2 spectral step, own value:     H(k0) + H(k1)
    float2 cc[8][16];      //                     partner's value: (H(k0) - H(k1)) W16^(+-r)
    uint32_t gidx[16][2];  // bytes n: (mu_j - 1) | 0x80 if sigma_j < 0, j = t + 16 n (input map)
    uint32_t sidx[16][2];  // bytes n: (beta_k - 1) | 0x80 if tau_k < 0, k = t + 16 n (output map)
};
constexpr int kTabBytes = (int)sizeof(FftTab);

// Products with sqrt(1/2) in the 8-point DFTs.  Its FP32 rounding lies below
// it, and every line passes through these products, so a plain product would
// shrink every transform by ~1e-8; the constant is kept as hi + lo (hi its
// FP32 rounding, lo the FP32 rounding of the remainder) and x sqrt(1/2) is
// formed as fma(x, hi, x lo): within an ulp and rounded to nearest, with no
// systematic gain.  (The other fixed twiddles are rounded once, per table
// entry, from double precision.)
struct KC { float hi, lo; };
constexpr KC kSqrtHalf{0.70710677f, 1.21016175e-08f};
__device__ __forceinline__ float kmul(float x, KC c) { return fmaf(x, c.hi, x * c.lo); }

// Complex sums and differences as packed two-lane FP32 adds (each lane rounded
// as a scalar add; a - b is a + (-b) exactly).
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, cneg(b)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// 4-point DFT in natural order; D = +1: exp(-2 pi i nk/4), D = -1: exp(+...)
template <int D> __device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = csub(a1, a3);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    if (D > 0) {
        a1 = make_float2(t1.x + t3.y, t1.y - t3.x);
        a3 = make_float2(t1.x - t3.y, t1.y + t3.x);
    } else {
        a1 = make_float2(t1.x - t3.y, t1.y + t3.x);
        a3 = make_float2(t1.x + t3.y, t1.y - t3.x);
    }
}

// 8-point DFT in registers, natural order in and out.
template <int D> __device__ __forceinline__ void dft8(float2 (&v)[8]) {
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<D>(e0, e1, e2, e3);
    dft4<D>(o0, o1, o2, o3);
    if (D > 0) {  // times W8^1, W8^2 = -i, W8^3
        o1 = make_float2(kmul(o1.x + o1.y, kSqrtHalf), kmul(o1.y - o1.x, kSqrtHalf));
        o2 = make_float2(o2.y, -o2.x);
        o3 = make_float2(kmul(o3.y - o3.x, kSqrtHalf), -kmul(o3.x + o3.y, kSqrtHalf));
    } else {      // times W8^-1, W8^-2 = +i, W8^-3
        o1 = make_float2(kmul(o1.x - o1.y, kSqrtHalf), kmul(o1.x + o1.y, kSqrtHalf));
        o2 = make_float2(-o2.y, o2.x);
        o3 = make_float2(-kmul(o3.x + o3.y, kSqrtHalf), kmul(o3.x - o3.y, kSqrtHalf));
    }
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

__device__ __forceinline__ float2 shfl_x1(float2 v) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1));
}

// This thread's twist factors and index maps, in registers for the kernel's
// lifetime; the other constants are read from the shared table where used.
struct Consts {
    float2 twist[8];
    uint32_t gidx[2], sidx[2];
};

__device__ __forceinline__ void load_consts(const FftTab *T, int t, Consts &K) {
#pragma unroll
    for (int n = 0; n < 8; ++n) K.twist[n] = T->twist[n][t];
    K.gidx[0] = T->gidx[t][0];
    K.gidx[1] = T->gidx[t][1];
    K.sidx[0] = T->sidx[t][0];
    K.sidx[1] = T->sidx[t][1];
}

__device__ __forceinline__ int byte_of(const uint32_t (&w)[2], int n) { return (w[n >> 2] >> (8 * (n & 3))) & 0xff; }

// The negacyclic convolution c_k = sum_j a_j h_(k-j) (h_(n+128) = -h_n) of this
// group's a_j, j = t + 16 n held in v[n]; on return v[n] = c_(t + 16 n).
// The DFT_128 of the twisted input is 128 = 8 x 16: an 8-point DFT over n in
// registers, twiddles W128^(t k1), a transpose so that the thread pair
// u = 2 k1 + par holds t = 2 s + par, and a second 8-point DFT over s; the
// radix-2 step that would finish the 16-point DFT over t, the product with the
// kernel's spectrum and the inverse radix-2 step are one 2 x 2 complex product
// per register with the partner's value (coefficients from double precision).
// buf(idx), idx < 128, is 1 KB of shared memory private to the group (any
// bijection onto it will do); the call starts and ends with a group barrier,
// so buf may be the storage the inputs were just gathered from.
template <class Buf>
__device__ __forceinline__ void neg_conv128(float2 (&v)[8], const Buf &buf, const FftTab *T, const Consts &K,
                                            int t) {
    const int k1 = t >> 1, par = t & 1;
#pragma unroll
    for (int n = 0; n < 8; ++n) v[n] = cmul(v[n], K.twist[n]);
    dft8<1>(v);
#pragma unroll
    for (int q = 1; q < 8; ++q) v[q] = cmul(v[q], T->w128[q][t]);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 8; ++q) buf(q * 16 + (t ^ (2 * q))) = v[q];
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 8; ++s) v[s] = buf(k1 * 16 + ((2 * s + par) ^ (2 * k1)));
    dft8<1>(v);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float2 o = shfl_x1(v[r]);
        v[r] = cadd(cmul(v[r], T->cs[r][t]), cmul(o, T->cc[r][t]));
    }
    dft8<-1>(v);
#pragma unroll
    for (int s = 0; s < 8; ++s) v[s] = cmul(v[s], T->w128i[s][t]);
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 8; ++s) buf(k1 * 16 + ((2 * s + par) ^ (2 * k1))) = v[s];
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = buf(q * 16 + (t ^ (2 * q)));
    dft8<-1>(v);
#pragma unroll
    for (int n = 0; n < 8; ++n) v[n] = cmulc(v[n], K.twist[n]);
    __syncwarp();
}

// Shared-memory views.  Half plane of P1 / P3: 128 x 128 complex slots.
struct RowBuf {  // contiguous line
    float2 *p;
    __device__ float2 &operator()(int i) const { return p[i]; }
};
struct ColBuf {  // the slots of "column" c of a [row][c ^ row] array
    float2 *p;
    int c;
    __device__ float2 &operator()(int i) const { return p[i * kM + (c ^ i)]; }
};

struct PassArgs256 {
    int B;
    const ApRhs<float> *rhs;
    float *work;
    int from_work;  // P1: q assembled in the workspace (else read fscale f from rhs)
    int mask_f, mask_out;
    double fscale, h, sigma;
    const double *fscale_dev, *sigma_dev;
    const uint8_t *labels;
    const int *rp_gin, *gin;
    const float *s2;    // sin^2(pi (n + 1)/(2 p)), n < 256
    const FftTab *tab;
};

__device__ __forceinline__ void copy_tab(FftTab *dst, const FftTab *src) {
    const int4 *s = reinterpret_cast<const int4 *>(src);
    int4 *d = reinterpret_cast<int4 *>(dst);
    for (int e = threadIdx.x; e < kTabBytes / 16; e += blockDim.x) d[e] = s[e];
}

// ---------------------------------------------------------------------------
// P1: forward DST along k then j of plane i; cluster of two CTAs per plane.
// ---------------------------------------------------------------------------
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1) k_fft_plane_fwd(PassArgs256 a) {
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *D = reinterpret_cast<float2 *>(smraw);
    FftTab *T = reinterpret_cast<FftTab *>(smraw + kPlaneF2 * sizeof(float2));
    copy_tab(T, a.tab);
    __syncthreads();
    const int tid = threadIdx.x, grp = tid >> 4, t = tid & 15;
    Consts K;
    load_consts(T, t, K);
    float2 *peer = cl.map_shared_rank(D, r ^ 1);
    const float fs = (float)(a.fscale_dev ? *a.fscale_dev : a.fscale);
    const int ncl = gridDim.x >> 1, cid = blockIdx.x >> 1;
    const size_t n3 = (size_t)kN * kN * kN;
    for (int item = cid; item < a.B * kN; item += ncl) {
        const int b = item / kN, i = item - b * kN;
        const size_t plane = (size_t)b * n3 + (size_t)i * kN * kN;
        // ---- load rows j in [128 r, 128 r + 128) (128 KB; all 16 float4 loads of a
        //      thread in flight at once: nothing overlaps this copy) -----------------
        float4 *D4 = reinterpret_cast<float4 *>(D);
        const size_t off = plane + (size_t)kM * r * kN;  // first float of the half plane
        if (a.from_work) {
            const float4 *src = reinterpret_cast<const float4 *>(a.work + off);
#pragma unroll 16
            for (int e = tid; e < kPlaneF2 / 2; e += kThreads) D4[e] = src[e];
        } else {
            const ApRhs<float> rb = a.rhs[b];
            const size_t loff = (size_t)i * kN * kN + (size_t)kM * r * kN;
            const uchar4 *lab4 = a.labels ? reinterpret_cast<const uchar4 *>(a.labels + loff) : nullptr;
            const float4 *src = rb.f ? reinterpret_cast<const float4 *>(rb.f + loff) : nullptr;
#pragma unroll 4
            for (int e = tid; e < kPlaneF2 / 2; e += kThreads) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (src) {
                    v = src[e];
                    v.x *= fs; v.y *= fs; v.z *= fs; v.w *= fs;
                    if (a.mask_f && lab4) {
                        const uchar4 l = lab4[e];
                        if (!(l.x & DPM_LBL_MPLUS)) v.x = 0.f;
                        if (!(l.y & DPM_LBL_MPLUS)) v.y = 0.f;
                        if (!(l.z & DPM_LBL_MPLUS)) v.z = 0.f;
                        if (!(l.w & DPM_LBL_MPLUS)) v.w = 0.f;
                    }
                }
                D4[e] = v;
            }
        }
        __syncthreads();
        // ---- k transform of each local row, in place: complex slot b' at b' ^ row ----
        for (int row = grp; row < kM; row += kGroups) {
            const float *x = reinterpret_cast<const float *>(D + row * kM);
            float2 v[8];
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int gb = byte_of(K.gidx, n), m = (gb & 0x7f) + 1;
                const float x1 = x[m - 1], x2 = x[kN - m];
                const float d = x1 - x2, s = (m & 1) ? x1 + x2 : -(x1 + x2);
                v[n] = (gb & 0x80) ? make_float2(-d, -s) : make_float2(d, s);
            }
            neg_conv128(v, RowBuf{D + row * kM}, T, K, t);
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int sb = byte_of(K.sidx, n), bo = sb & 0x7f;
                D[row * kM + (bo ^ row)] = (sb & 0x80) ? cneg(v[n]) : v[n];
            }
        }
        cl.sync();
        // ---- j fold across the pair: CTA 0 D = Y0[j'] - Y1[127-j'], CTA 1 S' = (-1)^j' (Y0 + Y1)
        for (int c = 0; c < 4; ++c) {
            float2 nv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = tid + kThreads * u, rr = e >> 7, bc = e & 127;
                const int row = rr < 16 ? 16 * c + rr : 127 - 16 * c - (rr - 16), prow = 127 - row;
                const float2 y0 = (r == 0 ? D : peer)[row * kM + (bc ^ row)];
                const float2 y1 = (r == 0 ? peer : D)[prow * kM + (bc ^ prow)];
                nv[u] = r == 0 ? csub(y0, y1) : ((row & 1) ? cneg(cadd(y0, y1)) : cadd(y0, y1));
            }
            cl.sync();
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = tid + kThreads * u, rr = e >> 7, bc = e & 127;
                const int row = rr < 16 ? 16 * c + rr : 127 - 16 * c - (rr - 16);
                D[row * kM + (bc ^ row)] = nv[u];
            }
        }
        __syncthreads();
        // ---- j transform of each k-pair column bc: output beta at row beta - 1 ----
        for (int bc = grp; bc < kM; bc += kGroups) {
            const ColBuf col{D, bc};
            float2 v[8];
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int gb = byte_of(K.gidx, n);
                const float2 z = col(gb & 0x7f);
                v[n] = (gb & 0x80) ? cneg(z) : z;
            }
            neg_conv128(v, col, T, K, t);
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int sb = byte_of(K.sidx, n);
                col(sb & 0x7f) = (sb & 0x80) ? cneg(v[n]) : v[n];
            }
        }
        __syncthreads();
        // ---- store [r][k-pair][j-mode] complex slots (in place over the half plane)
        float4 *dst = reinterpret_cast<float4 *>(a.work + off);
#pragma unroll 4
        for (int e = tid; e < kPlaneF2 / 2; e += kThreads) {
            const int line = e >> 6, be = 2 * (e & 63);
            const float2 p0 = D[be * kM + (line ^ be)], p1 = D[(be + 1) * kM + (line ^ (be + 1))];
            dst[e] = make_float4(p0.x, p0.y, p1.x, p1.y);
        }
        __syncthreads();
    }
    cl.sync();
}

// ---------------------------------------------------------------------------
// P2: i forward, times (2/p)^3 / lambda, i inverse, on tiles of 256 x 32 slots.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pen_f2(int i, int s) {  // complex slot (i, s) of the tile
    return i * kPenSlots + ((((s >> 1) ^ (i & 15)) << 1) | (s & 1));
}

__global__ void __launch_bounds__(kPenThreads, 2) k_fft_pencil(PassArgs256 a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *P = reinterpret_cast<float2 *>(smraw);                                 // 256 x 32 slots
    float2 *scr = P + kN * kPenSlots;                                              // 16 x 128
    float *w = reinterpret_cast<float *>(scr + kPenGroups * kM);                   // 256
    FftTab *T = reinterpret_cast<FftTab *>(w + kN);
    copy_tab(T, a.tab);
    const float w4 = (float)(4.0 / (a.h * a.h));
    for (int n = threadIdx.x; n < kN; n += kPenThreads) w[n] = w4 * a.s2[n];
    __syncthreads();
    const int tid = threadIdx.x, grp = tid >> 4, t = tid & 15;
    Consts K;
    load_consts(T, t, K);
    const float sig = (float)(a.sigma_dev ? *a.sigma_dev : a.sigma);
    const double nd = 2.0 / kP;
    const float norm = (float)(nd * nd * nd);
    const int tiles = kN * kN / 2 / kPenSlots;  // complex slots per plane / tile width
    const size_t n3 = (size_t)kN * kN * kN;
    const RowBuf sb{scr + grp * kM};
    float *Pf = reinterpret_cast<float *>(P);
    for (int item = blockIdx.x; item < a.B * tiles; item += gridDim.x) {
        const int b = item / tiles, tile = item - b * tiles;
        const size_t base = (size_t)b * n3 + (size_t)tile * kPenSlots * 2;  // float offset in plane 0
        // ---- load: 256 rows i of 32 slots (256 B each) -----------------------------
#pragma unroll 8
        for (int e = tid; e < kN * kPenSlots / 2; e += kPenThreads) {
            const int i = e >> 4, q = e & 15;
            const float4 v = *reinterpret_cast<const float4 *>(a.work + base + (size_t)i * kN * kN + 4 * q);
            reinterpret_cast<float4 *>(P)[i * (kPenSlots / 2) + (q ^ (i & 15))] = v;
        }
        __syncthreads();
        for (int pid = grp; pid < 2 * kPenSlots; pid += kPenGroups) {
            const int s = pid >> 1, comp = pid & 1;
            const int gs = tile * kPenSlots + s;                 // slot in the plane
            const int rr = gs >> 14, bl = (gs >> 7) & 127, be = gs & 127;
            const int J = rr ? kP - 2 * (be + 1) : 2 * (be + 1);
            const int kap = comp ? kP - 2 * (bl + 1) : 2 * (bl + 1);
            const float base_l = sig + w[kap - 1] + w[J - 1];
            auto X = [&](int i) -> float & { return Pf[2 * pen_f2(i, s) + comp]; };
            float2 v[8];
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int gb = byte_of(K.gidx, n), m = (gb & 0x7f) + 1;
                const float x1 = X(m - 1), x2 = X(kN - m);
                const float d = x1 - x2, sv = (m & 1) ? x1 + x2 : -(x1 + x2);
                v[n] = (gb & 0x80) ? make_float2(-d, -sv) : make_float2(d, sv);
            }
            neg_conv128(v, sb, T, K, t);
            // spectral scale and the U/V combination, at the forward output's position k
            float2 cmb[8];
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int bi = (byte_of(K.sidx, n) & 0x7f) + 1;
                // (2/p)^3 / lambda by the fast division (about 2 ulp, as the tensor-core
                // pencil): the IEEE division was ~8 % of the pass's instructions
                const float sre = __fdividef(norm, base_l + w[2 * bi - 1]);
                const float sim = __fdividef(norm, base_l + w[kP - 2 * bi - 1]);
                const float cr = v[n].x * sre, ci = v[n].y * sim;
                cmb[n] = make_float2(cr + ci, cr - ci);
            }
            // inverse input at position (128 - k) mod 128, negated unless k = 0:
            // thread (16 - t) & 15, register 7 - n (t != 0) or (8 - n) & 7 (t = 0)
            const int src = (threadIdx.x & 16) | ((16 - t) & 15);
            float2 rcv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float rx = __shfl_sync(0xffffffffu, cmb[q].x, src);
                const float ry = __shfl_sync(0xffffffffu, cmb[q].y, src);
                rcv[7 - q] = make_float2(rx, ry);
            }
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const float2 z = (t == 0) ? rcv[(n + 7) & 7] : rcv[n];
                v[n] = (t == 0 && n == 0) ? z : cneg(z);
            }
            neg_conv128(v, sb, T, K, t);
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int sbt = byte_of(K.sidx, n), nn = (sbt & 0x7f) + 1;
                const float2 z = (sbt & 0x80) ? cneg(v[n]) : v[n];  // (T_U(nn), T_V(nn))
                if (nn & 1) {
                    X(nn - 1) = z.x;
                    X(kN - nn) = -z.y;
                } else {
                    X(nn - 1) = z.y;
                    X(kN - nn) = -z.x;
                }
            }
            __syncwarp();
        }
        __syncthreads();
#pragma unroll 4
        for (int e = tid; e < kN * kPenSlots / 2; e += kPenThreads) {
            const int i = e >> 4, q = e & 15;
            *reinterpret_cast<float4 *>(a.work + base + (size_t)i * kN * kN + 4 * q) =
                reinterpret_cast<const float4 *>(P)[i * (kPenSlots / 2) + (q ^ (i & 15))];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// P3: inverse along j then k of plane i (cluster of two CTAs), then the outputs.
// ---------------------------------------------------------------------------
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1) k_fft_plane_inv(PassArgs256 a) {
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *D = reinterpret_cast<float2 *>(smraw);
    FftTab *T = reinterpret_cast<FftTab *>(smraw + kPlaneF2 * sizeof(float2));
    copy_tab(T, a.tab);
    __syncthreads();
    const int tid = threadIdx.x, grp = tid >> 4, t = tid & 15;
    Consts K;
    load_consts(T, t, K);
    float2 *peer = cl.map_shared_rank(D, r ^ 1);
    const int ncl = gridDim.x >> 1, cid = blockIdx.x >> 1;
    const size_t n3 = (size_t)kN * kN * kN;
    const uint8_t keep = DPM_LBL_MPLUS | DPM_LBL_GEX;
    for (int item = cid; item < a.B * kN; item += ncl) {
        const int b = item / kN, i = item - b * kN;
        const size_t off = (size_t)b * n3 + (size_t)i * kN * kN + (size_t)kM * r * kN;
        // ---- load [k-pair][j-mode] of this CTA's j-mode half, natural layout -------
        const float4 *src = reinterpret_cast<const float4 *>(a.work + off);
        float4 *D4 = reinterpret_cast<float4 *>(D);
#pragma unroll 16
        for (int e = tid; e < kPlaneF2 / 2; e += kThreads) D4[e] = src[e];
        cl.sync();
        // ---- j unfold across the pair: CTA 0 U = A0 + A1, CTA 1 V = A0 - A1 ---------
        for (int c = 0; c < 4; ++c) {
            float2 nv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = 4096 * c + tid + kThreads * u;
                const float2 mine = D[e], theirs = peer[e];
                nv[u] = r == 0 ? cadd(mine, theirs) : csub(theirs, mine);
            }
            cl.sync();
#pragma unroll
            for (int u = 0; u < 8; ++u) D[4096 * c + tid + kThreads * u] = nv[u];
        }
        __syncthreads();
        // ---- j inverse per k-pair line bc; row n of the output -> local row lr ----
        for (int bc = grp; bc < kM; bc += kGroups) {
            const RowBuf line{D + bc * kM};
            float2 v[8];
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int gb = byte_of(K.gidx, n);
                const float2 z = line(gb & 0x7f);
                v[n] = (gb & 0x80) ? cneg(z) : z;
            }
            neg_conv128(v, line, T, K, t);
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int sbt = byte_of(K.sidx, n), nn = (sbt & 0x7f) + 1;
                const float2 z = (sbt & 0x80) ? cneg(v[n]) : v[n];
                int lr;
                float2 val;
                if (r == 0) {  // T_U: x_n (n odd), -x_{p-n} (n even)
                    if (nn & 1) { lr = (nn - 1) >> 1; val = z; }
                    else { lr = kM - (nn >> 1); val = cneg(z); }
                } else {       // T_V: x_n (n even), -x_{p-n} (n odd)
                    if (nn & 1) { lr = (kN - 1 - nn) >> 1; val = cneg(z); }
                    else { lr = (nn >> 1) - 1; val = z; }
                }
                D[bc * kM + (lr ^ bc)] = val;
            }
        }
        __syncthreads();
        // ---- k inverse per local row lr (complex over the k-pairs) -----------------
        float *Df = reinterpret_cast<float *>(D);
        for (int lr = grp; lr < kM; lr += kGroups) {
            const ColBuf col{D, lr};
            float2 v[8];
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int gb = byte_of(K.gidx, n);
                const float2 y = col(gb & 0x7f);
                const float2 uv = make_float2(y.x + y.y, y.x - y.y);
                v[n] = (gb & 0x80) ? cneg(uv) : uv;
            }
            neg_conv128(v, col, T, K, t);
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int sbt = byte_of(K.sidx, n), nn = (sbt & 0x7f) + 1;
                const float2 z = (sbt & 0x80) ? cneg(v[n]) : v[n];
                const float xa = (nn & 1) ? z.x : z.y, xb = (nn & 1) ? -z.y : -z.x;
                const int ka = nn - 1, kb = kN - nn;  // x_k stored at float 2 (slot (k/2, lr)) + (k & 1)
                Df[2 * ((ka >> 1) * kM + (lr ^ (ka >> 1))) + (ka & 1)] = xa;
                Df[2 * ((kb >> 1) * kM + (lr ^ (kb >> 1))) + (kb & 1)] = xb;
            }
        }
        __syncthreads();
        // ---- outputs: rows j = 2 lr + r of plane i ------------------------------------
        const ApRhs<float> rb = a.rhs[b];
        const size_t pl = (size_t)i * kN * kN;
        if (rb.out_dense) {
#pragma unroll 4
            for (int e = tid; e < kPlaneF2; e += kThreads) {
                const int lr = e >> 7, sl = e & 127;
                float2 val = D[sl * kM + (lr ^ sl)];
                const size_t node = pl + (size_t)(2 * lr + r) * kN + 2 * sl;
                if (a.mask_out) {
                    const uchar2 l = *reinterpret_cast<const uchar2 *>(a.labels + node);
                    if (!(l.x & keep)) val.x = 0.f;
                    if (!(l.y & keep)) val.y = 0.f;
                }
                *reinterpret_cast<float2 *>(rb.out_dense + node) = val;
            }
        }
        if (rb.out_trace && a.rp_gin) {
            const int e0 = a.rp_gin[i * kN], e1 = a.rp_gin[i * kN + kN];
            for (int e = e0 + tid; e < e1; e += kThreads) {
                const int node = a.gin[e], j = (node >> 8) & 255, k = node & 255;
                if ((j & 1) != r) continue;
                const int lr = j >> 1;
                rb.out_trace[e] = Df[2 * ((k >> 1) * kM + (lr ^ (k >> 1))) + (k & 1)];
            }
        }
        __syncthreads();
    }
    cl.sync();
}

// ---------------------------------------------------------------------------
// Right-hand side assembly in the workspace (when some right-hand side has a
// density on gamma): X = fscale f (on M^+ when masked), then X += L[v_gamma]
// on the shell: (sigma + 6/h^2) v(self) - (1/h^2) sum of v over the 6 neighbours.
// ---------------------------------------------------------------------------
__global__ void k_fft_q(const ApRhs<float> *rhs, int mask_f, double fscale, const double *fscale_dev,
                        const uint8_t *lab, float *X) {
    const int b = blockIdx.y;
    const ApRhs<float> rb = rhs[b];
    const float fs = (float)(fscale_dev ? *fscale_dev : fscale);
    const size_t n4 = (size_t)kN * kN * kN / 4;
    float4 *x = reinterpret_cast<float4 *>(X + (size_t)b * kN * kN * kN);
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n4; q += (size_t)gridDim.x * blockDim.x) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rb.f) {
            v = reinterpret_cast<const float4 *>(rb.f)[q];
            v.x *= fs; v.y *= fs; v.z *= fs; v.w *= fs;
            if (mask_f) {
                const uchar4 l = reinterpret_cast<const uchar4 *>(lab)[q];
                if (!(l.x & DPM_LBL_MPLUS)) v.x = 0.f;
                if (!(l.y & DPM_LBL_MPLUS)) v.y = 0.f;
                if (!(l.z & DPM_LBL_MPLUS)) v.z = 0.f;
                if (!(l.w & DPM_LBL_MPLUS)) v.w = 0.f;
            }
        }
        x[q] = v;
    }
}

__global__ void k_fft_shell(int n_shell, double c6, float coff, double sigma, const double *sigma_dev,
                            const ApRhs<float> *rhs, const int *shell, const int *shell_nb, float *X) {
    __shared__ float cd;
    if (threadIdx.x == 0) cd = (float)((sigma_dev ? *sigma_dev : sigma) + c6);
    __syncthreads();
    const int b = blockIdx.y;
    const ApRhs<float> rb = rhs[b];
    if (!rb.dens) return;
    float *x = X + (size_t)b * kN * kN * kN;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_shell; e += gridDim.x * blockDim.x) {
        const int *nb = shell_nb + 8 * (size_t)e;
        float acc = 0.f;
#pragma unroll
        for (int q = 1; q < 7; ++q)
            if (nb[q] >= 0) acc += rb.dens[nb[q]];
        const float self = nb[0] >= 0 ? rb.dens[nb[0]] : 0.f;
        x[shell[e]] += cd * self - coff * acc;
    }
}

// ---------------------------------------------------------------------------
// Host: constant tables (double precision, rounded once), per device.
// ---------------------------------------------------------------------------
void build_tab(FftTab &T) {
    using cd = std::complex<double>;
    const double pi = 3.14159265358979323846;
    int pw[256];
    pw[0] = 1;
    for (int j = 1; j < 256; ++j) pw[j] = (pw[j - 1] * 3) % kP;
    auto fold = [](int v, int &sg) { sg = v <= kM ? 1 : -1; return v <= kM ? v : kP - v; };
    // h_n = w_(-n), w_n = sin(2 pi 3^n / p); twisted by zeta^n; DFT_128 / 128
    cd ht[kM];
    for (int n = 0; n < kM; ++n) {
        const double hv = sin(2.0 * pi * (double)pw[(256 - n) % 256] / kP);
        ht[n] = hv * std::polar(1.0, pi * n / kM);
    }
    cd H[kM];
    for (int k = 0; k < kM; ++k) {
        cd s = 0;
        for (int n = 0; n < kM; ++n) s += ht[n] * std::polar(1.0, -2.0 * pi * (double)((n * k) % kM) / kM);
        H[k] = s / (double)kM;
    }
    auto f2 = [](cd z) { return make_float2((float)z.real(), (float)z.imag()); };
    for (int t = 0; t < 16; ++t) {
        uint32_t g[2] = {0, 0}, sdx[2] = {0, 0};
        const int k1 = t >> 1, par = t & 1;
        for (int n = 0; n < 8; ++n) {
            T.twist[n][t] = f2(std::polar(1.0, pi * (double)(t + 16 * n) / kM));
            T.w128[n][t] = f2(std::polar(1.0, -2.0 * pi * (double)((t * n) % kM) / kM));
            T.w128i[n][t] = f2(std::polar(1.0, 2.0 * pi * (double)(((2 * n + par) * k1) % kM) / kM));
            // thread pair (k1, par): outputs k0 = k1 + 8 n (par 0) and k0 + 64 (par 1)
            const cd h0 = H[k1 + 8 * n], h1 = H[k1 + 8 * n + 64];
            const cd w = std::polar(1.0, (par ? 2.0 : -2.0) * pi * (double)n / 16.0);
            T.cs[n][t] = f2(h0 + h1);
            T.cc[n][t] = f2((h0 - h1) * w);
            const int j = t + 16 * n;
            int sg, tg;
            const int mu = fold(pw[j], sg);
            const int be = fold(pw[(256 - j) % 256], tg);
            g[n >> 2] |= (uint32_t)((mu - 1) | (sg < 0 ? 0x80 : 0)) << (8 * (n & 3));
            sdx[n >> 2] |= (uint32_t)((be - 1) | (tg < 0 ? 0x80 : 0)) << (8 * (n & 3));
        }
        T.gidx[t][0] = g[0];
        T.gidx[t][1] = g[1];
        T.sidx[t][0] = sdx[0];
        T.sidx[t][1] = sdx[1];
    }
}

const FftTab *fft_tab() {
    static std::mutex mu;
    static std::map<int, void *> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return static_cast<const FftTab *>(it->second);
    FftTab h;
    build_tab(h);
    void *d = nullptr;
    if (cudaMalloc(&d, sizeof(FftTab)) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, &h, sizeof(FftTab), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    cache[dev] = d;
    return static_cast<const FftTab *>(d);
}

constexpr int kSmemPlane = kPlaneF2 * (int)sizeof(float2) + kTabBytes;
constexpr int kSmemPencil = (kN * kPenSlots + kPenGroups * kM) * (int)sizeof(float2) + kN * 4 + kTabBytes;

int configure_fft() {
    static PerDeviceOnce once;
    return once.run([] {
        DPM_CUDA(cudaFuncSetAttribute(k_fft_plane_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemPlane));
        DPM_CUDA(cudaFuncSetAttribute(k_fft_plane_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemPlane));
        DPM_CUDA(cudaFuncSetAttribute(k_fft_pencil, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemPencil));
        return (int)DPM_OK;
    });
}

}  // namespace

bool fft_supported(int N) { return N == kN; }

int ap_solve_fft256(const ApParams &p, const ApRhs<float> *rhs_dev, float *work, cudaStream_t s) {
    if (p.N != kN) {
        set_error("FFT-style AP solve supports N = 256 only (got %d)", p.N);
        return DPM_EUNSUPPORTED;
    }
    if (p.cond_flag) {
        set_error("FFT-style AP solve has no conditional right-hand sides");
        return DPM_EINVAL;
    }
    if ((p.mask_f || p.mask_out) && !p.labels) { set_error("FFT-style AP solve: labels missing"); return DPM_EINVAL; }
    DPM_RET(configure_fft());
    const FftTab *tab = fft_tab();
    const float *ftab = dst_fold_table<float>(kN);
    if (!tab || !ftab) { set_error("FFT-style AP solve: table allocation failed"); return DPM_ENOMEM; }
    int dev = 0, sms = 0;
    DPM_CUDA(cudaGetDevice(&dev));
    DPM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int H = kN / 2, NEp = (H + 3) & ~3;
    const float *s2 = ftab + (size_t)H * NEp + (size_t)H * NEp;  // sin^2 weights after the fold tables
    // a density on gamma anywhere in the batch: assemble q in the workspace first
    const bool shell = p.n_shell > 0 && p.shell_nb;
    PassArgs256 a{p.B, rhs_dev, work, shell ? 1 : 0, p.mask_f, p.mask_out, p.fscale, p.h, p.sigma,
                  p.fscale_dev, p.sigma_dev, p.labels, p.rp_gin, p.gin, s2, tab};
    if (shell) {
        DPM_PROF("fft256_rhs", s);
        const dim3 ge(4 * sms, p.B);
        k_fft_q<<<ge, 256, 0, s>>>(rhs_dev, p.mask_f, p.fscale, p.fscale_dev, p.labels, work);
        DPM_LAUNCHED();
        const dim3 gs((unsigned)std::min<int64_t>((p.n_shell + 255) / 256, 256), p.B);
        k_fft_shell<<<gs, 256, 0, s>>>((int)p.n_shell, 6.0 / (p.h * p.h), (float)(1.0 / (p.h * p.h)), p.sigma,
                                       p.sigma_dev, rhs_dev, p.shell, p.shell_nb, work);
        DPM_LAUNCHED();
    }
    const int gridc = std::max(2, (sms / 2) * 2);  // one CTA per SM, clusters of two
    {
        DPM_PROF("fft256_plane_fwd", s);
        k_fft_plane_fwd<<<gridc, kThreads, kSmemPlane, s>>>(a);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF("fft256_pencil", s);
        k_fft_pencil<<<std::max(1, 2 * sms), kPenThreads, kSmemPencil, s>>>(a);
        DPM_LAUNCHED();
    }
    {
        DPM_PROF("fft256_plane_inv", s);
        k_fft_plane_inv<<<gridc, kThreads, kSmemPlane, s>>>(a);
        DPM_LAUNCHED();
    }
    return DPM_OK;
}

}  // namespace dpm
