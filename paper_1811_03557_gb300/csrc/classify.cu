// Node classification and index lists (Definition 2.1).
//
// M^+ / M^- are decided per node in IEEE double with explicit round-to-nearest
// intrinsics (no FMA contraction), so the labels are reproducible bit for bit:
//   x_j = lo + (j*h), t = (x - c)/a, inside iff ((tx*tx + ty*ty) + tz*tz) < 1.
// With M^+ at least 2 nodes away from every cube face, the point sets of
// Definition 2.1 reduce to 6-neighbour tests:
//   gamma_in = M^+ nodes with a neighbour in M^-,
//   gamma_ex = M^- nodes with a neighbour in M^+,
//   N^+ = M^+ u gamma_ex.
// The "shell" (M^- nodes that are in gamma_ex or next to a node of gamma) is
// where L[v_gamma] of a density on gamma can be nonzero.
#include <cub/block/block_scan.cuh>

#include "dpm_internal.cuh"

namespace dpm {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 4096;  // nodes per compaction block
constexpr int kLists = 5;     // M+, gamma_in, gamma_ex, gamma, shell

// kind 2 (spherical shell): inside iff the form of the outer sphere (radius ax)
// is < 1 and that of the inner sphere (radius r_in) is > 1.  Kinds 3 / 4: the
// form of the sphere of radius ax is < 1 and that of the sphere of radius r_in
// about (cx, cy, cz + zoff) is < 1 (3) or > 1 (4).
__global__ void k_inside(int N, double lo, double h, double cx, double cy, double cz, double ax,
                         double ay, double az, int kind, double r_in, double zoff, uint8_t *labels) {
    int64_t n3 = (int64_t)N * N * N;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n3;
         p += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(p % N), j = (int)((p / N) % N), i = (int)(p / ((int64_t)N * N));
        double x = __dadd_rn(lo, __dmul_rn((double)(i + 1), h));
        double y = __dadd_rn(lo, __dmul_rn((double)(j + 1), h));
        double z = __dadd_rn(lo, __dmul_rn((double)(k + 1), h));
        double tx = __ddiv_rn(__dsub_rn(x, cx), ax);
        double ty = __ddiv_rn(__dsub_rn(y, cy), ay);
        double tz = __ddiv_rn(__dsub_rn(z, cz), az);
        double s = __dadd_rn(__dadd_rn(__dmul_rn(tx, tx), __dmul_rn(ty, ty)), __dmul_rn(tz, tz));
        bool in = s < 1.0;
        if (kind >= 2) {
            const double czz = kind == 2 ? cz : __dadd_rn(cz, zoff);
            const double ux = __ddiv_rn(__dsub_rn(x, cx), r_in);
            const double uy = __ddiv_rn(__dsub_rn(y, cy), r_in);
            const double uz = __ddiv_rn(__dsub_rn(z, czz), r_in);
            const double si = __dadd_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)), __dmul_rn(uz, uz));
            in = in && (kind == 3 ? si < 1.0 : si > 1.0);
        }
        labels[p] = in ? (uint8_t)DPM_LBL_MPLUS : (uint8_t)0;
    }
}

__device__ __forceinline__ bool in_plus(const uint8_t *lab, int N, int i, int j, int k) {
    if (i < 0 || j < 0 || k < 0 || i >= N || j >= N || k >= N) return false;  // ghost layer
    return lab[((int64_t)i * N + j) * N + k] & DPM_LBL_MPLUS;
}
__device__ __forceinline__ bool in_minus(const uint8_t *lab, int N, int i, int j, int k) {
    if (i < 0 || j < 0 || k < 0 || i >= N || j >= N || k >= N) return false;
    return !(lab[((int64_t)i * N + j) * N + k] & DPM_LBL_MPLUS);
}

// gamma_in / gamma_ex bits, and the margin check (flag[0] = 1 on violation).
__global__ void k_gamma(int N, uint8_t *labels, int *flag) {
    int64_t n3 = (int64_t)N * N * N;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n3;
         p += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(p % N), j = (int)((p / N) % N), i = (int)(p / ((int64_t)N * N));
        uint8_t l = labels[p];
        bool plus = l & DPM_LBL_MPLUS;
        uint8_t add = 0;
        if (plus) {
            if (i < 2 || j < 2 || k < 2 || i > N - 3 || j > N - 3 || k > N - 3) flag[0] = 1;
            if (in_minus(labels, N, i - 1, j, k) || in_minus(labels, N, i + 1, j, k) ||
                in_minus(labels, N, i, j - 1, k) || in_minus(labels, N, i, j + 1, k) ||
                in_minus(labels, N, i, j, k - 1) || in_minus(labels, N, i, j, k + 1))
                add = DPM_LBL_GIN;
        } else {
            if (in_plus(labels, N, i - 1, j, k) || in_plus(labels, N, i + 1, j, k) ||
                in_plus(labels, N, i, j - 1, k) || in_plus(labels, N, i, j + 1, k) ||
                in_plus(labels, N, i, j, k - 1) || in_plus(labels, N, i, j, k + 1))
                add = DPM_LBL_GEX;
        }
        labels[p] = l | add;  // only bits 1-2 change; neighbours read bit 0 only
    }
}

__device__ __forceinline__ bool in_gamma(const uint8_t *lab, int N, int i, int j, int k) {
    if (i < 0 || j < 0 || k < 0 || i >= N || j >= N || k >= N) return false;
    return lab[((int64_t)i * N + j) * N + k] & (DPM_LBL_GIN | DPM_LBL_GEX);
}

__global__ void k_shell(int N, uint8_t *labels) {
    int64_t n3 = (int64_t)N * N * N;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n3;
         p += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(p % N), j = (int)((p / N) % N), i = (int)(p / ((int64_t)N * N));
        uint8_t l = labels[p];
        if (l & DPM_LBL_MPLUS) continue;
        bool sh = (l & DPM_LBL_GEX) || in_gamma(labels, N, i - 1, j, k) ||
                  in_gamma(labels, N, i + 1, j, k) || in_gamma(labels, N, i, j - 1, k) ||
                  in_gamma(labels, N, i, j + 1, k) || in_gamma(labels, N, i, j, k - 1) ||
                  in_gamma(labels, N, i, j, k + 1);
        if (sh) labels[p] = l | DPM_LBL_SHELL;
    }
}

__device__ __forceinline__ void preds(uint8_t l, int out[kLists]) {
    out[0] = (l & DPM_LBL_MPLUS) ? 1 : 0;
    out[1] = (l & DPM_LBL_GIN) ? 1 : 0;
    out[2] = (l & DPM_LBL_GEX) ? 1 : 0;
    out[3] = (l & (DPM_LBL_GIN | DPM_LBL_GEX)) ? 1 : 0;
    out[4] = (l & DPM_LBL_SHELL) ? 1 : 0;
}

__global__ void k_count(int64_t n3, const uint8_t *labels, int *blk_counts) {
    int64_t base = (int64_t)blockIdx.x * kChunk;
    int c[kLists] = {0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < kChunk; t += kThreads) {
        int64_t p = base + t;
        if (p < n3) {
            int q[kLists];
            preds(labels[p], q);
#pragma unroll
            for (int l = 0; l < kLists; ++l) c[l] += q[l];
        }
    }
    __shared__ int red[kLists][kThreads / 32];
#pragma unroll
    for (int l = 0; l < kLists; ++l) {
        int v = c[l];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[l][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < kLists) {
        int v = 0;
        for (int w = 0; w < kThreads / 32; ++w) v += red[threadIdx.x][w];
        blk_counts[blockIdx.x * kLists + threadIdx.x] = v;
    }
}

// Exclusive scan of the per-block counts (one block; nblk small).
__global__ void k_scan(int nblk, const int *blk_counts, int *blk_off, long long *totals) {
    using Scan = cub::BlockScan<long long, kThreads>;
    __shared__ typename Scan::TempStorage tmp;
    __shared__ long long carry;
    for (int l = 0; l < kLists; ++l) {
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (int base = 0; base < nblk; base += kThreads) {
            int b = base + threadIdx.x;
            long long v = (b < nblk) ? blk_counts[b * kLists + l] : 0;
            long long ex, agg;
            Scan(tmp).ExclusiveSum(v, ex, agg);
            if (b < nblk) blk_off[b * kLists + l] = (int)(carry + ex);
            __syncthreads();
            if (threadIdx.x == 0) carry += agg;
            __syncthreads();
        }
        if (threadIdx.x == 0) totals[l] = carry;
        __syncthreads();
    }
}

__global__ void k_scatter(int64_t n3, const uint8_t *labels, const int *blk_off, int *l_gin,
                          int *l_gex, int *l_gamma, int *l_shell) {
    using Scan = cub::BlockScan<int, kThreads>;
    __shared__ typename Scan::TempStorage tmp;
    __shared__ int run[kLists];
    if (threadIdx.x < kLists) run[threadIdx.x] = blk_off[blockIdx.x * kLists + threadIdx.x];
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kChunk;
    for (int t0 = 0; t0 < kChunk; t0 += kThreads) {
        int64_t p = base + t0 + threadIdx.x;
        int q[kLists] = {0, 0, 0, 0, 0};
        if (p < n3) preds(labels[p], q);
        int *dst[kLists] = {nullptr, l_gin, l_gex, l_gamma, l_shell};
        for (int l = 1; l < kLists; ++l) {
            int ex, agg;
            Scan(tmp).ExclusiveSum(q[l], ex, agg);
            if (q[l]) dst[l][run[l] + ex] = (int)p;
            __syncthreads();
            if (threadIdx.x == 0) run[l] += agg;
            __syncthreads();
        }
    }
}

__global__ void k_gmap(int n, const int *list, int *gmap) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        gmap[list[e]] = e;
}

__global__ void k_lookup(int n, const int *list, const int *gmap, int *pos) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        pos[e] = gmap[list[e]];
}

__global__ void k_shell_nb(int n, int N, const int *shell, const int *gmap, int *nb) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        int p = shell[e];
        int k = p % N, j = (p / N) % N, i = p / (N * N);
        int o[8];
        o[0] = gmap[p];
        o[1] = i > 0 ? gmap[p - N * N] : -1;
        o[2] = i < N - 1 ? gmap[p + N * N] : -1;
        o[3] = j > 0 ? gmap[p - N] : -1;
        o[4] = j < N - 1 ? gmap[p + N] : -1;
        o[5] = k > 0 ? gmap[p - 1] : -1;
        o[6] = k < N - 1 ? gmap[p + 1] : -1;
        o[7] = -1;
#pragma unroll
        for (int t = 0; t < 8; ++t) nb[e * 8 + t] = o[t];
    }
}

// rp[r] = first entry of `list` with linear index >= r*N, r = 0..nrows.
__global__ void k_rowptr(int nrows, int N, int n, const int *list, int *rp) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r <= nrows; r += gridDim.x * blockDim.x) {
        long long key = (long long)r * N;
        int a = 0, b = n;
        while (a < b) {
            int m = (a + b) >> 1;
            if ((long long)list[m] < key) a = m + 1; else b = m;
        }
        rp[r] = a;
    }
}

int grid_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    return (int)(b < 65535 * 16 ? (b > 0 ? b : 1) : 65535 * 16);
}

}  // namespace

int classify_labels(const dpm_geom &g, int N, double lo, double hi, uint8_t *labels, cudaStream_t s) {
    if (g.kind != 0 && g.kind != 1) { set_error("classify_labels: sphere or ellipsoid only"); return DPM_EINVAL; }
    const double h = (hi - lo) / (double)(N + 1);
    const double ax = g.axes[0], ay = g.kind == 1 ? g.axes[1] : g.axes[0], az = g.kind == 1 ? g.axes[2] : g.axes[0];
    const int64_t n3 = (int64_t)N * N * N;
    DevBuf flag;  // the margin check does not apply here
    DPM_RET(flag.alloc(sizeof(int)));
    k_inside<<<grid_for(n3), kThreads, 0, s>>>(N, lo, h, g.center[0], g.center[1], g.center[2], ax, ay, az,
                                               g.kind, 0.0, 0.0, labels);
    DPM_LAUNCHED();
    k_gamma<<<grid_for(n3), kThreads, 0, s>>>(N, labels, flag.as<int>());
    DPM_LAUNCHED();
    DPM_CUDA(cudaStreamSynchronize(s));
    return DPM_OK;
}

int build_grid_index(const dpm_geom &g, int N, double lo, double hi, GridIndex &gi,
                     cudaStream_t s) {
    if (N < 6 || N > 1024) { set_error("N=%d out of range [6,1024]", N); return DPM_EINVAL; }
    if (!(hi > lo)) { set_error("need lo < hi"); return DPM_EINVAL; }
    if (g.kind < 0 || g.kind > 4) { set_error("geometry kind %d unknown", g.kind); return DPM_EINVAL; }
    if (g.kind >= 3 && !(g.axes[1] > 0)) { set_error("kinds 3/4: need axes[1] > 0"); return DPM_EINVAL; }
    double ax = g.axes[0], ay = g.kind == 1 ? g.axes[1] : g.axes[0],
           az = g.kind == 1 ? g.axes[2] : g.axes[0];
    if (!(ax > 0 && ay > 0 && az > 0)) { set_error("axes must be positive"); return DPM_EINVAL; }
    if (g.kind == 2 && !(g.axes[1] > 0 && g.axes[1] < g.axes[0])) {
        set_error("shell radii: need 0 < inner (axes[1]) < outer (axes[0])");
        return DPM_EINVAL;
    }
    gi.N = N; gi.lo = lo; gi.hi = hi;
    gi.h = (hi - lo) / (double)(N + 1);
    int64_t n3 = (int64_t)N * N * N;
    DPM_RET(gi.labels.alloc(n3));
    DevBuf flag;
    DPM_RET(flag.alloc(sizeof(int)));
    DPM_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    uint8_t *lab = gi.labels.as<uint8_t>();
    k_inside<<<grid_for(n3), kThreads, 0, s>>>(N, lo, gi.h, g.center[0], g.center[1], g.center[2],
                                               ax, ay, az, g.kind, g.axes[1], g.kind >= 3 ? g.axes[2] : 0.0,
                                               lab);
    DPM_LAUNCHED();
    k_gamma<<<grid_for(n3), kThreads, 0, s>>>(N, lab, flag.as<int>());
    DPM_LAUNCHED();
    k_shell<<<grid_for(n3), kThreads, 0, s>>>(N, lab);
    DPM_LAUNCHED();
    int nblk = (int)((n3 + kChunk - 1) / kChunk);
    DevBuf cnt, off, tot;
    DPM_RET(cnt.alloc(sizeof(int) * nblk * kLists));
    DPM_RET(off.alloc(sizeof(int) * nblk * kLists));
    DPM_RET(tot.alloc(sizeof(long long) * kLists));
    k_count<<<nblk, kThreads, 0, s>>>(n3, lab, cnt.as<int>());
    DPM_LAUNCHED();
    k_scan<<<1, kThreads, 0, s>>>(nblk, cnt.as<int>(), off.as<int>(), tot.as<long long>());
    DPM_LAUNCHED();
    long long h_tot[kLists];
    int h_flag = 0;
    DPM_CUDA(cudaMemcpyAsync(h_tot, tot.p, sizeof(h_tot), cudaMemcpyDeviceToHost, s));
    DPM_CUDA(cudaMemcpyAsync(&h_flag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    DPM_CUDA(cudaStreamSynchronize(s));
    gi.n_mplus = h_tot[0]; gi.n_gin = h_tot[1]; gi.n_gex = h_tot[2];
    gi.n_gamma = h_tot[3]; gi.n_shell = h_tot[4];
    if (gi.n_mplus == 0) { set_error("no node of the grid lies inside the domain"); return DPM_EINVAL; }
    if (h_flag) {
        set_error("the domain reaches within 2 nodes of a face of the cube [%g,%g]^3 (N=%d)", lo, hi, N);
        return DPM_EINVAL;
    }
    DPM_RET(gi.gin.alloc(sizeof(int) * gi.n_gin));
    DPM_RET(gi.gex.alloc(sizeof(int) * gi.n_gex));
    DPM_RET(gi.gamma.alloc(sizeof(int) * gi.n_gamma));
    DPM_RET(gi.shell.alloc(sizeof(int) * gi.n_shell));
    k_scatter<<<nblk, kThreads, 0, s>>>(n3, lab, off.as<int>(), gi.gin.as<int>(),
                                       gi.gex.as<int>(), gi.gamma.as<int>(), gi.shell.as<int>());
    DPM_LAUNCHED();
    DevBuf gmap;
    DPM_RET(gmap.alloc(sizeof(int) * n3));
    DPM_CUDA(cudaMemsetAsync(gmap.p, 0xff, sizeof(int) * n3, s));
    k_gmap<<<grid_for(gi.n_gamma), kThreads, 0, s>>>((int)gi.n_gamma, gi.gamma.as<int>(),
                                                    gmap.as<int>());
    DPM_LAUNCHED();
    DPM_RET(gi.gin_pos.alloc(sizeof(int) * gi.n_gin));
    DPM_RET(gi.gex_pos.alloc(sizeof(int) * gi.n_gex));
    k_lookup<<<grid_for(gi.n_gin), kThreads, 0, s>>>((int)gi.n_gin, gi.gin.as<int>(),
                                                    gmap.as<int>(), gi.gin_pos.as<int>());
    DPM_LAUNCHED();
    k_lookup<<<grid_for(gi.n_gex), kThreads, 0, s>>>((int)gi.n_gex, gi.gex.as<int>(),
                                                    gmap.as<int>(), gi.gex_pos.as<int>());
    DPM_LAUNCHED();
    DPM_RET(gi.shell_nb.alloc(sizeof(int) * 8 * gi.n_shell));
    k_shell_nb<<<grid_for(gi.n_shell), kThreads, 0, s>>>((int)gi.n_shell, N, gi.shell.as<int>(),
                                                        gmap.as<int>(), gi.shell_nb.as<int>());
    DPM_LAUNCHED();
    int nrows = N * N;
    DPM_RET(gi.rp_gin.alloc(sizeof(int) * (nrows + 1)));
    DPM_RET(gi.rp_shell.alloc(sizeof(int) * (nrows + 1)));
    k_rowptr<<<grid_for(nrows + 1), kThreads, 0, s>>>(nrows, N, (int)gi.n_gin, gi.gin.as<int>(),
                                                     gi.rp_gin.as<int>());
    DPM_LAUNCHED();
    k_rowptr<<<grid_for(nrows + 1), kThreads, 0, s>>>(nrows, N, (int)gi.n_shell,
                                                     gi.shell.as<int>(), gi.rp_shell.as<int>());
    DPM_LAUNCHED();
    DPM_CUDA(cudaStreamSynchronize(s));  // temporaries (gmap, counts) are freed on return
    return DPM_OK;
}

}  // namespace dpm
