// Internal declarations shared by the CUDA translation units of libdpm.
#pragma once

#include <cuda_runtime.h>
#include <mutex>
#include <vector>
#include <stdint.h>
#include <stddef.h>

#include "../../include/dpm.h"

namespace dpm {

void set_error(const char *fmt, ...);
const char *cuda_err(cudaError_t e);

// A failed runtime call also records its error as the thread's last error;
// it is cleared here (a non-sticky error) so that the next launch check does
// not report it again.
#define DPM_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            (void)cudaGetLastError();                                                   \
            dpm::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                           __FILE__, __LINE__);                                         \
            return e_ == cudaErrorMemoryAllocation ? DPM_ENOMEM : DPM_ECUDA;            \
        }                                                                               \
    } while (0)

// Kernel-launch bookkeeping: every launch is followed by DPM_LAUNCHED() (it
// counts the launch and checks the launch error).  A launch whose device time
// should be attributable sits inside a DPM_PROF("name", stream) scope, which
// records CUDA events around it while profiling is enabled.
void count_launch();
int prof_begin(const char *name, cudaStream_t s);   // -1 when profiling is off
void prof_end(int rec, cudaStream_t s);

#define DPM_LAUNCHED()              \
    do {                            \
        dpm::count_launch();        \
        DPM_CUDA(cudaGetLastError()); \
    } while (0)

struct ProfScope {
    int rec;
    cudaStream_t s;
    ProfScope(const char *name, cudaStream_t st) : rec(prof_begin(name, st)), s(st) {}
    ~ProfScope() { prof_end(rec, s); }
};
#define DPM_PROF(name, stream) dpm::ProfScope prof_scope_##__LINE__(name, stream)

#define DPM_RET(expr)                        \
    do {                                     \
        int r_ = (expr);                     \
        if (r_ != DPM_OK) return r_;         \
    } while (0)

// A set-up step that must run once on every device: kernel attributes such
// as the dynamic shared memory limit belong to each device's context, so a
// process that uses several devices configures each of them.  `run()` calls
// `f()` the first time it sees the current device (devices 0..63; any other
// device runs `f()` on every call) and remembers it only when `f()` succeeds.
struct PerDeviceOnce {
    std::mutex mu;
    uint64_t done = 0;
    template <class F> int run(F f) {
        int dev = 0;
        DPM_CUDA(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && ((done >> dev) & 1ull)) return DPM_OK;
        const int r = f();
        if (r == DPM_OK && dev >= 0 && dev < 64) done |= 1ull << dev;
        return r;
    }
};

// Raise `func`'s dynamic shared-memory limit to the most the current device
// allows a CTA beside the kernel's own static shared memory.
inline int raise_dynamic_smem_limit(const void *func) {
    int dev = 0, optin = 0;
    DPM_CUDA(cudaGetDevice(&dev));
    DPM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    DPM_CUDA(cudaFuncGetAttributes(&fa, func));
    DPM_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - (int)fa.sharedSizeBytes));
    return DPM_OK;
}

// Owning device buffer.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    int alloc(size_t n) {  // exact size; contents undefined
        if (n == bytes && p) return DPM_OK;
        release();
        if (n == 0) return DPM_OK;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error("cudaMalloc(%zu bytes) failed: %s", n, cudaGetErrorString(e));
            return DPM_ENOMEM;
        }
        bytes = n;
        return DPM_OK;
    }
    int reserve(size_t n) {  // at least n bytes
        if (n <= bytes && p) return DPM_OK;
        return alloc(n);
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// ---------------------------------------------------------------------------
// Point sets and the index structures built from them (Definition 2.1).
// ---------------------------------------------------------------------------
struct GridIndex {
    int N = 0;
    double lo = 0, hi = 0, h = 0;
    int64_t n_mplus = 0, n_gin = 0, n_gex = 0, n_gamma = 0, n_shell = 0;
    DevBuf labels;     // uint8[N^3]
    DevBuf gin;        // int32[n_gin]   ascending linear indices of gamma_in
    DevBuf gex;        // int32[n_gex]
    DevBuf gamma;      // int32[n_gamma] ascending (union of the two)
    DevBuf shell;      // int32[n_shell] ascending, nodes with DPM_LBL_SHELL
    DevBuf shell_nb;   // int32[n_shell][8]: gamma positions of (self,-x,+x,-y,+y,-z,+z), -1 if none
    DevBuf rp_gin;     // int32[N^2+1]: gamma_in entries of grid row r=(i*N+j)
    DevBuf rp_shell;   // int32[N^2+1]
    DevBuf gin_pos;    // int32[n_gin]: position of each gamma_in node in `gamma`
    DevBuf gex_pos;    // int32[n_gex]
};

// Classify and build every list.  Synchronises `s` (the sizes come back to
// the host).  Returns DPM_EINVAL on a geometry the library rejects.
int build_grid_index(const dpm_geom &g, int N, double lo, double hi, GridIndex &gi,
                     cudaStream_t s);
// Labels only (M^+, gamma_in, gamma_ex bits) of a sphere or ellipsoid on an
// N^3 grid, without the margin check: the domain may leave the cube (used for
// the Gamma / Z split of the domain decomposition).  Synchronises `s`.
int classify_labels(const dpm_geom &g, int N, double lo, double hi, uint8_t *labels, cudaStream_t s);

// ---------------------------------------------------------------------------
// Gamma geometry and spherical harmonics (Definition 2.6, eq. spectral_approximation_sd)
// ---------------------------------------------------------------------------
struct GammaGeom {
    int K = 0, nsh = 0;
    DevBuf foot;     // double[n_gamma][3]
    DevBuf normal;   // double[n_gamma][3]
    DevBuf dist;     // double[n_gamma]
    DevBuf phi;      // double[n_gamma][nsh] real orthonormal SH at the foot point
    DevBuf phi32;    // float copy of phi (FP32 paths' extension), built on demand
};
int build_gamma_geom(const dpm_geom &g, const GridIndex &gi, int K, GammaGeom &gg,
                     cudaStream_t s);

// ---------------------------------------------------------------------------
// Auxiliary-problem solver (Definition 2.4)
// ---------------------------------------------------------------------------
template <class T> struct ApRhs {
    const T *f;      // dense N^3 source (scaled by fscale), or null
    const T *dens;   // density on gamma [n_gamma] (potential part), or null
    T *out_dense;    // dense N^3 output, or null
    T *out_trace;    // trace on gamma_in [n_gin], or null
    int cond;        // 1: skipped unless *cond_flag != 0
    int pad_;
    // tensor-core N = 128 path, a density that does not change between solves:
    // pre[e] = {v(self), sum of v over the 6 neighbours} on the shell, so the
    // shell right-hand side is a streaming pass instead of a gather (null: from dens)
    const float2 *pre = nullptr;
};

struct ApParams {
    int N = 0, B = 0;
    double h = 0, sigma = 0, fscale = 1;
    const double *sigma_dev = nullptr;   // overrides sigma when set
    const double *fscale_dev = nullptr;  // overrides fscale when set
    const int *cond_flag = nullptr;      // see ApRhs::cond
    int mask_f = 1;    // 1: f is applied on M^+ only (else everywhere)
    int mask_out = 1;  // 1: out_dense is zero off N^+ (else the raw AP solution)
    // index data (required when mask_f/mask_out or any dens/out_trace is used)
    const uint8_t *labels = nullptr;
    const int *shell = nullptr, *shell_nb = nullptr, *rp_shell = nullptr;
    const int *gin = nullptr, *rp_gin = nullptr;
    int64_t n_shell = 0;       // shell size (the tensor-core solver stages L[v] on it)
    float *scratch = nullptr;  // tensor-core solver: B * n_shell floats
};

// Fills the index members of p from gi.
void ap_params_from_index(ApParams &p, const GridIndex &gi);

// work: B*N^3 elements of T.  rhs: device array of B descriptors.
template <class T>
int ap_solve_simt(const ApParams &p, const ApRhs<T> *rhs_dev, T *work, cudaStream_t s);
// Right-hand sides of grids of different N (problem prob_of[b] for rhs[b]) in
// one set of five SIMT launches; work / items_dev grown on demand.
template <class T>
int ap_solve_simt_group(const std::vector<ApParams> &probs, const std::vector<ApRhs<T>> &rhs,
                        const std::vector<int> &prob_of, DevBuf &work, DevBuf &items_dev, cudaStream_t s);
// The same group prepared once for replays (a device-resident time step):
// ap_group_bytes is the workspace the group needs; ap_group_build writes its
// launch descriptors to items_dev (cubes at `work`, which must hold that many
// bytes and stay in place), synchronising s; ap_group_launch runs the five
// passes on them without any host copy or allocation (capturable).
template <class T>
size_t ap_group_bytes(const std::vector<ApParams> &probs, const std::vector<int> &prob_of);
template <class T>
int ap_group_build(const std::vector<ApParams> &probs, const std::vector<ApRhs<T>> &rhs,
                   const std::vector<int> &prob_of, void *work, DevBuf &items_dev, int *maxN, int *minN,
                   cudaStream_t s);
template <class T>
int ap_group_launch(const void *items_dev, int B, int maxN, int minN, cudaStream_t s);
// Tuned SIMT tile width for (N, FP64?, B) on the current device, 0 if none.
int simt_tile_choice(int N, int f64, int B);
// pre[c][e] for the ncol densities dens + c ng (see ApRhs::pre)
int tc_shell_pre(int64_t n_shell, const int *shell_nb, const float *dens, int64_t ng, int ncol, float2 *pre,
                 cudaStream_t s);
int ap_solve_tc(const ApParams &p, const ApRhs<float> *rhs_dev, float *work, cudaStream_t s);
// N = 256: six out-of-place passes; work holds 2 B N^3 floats.
int ap_solve_tc256(const ApParams &p, const ApRhs<float> *rhs_dev, float *work, cudaStream_t s);
int tc256_status_check();
// N = 256: FFT-style FP32 solver (fold + Rader convolutions), three passes in
// place; work holds B N^3 floats.
int ap_solve_fft256(const ApParams &p, const ApRhs<float> *rhs_dev, float *work, cudaStream_t s);
bool fft_supported(int N);
// AP workspace cubes per right-hand side (the N = 256 tensor-core solver ping-pongs).
inline size_t ap_cubes_per_rhs(int prec, int N) { return (prec == 2 && N == 256) ? 2 : 1; }
// floats of ApParams::scratch the tensor-core solver needs for B right-hand sides
size_t tc_scratch_elems(const ApParams &p, int B);
bool tc_supported(int N);
// DPM_ETIMEOUT if a bounded MMA wait of the tensor-core kernels expired
// since the last check (synchronous; call where the stream is synchronised).
int tc_status_check();

// DST-I fold tables (device, per N and type), built on first use.
template <class T> const T *dst_fold_table(int N);

// ---------------------------------------------------------------------------
// FP64 least squares (Householder QR, resident R^{-1} Q^T)
// ---------------------------------------------------------------------------
struct LsqFactor {
    // kEquilibrated64: FP64 Gram of A, equilibrated (D G D), FP64 Cholesky: for
    // matrices whose kappa^2 is beyond FP32 (kMixed) but whose column scales differ.
    enum Method { kMixed = 0, kCholeskyQR = 1, kHouseholder = 2, kEquilibrated64 = 3 };
    int m = 0, n = 0;
    int method = kMixed;
    bool equilibrated = false;
    bool rinv32 = false;  // R^{-1} stored in FP32 (the in-shared-memory mixed factor)
    const float *A32 = nullptr;  // FP32 copy of A kept by that factor (in X), else null
    const float *A32s = nullptr; // FP32 copy of A D kept by the mixed factor for larger n (in X)
    // A as two floats, A = Ahi + Alo to ~2^-48 (mixed factor, n > 168): the FP32
    // paths' residual b - A C in two-float arithmetic instead of FP64
    const float *Ahi = nullptr, *Alo = nullptr;
    DevBuf A2;
    // Optional block structure of a block-banded A (stored dense, zeros outside
    // the blocks), set by lsq_set_band: int[2n] the row interval [lo, hi) of
    // each column's nonzeros, then int[2 ceil(m/32)] the column interval of
    // each 32-row group.  Empty: A is treated as dense.
    DevBuf band;
    DevBuf A;      // double[m*n] column-major (Householder overwrites it)
    DevBuf tau;    // double[n] Householder scalars
    DevBuf X;      // scratch of the Gram / Cholesky factorisation
    DevBuf work;   // A copy (Householder only), R, solve scratch
};
// The unfactored A the solves read: a copy for Householder QR (which
// overwrites A), A itself for the Cholesky-based methods.
inline const double *lsq_matrix(const LsqFactor &f) {
    return f.method == LsqFactor::kHouseholder ? f.work.as<double>() : f.A.as<double>();
}
// ---------------------------------------------------------------------------
// Domain decomposition, Case 1 (Section 3): kernels in dd.cu
// ---------------------------------------------------------------------------
int dd_surface_flags(int64_t n, const double *foot, const double c[3], double r_mid, uint8_t *surf,
                     cudaStream_t s);
template <class T>
int dd_columns(int64_t n, int64_t m, int nsh, int nz, int ng, int ncol_l, const double *phi,
               const double *dist, const uint8_t *surf, const int *gin_pos, T *psi, double *psi_in,
               cudaStream_t s);
template <class T>
int dd_assemble(int64_t m1, int64_t m2, int nzc, int ncol, const double *psi_in1, const T *tr1,
                const double *psi_in2, const T *tr2, double *A, cudaStream_t s);
template <class T>
int dd_extend(int64_t n, int nsh, int nz, int ng, const double *phi, const double *dist,
              const uint8_t *surf, const double *C, int ldc, const double *neumann, T *dens, int ldd,
              int nr, int clamp, cudaStream_t s);
template <class T>
int dd_neumann_density(int64_t n, const double *dist, const uint8_t *surf, const double *gn, T *v,
                       cudaStream_t s);
template <class T>
int dd_rhs(int64_t m1, int64_t m2, const T *tr_p1, const T *tr_p2, const T *v, const int *gin_pos2,
           const T *tr_v2, T *b, cudaStream_t s);

// Domain decomposition, Case 2 (dd2.cu): the Gamma / Z split of a grid
// boundary (flags bit 0 Gamma, bit 1 Z), distances to both spheres, the cosines
// of the polar angles, the foot points; zonal harmonics; column densities and
// row values; the stacked BEP; right-hand sides; Neumann density; extension.
int dd2_split(const GridIndex &gi, const uint8_t *lab_o, const uint8_t *lab_b, const double c0[3], double R,
              const double cz[3], double rz, uint8_t *flags, double *dG, double *dZ, double *cosG,
              double *cosZ, double *footG, double *footZ, cudaStream_t s);
int dd2_zonal(int64_t n, int M, const double *x, double a, double b, double *Y, cudaStream_t s);
template <class T>
int dd2_columns(int64_t n, int64_t m, int MZ, int MG, int GS, const uint8_t *flags, const double *dG,
                const double *dZ, const double *YG, const double *YZ, const int *row_e, const uint8_t *row_s,
                T *psi, double *own, cudaStream_t s);
template <class T>
int dd2_assemble(int64_t m1, int64_t m2, int ncol, const double *own1, const T *tr1, int64_t g1,
                 const int *ri1, const double *own2, const T *tr2, int64_t g2, const int *ri2, double *A,
                 cudaStream_t s);
template <class T>
int dd2_rhs(int64_t m, const int *row_i, const int *row_e, const uint8_t *row_s, const T *trp,
            const double *vG, const T *trv, T *b, cudaStream_t s);
template <class T>
int dd2_neumann(int64_t n, const uint8_t *flags, const double *dG, const double *gn, double *vG, T *veff,
                cudaStream_t s);
template <class T>
int dd2_extend(int64_t n, int MZ, int MG, int GS, const uint8_t *flags, const double *dG, const double *dZ,
               const double *YG, const double *YZ, const double *C, int ldc, const double *gn, T *dens,
               int ldd, int nr, int clamp, cudaStream_t s);
int dd2_init_foot(int64_t n, const uint8_t *flags, const double *footG, const double *footZ, double *foot,
                  cudaStream_t s);

// Layered domain decomposition (ddml.cu): the column layout by sphere
// (1..L, L = Gamma): columns [off[m-1], off[m]) of n[m-1] harmonics per term.
constexpr int kMlMax = 16;
struct MlColumns {
    int L;
    int off[kMlMax + 1];
    int n[kMlMax];
};
int ml_sphere_flags(int64_t n, const double *foot, const double c[3], double r_mid, int m_in, int ball,
                    uint8_t *sphere, cudaStream_t s);
template <class T>
int ml_columns(int64_t n, int64_t m, int nsh, const MlColumns &cm, int ncl, const int *cols, const uint8_t *sphere,
               const double *dist, const double *phi, const int *gin_pos, T *psi, double *psi_in, cudaStream_t s);
template <class T>
int ml_assemble(int64_t m, int ncl, int64_t mtot, int64_t row0, const int *cols, const double *psi_in, const T *trace,
                double *A, cudaStream_t s);
// u on the grid boundary of one sub-domain (spheres mlo..mhi) from the
// coefficients; FP32 sums from the transposed FP32 table phit when given (T =
// float), else FP64 from phi.
template <class T>
int ml_extend(int64_t n, int nsh, const MlColumns &cm, const uint8_t *sphere, const double *dist, const double *phi,
              const float *phit, int mlo, int mhi, const double *C, int ldc, const double *gn, T *dens, int ldd,
              int nr, int clamp, cudaStream_t s);
template <class T>
int ml_neumann(int64_t n, int L, const uint8_t *sphere, const double *dist, const double *gn, T *v, cudaStream_t s);
template <class T>
int ml_rhs(int64_t m, const T *trp, const T *v, const int *gin_pos, const T *trv, T *b, cudaStream_t s);

// Scalars of the device-resident PKS step (Step 3's dt and the time).
struct StepScalars {
    double dt, sigma, t, dt_prev;
    long long step;
    int rebuilt, bad;  // bad: a non-positive / non-finite dt was replaced by dt_max
    // Step 4b on the device: rebuild_now = need_build or dt < dt_prev (set with
    // dt); need_build = no factor for the current sigma yet (cleared by a rebuild)
    int rebuild_now, need_build;
};
int pks_step_dt(const unsigned long long *gmax, double h, double chi, double dt_max, int mode,
                StepScalars *sc, cudaStream_t s);
// Expected relative loss of a tensor-core AP solve to the round-toward-zero
// FP32 accumulation of tcgen05.mma.  A truncating step loses on average half
// an ulp of the running sum; for sums whose significand m in [1, 2) is
// log-uniformly distributed the mean of ulp/|sum| = 2^-23/m is 2^-23/(2 ln 2),
// so a step loses 2^-25/ln 2 (4.3e-8) of the sum.  A folded transform issues
// its main term (hi*hi, after the small cross terms) in S = K/16 steps whose
// partial sums are about k/S of the result (k = 1..S, equally sized K slices):
// (S + 1)/2 full-size steps' worth.  A solve is six transforms (three axes,
// forward and inverse).  S = 4 (N = 128): 6.45e-7; S = 8 (N = 256): 1.16e-6.
constexpr double tc_rz_bias(int S) { return 6.0 * 0.5 * (S + 1) * 0x1p-25 / 0.69314718055994531; }
// rebuilt < 0: the step's rebuild flag is the device's rebuild_now.
int pks_step_end(StepScalars *sc, int rebuilt, cudaStream_t s);
// The condition of a conditional graph node (captured steps): rebuild_now.
int pks_set_rebuild_cond(cudaGraphConditionalHandle h, const StepScalars *sc, cudaStream_t s);
// dt from the CFL bounds of several grids (the decomposed loops): the smallest
// over the grids and axes, as pks_step_dt takes it for one grid.
constexpr int kMaxStepGrids = 16;
struct StepGrids {
    int n = 0;
    const unsigned long long *gmax[kMaxStepGrids] = {};
    double h[kMaxStepGrids] = {};
};
int pks_step_dt_grids(const StepGrids &g, double chi, double dt_max, int mode, StepScalars *sc, cudaStream_t s);

constexpr int kLsqMaxRhs = 64;  // right-hand sides per lsq_apply call
// Factor A (already in f.A, m x n col-major): R with R^T R = A^T A.
int lsq_factor(LsqFactor &f, const int *cond_flag, cudaStream_t s);
// The same without the host read of the pivot status (no synchronisation;
// for stream capture): lsq_status reads it later.
int lsq_factor_async(LsqFactor &f, cudaStream_t s);
// Declare A block-banded: block b holds rows [row0[b], row0[b+1]) and is
// nonzero only in columns [c0[b], c1[b]); every other entry of A is zero.
// The products with A and A^T then skip the zero blocks (same results: only
// exact zero terms are left out).  Synchronises s (host arrays are staged).
int lsq_set_band(LsqFactor &f, const std::vector<int64_t> &row0, const std::vector<int> &c0,
                 const std::vector<int> &c1, cudaStream_t s);
int lsq_status(const LsqFactor &f, cudaStream_t s);
// C[r][0..n) = X b[r] for nr right-hand sides (b: [nr][m] in T, C: [nr][n] double)
template <class T>
int lsq_apply(const LsqFactor &f, const T *b, int ldb, double *C, int nr, cudaStream_t s);

// ---------------------------------------------------------------------------
// BEP assembly helpers
// ---------------------------------------------------------------------------
// psi[k][g] (T) for k < ncol: phi or (d^2/2) phi.  Also psi_in (double) at gamma_in.
template <class T>
int make_basis_densities(const GammaGeom &gg, const GridIndex &gi, int beta, T *psi,
                         double *psi_in, cudaStream_t s);
// A[k*m + r] = psi_in[k*m + r] - trace[k*m + r]
template <class T>
int assemble_bep(const double *psi_in, const T *trace, double *A, int64_t m, int ncol,
                 const int *cond_flag, cudaStream_t s);
// u_gamma[r][g] = sum phi C0 + d*gN + beta (d^2/2) sum phi C2 (+ clamp)
// gg.phi32 = the FP32 table of the harmonics, transposed ([nu][node]), built
// once on demand (the FP32 paths' extensions read it).
int gamma_phi32(const GammaGeom &gg, int64_t n_gamma, cudaStream_t s);
template <class T>
int extend_density(const GammaGeom &gg, int64_t n_gamma, int beta, const double *C, int ldc,
                   const double *neumann, T *dens, int ldd, int nr, int clamp, cudaStream_t s);

}  // namespace dpm

struct dpm_ctx {
    int device = 0;
    int num_sms = 0;
    dpm::DevBuf work;      // AP workspace
    dpm::DevBuf rhs_desc;  // descriptor scratch
    dpm::DevBuf scratch;   // small scalars
};
