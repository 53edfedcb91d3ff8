// C ABI of libdpm (include/dpm.h): argument checking, handle lifetime, and
// the sequencing of the kernels for the DPM steps.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include "dpm_internal.cuh"

namespace dpm {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

// ---- launch counter and event profiler --------------------------------------
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};
std::mutex g_pmu;
std::vector<ProfRec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::atomic<bool> g_prof{false};

cudaEvent_t pool_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

int prof_begin(const char *name, cudaStream_t s) {
    if (!g_prof.load(std::memory_order_relaxed)) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return -1;  // graph replays are timed as a whole
    std::lock_guard<std::mutex> lk(g_pmu);
    cudaEvent_t a = pool_event(), b = pool_event();
    if (!a || !b) return -1;
    cudaEventRecord(a, s);
    g_recs.push_back({name, a, b});
    return (int)g_recs.size() - 1;
}

void prof_end(int rec, cudaStream_t s) {
    if (rec < 0) return;
    std::lock_guard<std::mutex> lk(g_pmu);
    if (rec < (int)g_recs.size()) cudaEventRecord(g_recs[rec].b, s);
}

template <class T>
int pks_flux(int, double, double, double, const double *, const uint8_t *, const T *, const T *,
             T *, T *, cudaStream_t);
template <class T> int pks_cfl(int, const uint8_t *, const T *, unsigned long long *, cudaStream_t);
template <class T>
int pks_diag(int, double, double, const uint8_t *, const T *, const T *, double *, double *,
             cudaStream_t, const double *origin = nullptr);
int pks_diag_blocks(int N);
template <class T>
int pks_init(const GridIndex &, const GammaGeom &, const dpm_gaussian &, const dpm_gaussian &,
             T *, T *, cudaStream_t);
template <class T> int mask_copy(int, const uint8_t *, const T *, T *, cudaStream_t);

namespace {

size_t elem_size(int prec) { return prec == DPM_PREC_FP64 ? sizeof(double) : sizeof(float); }

bool prec_ok(int prec) {
    return prec == DPM_PREC_FP32 || prec == DPM_PREC_FP64 || prec == DPM_PREC_TC32 || prec == DPM_PREC_FFT32;
}

// Run B right-hand sides through the AP solver in chunks that fit the
// workspace (`work`, grown on demand up to kWorkCap bytes).
constexpr size_t kWorkCap = size_t(8) << 30;

template <class T>
int run_ap_dev(int prec, ApParams p, const ApRhs<T> *desc_dev, int B, DevBuf &work, cudaStream_t s);

template <class T>
int run_ap(int prec, ApParams p, const std::vector<ApRhs<T>> &rhs, DevBuf &work, DevBuf &desc,
           cudaStream_t s) {
    const int B = (int)rhs.size();
    if (B == 0) return DPM_OK;
    const size_t cube = (size_t)p.N * p.N * p.N * sizeof(T) * ap_cubes_per_rhs(prec, p.N);
    size_t cb = std::max<size_t>(1, std::min<size_t>(B, kWorkCap / cube));
    size_t extra = 0;  // tensor-core solver: staged shell right-hand sides after the cubes
    if (prec == DPM_PREC_TC32) extra = tc_scratch_elems(p, (int)cb) * sizeof(float);
    if (prec == DPM_PREC_TC32 || prec == DPM_PREC_FFT32) {
        // the tensor-core passes stage dense inputs with bulk copies, the FFT-style
        // passes read them as float4 (both 16-byte aligned)
        for (const auto &r : rhs)
            if (reinterpret_cast<uintptr_t>(r.f) & 15) {
                set_error("%s AP solve: f must be 16-byte aligned", prec == DPM_PREC_TC32 ? "tensor-core" : "FFT-style");
                return DPM_EINVAL;
            }
    }
    DPM_RET(work.reserve(cb * cube + extra));
    DPM_RET(desc.reserve(sizeof(ApRhs<T>) * B));
    DPM_CUDA(cudaMemcpyAsync(desc.p, rhs.data(), sizeof(ApRhs<T>) * B, cudaMemcpyHostToDevice, s));
    // The copy above is from pageable memory: it has been staged when it
    // returns, so `rhs` may go out of scope afterwards.
    return run_ap_dev<T>(prec, p, desc.as<ApRhs<T>>(), B, work, s);
}

// The same with the descriptors already in device memory and the workspace
// already sized (no allocation, no host copy: usable under stream capture).
template <class T>
int run_ap_dev(int prec, ApParams p, const ApRhs<T> *desc_dev, int B, DevBuf &work, cudaStream_t s) {
    if (B == 0) return DPM_OK;
    const size_t cube = (size_t)p.N * p.N * p.N * sizeof(T) * ap_cubes_per_rhs(prec, p.N);
    size_t cb = std::max<size_t>(1, std::min<size_t>(B, kWorkCap / cube));
    size_t extra = 0;
    if (prec == DPM_PREC_TC32) extra = tc_scratch_elems(p, (int)cb) * sizeof(float);
    if (work.bytes < cb * cube + extra) { set_error("AP workspace not sized for %d right-hand sides", B); return DPM_EINVAL; }
    if (prec == DPM_PREC_TC32) p.scratch = reinterpret_cast<float *>(static_cast<char *>(work.p) + cb * cube);
    for (int b0 = 0; b0 < B; b0 += (int)cb) {
        ApParams q = p;
        q.B = std::min<int>((int)cb, B - b0);
        const ApRhs<T> *d = desc_dev + b0;
        if (prec == DPM_PREC_TC32 || prec == DPM_PREC_FFT32) {
            if constexpr (sizeof(T) == 4) {
                if (prec == DPM_PREC_TC32) DPM_RET(ap_solve_tc(q, d, work.as<float>(), s));
                else DPM_RET(ap_solve_fft256(q, d, work.as<float>(), s));
            } else {
                set_error("tensor-core and FFT-style solves are FP32-storage only");
                return DPM_EINVAL;
            }
        } else {
            DPM_RET(ap_solve_simt<T>(q, d, work.as<T>(), s));
        }
    }
    return DPM_OK;
}

// Device-resident time steps replayed as a CUDA graph (the decomposed loops):
// the step's scalars (dt, sigma, t, step) live in `scal`; the first step runs
// uncaptured so that every workspace, table and tuned tile it needs exists, the
// second is captured on a private stream and instantiated, and every step after
// that is one graph launch.
struct GraphStepper {
    int on = 0;
    bool warm = false;
    DevBuf scal;  // StepScalars
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;
    cudaStream_t aux = nullptr;  // captures the bodies of conditional nodes
    long long gkernels = 0;  // kernel launches per replay
    GraphStepper() = default;
    GraphStepper(const GraphStepper &) = delete;
    GraphStepper &operator=(const GraphStepper &) = delete;
    ~GraphStepper() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (cap) cudaStreamDestroy(cap);
        if (aux) cudaStreamDestroy(aux);
    }
    StepScalars *sc() const { return scal.as<StepScalars>(); }
    int push(double t, double dt_prev, int64_t step, int rebuilt, int need_build, cudaStream_t s) {
        if (!scal.p) DPM_RET(scal.alloc(sizeof(StepScalars)));
        StepScalars h{};
        h.t = t;
        h.dt_prev = dt_prev;
        h.step = step;
        h.rebuilt = rebuilt;
        h.need_build = need_build;
        DPM_CUDA(cudaMemcpyAsync(scal.p, &h, sizeof(h), cudaMemcpyHostToDevice, s));
        DPM_CUDA(cudaStreamSynchronize(s));
        return DPM_OK;
    }
    int pull(double &t, double &dt_prev, int64_t &step, int &rebuilt, int *bad, cudaStream_t s) const {
        StepScalars h{};
        DPM_CUDA(cudaMemcpyAsync(&h, scal.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        DPM_CUDA(cudaStreamSynchronize(s));
        t = h.t;
        dt_prev = h.dt;
        step = h.step;
        rebuilt = h.rebuilt;
        if (bad) *bad = h.bad;
        return DPM_OK;
    }
    template <class F> int step(F &&dev_step, cudaStream_t s) {
        if (!gexec) {
            if (!warm) {
                DPM_RET(dev_step(s));
                warm = true;
                return DPM_OK;
            }
            if (!cap) DPM_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            DPM_CUDA(cudaStreamSynchronize(s));  // the capture stream records only
            cudaGraph_t g = nullptr;
            DPM_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
            const long long l0 = g_launches.load();
            const int r = dev_step(cap);
            const cudaError_t e = cudaStreamEndCapture(cap, &g);
            gkernels = g_launches.load() - l0;
            g_launches.fetch_sub(gkernels);  // counted when replayed
            if (r != DPM_OK) {
                if (g) cudaGraphDestroy(g);
                return r;
            }
            DPM_CUDA(e);
            const cudaError_t ie = cudaGraphInstantiate(&gexec, g, 0);
            cudaGraphDestroy(g);
            DPM_CUDA(ie);
        }
        DPM_CUDA(cudaGraphLaunch(gexec, s));
        g_launches.fetch_add(gkernels);
        return DPM_OK;
    }
    void stop() {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        warm = false;
        on = 0;
    }
};

// Step 4b inside a captured step: an if/else conditional graph node whose
// condition a kernel sets from sc->rebuild_now (dt decreased, or no factor for
// the current sigma yet); `yes` (the rebuild) and `no` are captured into its
// two bodies on `aux`.  Uncaptured (the warm-up step) `yes` runs: a rebuild at
// an unchanged sigma reproduces the factor it replaces, bit for bit.  The
// launch count of a replay is taken with both bodies (an upper bound).
template <class Y, class N>
int step_branch(const StepScalars *sc, cudaStream_t s, cudaStream_t &aux, Y &&yes, N &&no) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    DPM_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &graph, &deps, nullptr, &nd));
    if (st != cudaStreamCaptureStatusActive) return yes(s);
    cudaGraphConditionalHandle h;
    DPM_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 0, 0));
    DPM_RET(pks_set_rebuild_cond(h, sc, s));
    DPM_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &graph, &deps, nullptr, &nd));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 2;
    cudaGraphNode_t node = nullptr;
    DPM_CUDA(cudaGraphAddNode(&node, graph, deps, nullptr, nd, &cp));
    if (!aux) DPM_CUDA(cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
        DPM_CUDA(cudaStreamBeginCaptureToGraph(aux, cp.conditional.phGraph_out[b], nullptr, nullptr, 0,
                                               cudaStreamCaptureModeRelaxed));
        const int r = b == 0 ? yes(aux) : no(aux);
        cudaGraph_t body = nullptr;
        const cudaError_t e = cudaStreamEndCapture(aux, &body);
        DPM_RET(r);
        DPM_CUDA(e);
    }
    DPM_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return DPM_OK;
}

// The batched solves of a decomposed device-resident step, prepared once: per
// batch, the SIMT grids' right-hand sides as one group (descriptors in
// `items`, cubes in the shared group workspace) and every other grid's
// descriptors on its own (run_ap_dev on the grid's workspace).
struct PreparedBatch {
    DevBuf items;
    int B = 0, maxN = 0, minN = 0;
    DevBuf desc[DPM_ML_MAX];
    int nb[DPM_ML_MAX] = {};
};

// One sub-domain's solver: precision, parameters (sigma read from the device)
// and workspace.
struct SubSolve {
    int prec = 0;
    ApParams p;
    DevBuf *work = nullptr;
};

inline bool simt_prec(int prec) { return prec == DPM_PREC_FP32 || prec == DPM_PREC_FP64; }

// rhs[b][l]: batch b's right-hand sides of sub-domain l.  The group workspace is
// sized for the largest batch before any descriptor is built (they point into
// it); synchronises s.
template <class T>
int prepare_batches(const std::vector<SubSolve> &subs, const std::vector<std::vector<std::vector<ApRhs<T>>>> &rhs,
                    PreparedBatch *bt, DevBuf &gwork, cudaStream_t s) {
    const int L = (int)subs.size(), nbat = (int)rhs.size();
    if (L > DPM_ML_MAX) { set_error("prepared solves: at most %d sub-domains", DPM_ML_MAX); return DPM_EINVAL; }
    std::vector<ApParams> prm(L);
    for (int l = 0; l < L; ++l) prm[l] = subs[l].p;
    std::vector<std::vector<ApRhs<T>>> gr(nbat);
    std::vector<std::vector<int>> gof(nbat);
    size_t gbytes = 0;
    for (int b = 0; b < nbat; ++b) {
        for (int l = 0; l < L; ++l)
            if (simt_prec(subs[l].prec))
                for (auto &e : rhs[b][l]) {
                    gr[b].push_back(e);
                    gof[b].push_back(l);
                }
        gbytes = std::max(gbytes, ap_group_bytes<T>(prm, gof[b]));
    }
    DPM_RET(gwork.reserve(std::max<size_t>(gbytes, 16)));
    for (int b = 0; b < nbat; ++b) {
        PreparedBatch &pb = bt[b];
        pb.B = (int)gr[b].size();
        DPM_RET(ap_group_build<T>(prm, gr[b], gof[b], gwork.p, pb.items, &pb.maxN, &pb.minN, s));
        for (int l = 0; l < L; ++l) {
            pb.nb[l] = 0;
            if (simt_prec(subs[l].prec) || rhs[b][l].empty()) continue;
            const int B = (int)rhs[b][l].size();
            const int N = prm[l].N;
            const size_t cube = (size_t)N * N * N * sizeof(T) * ap_cubes_per_rhs(subs[l].prec, N);
            const size_t cb = std::max<size_t>(1, std::min<size_t>(B, kWorkCap / cube));
            size_t extra = 0;
            if (subs[l].prec == DPM_PREC_TC32) extra = tc_scratch_elems(prm[l], (int)cb) * sizeof(float);
            DPM_RET(subs[l].work->reserve(cb * cube + extra));
            DPM_RET(pb.desc[l].reserve(sizeof(ApRhs<T>) * B));
            DPM_CUDA(cudaMemcpyAsync(pb.desc[l].p, rhs[b][l].data(), sizeof(ApRhs<T>) * B, cudaMemcpyHostToDevice, s));
            pb.nb[l] = B;
        }
    }
    DPM_CUDA(cudaStreamSynchronize(s));  // the host descriptor vectors go out of scope
    return DPM_OK;
}

template <class T> int run_prepared(const PreparedBatch &pb, const std::vector<SubSolve> &subs, cudaStream_t s) {
    DPM_RET(ap_group_launch<T>(pb.items.p, pb.B, pb.maxN, pb.minN, s));
    for (int l = 0; l < (int)subs.size(); ++l)
        if (pb.nb[l]) DPM_RET(run_ap_dev<T>(subs[l].prec, subs[l].p, pb.desc[l].as<ApRhs<T>>(), pb.nb[l], *subs[l].work, s));
    return DPM_OK;
}

template <class T>
__global__ void k_neumann_rhs(int m, const T *trace0, const T *dgn, const int *gin_pos,
                              const T *trace1, T *b) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    // b = Tr G f - Tr_{gamma_in} (I - P)(d g_N)
    b[r] = trace0[r] - (dgn[gin_pos[r]] - trace1[r]);
}

}  // namespace
}  // namespace dpm

using namespace dpm;

// ---------------------------------------------------------------------------
struct dpm_bep {
    dpm_ctx *ctx = nullptr;
    dpm_geom geom{};
    int N = 0, K = 0, beta = 0, ncol = 0, prec = 0;
    double lo = 0, hi = 0, sigma = 0;
    GridIndex gi;
    GammaGeom gg;
    DevBuf psi;     // T[ncol][n_gamma]
    DevBuf shpre;   // float2[ncol][n_shell]: shell pairs of the basis columns (tensor cores, N = 128)
    DevBuf psi_in;  // double[ncol][n_gin]
    DevBuf trace;   // T[ncol + 4][n_gin]
    DevBuf dens;    // T[4][n_gamma]
    DevBuf coef;    // double[4][ncol]
    DevBuf zero;    // double[ncol] zeros
    DevBuf desc;
    DevBuf work;
    LsqFactor lsq;
    DevBuf btrace, bdens, bcoef;  // batched-solve buffers
    bool factored = false;
};

struct dpm_pks {
    dpm_ctx *ctx = nullptr;
    dpm_pks_params prm{};
    dpm_bep bep;
    DevBuf rho, c, frho, fc;
    DevBuf gmax;       // 3 non-negative doubles as uint64 bit patterns
    DevBuf diag_part;  // double[nblk][6]
    DevBuf diag_out;   // double[6]
    double t = 0, dt_prev = 0;
    int64_t step = 0;
    int last_rebuilt = 0;
    // device-resident step replayed as a CUDA graph (dpm_pks_set_graph)
    int graph_on = 0;
    bool dev_warm = false;
    DevBuf scal;                     // StepScalars
    DevBuf desc_rb, desc_green;      // ApRhs: ncol BEP columns + 2 particular; 2 Green's
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;      // capture stream
    cudaStream_t aux = nullptr;      // captures the bodies of the Step 4b conditional node
    int64_t gkernels = 0;            // kernel nodes per replay
    ~dpm_pks() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (cap) cudaStreamDestroy(cap);
        if (aux) cudaStreamDestroy(aux);
    }
};

extern "C" const char *dpm_last_error(void) { return g_err; }

extern "C" int64_t dpm_launch_count(void) { return (int64_t)g_launches.load(); }

extern "C" int dpm_profile_enable(int on) {
    g_prof.store(on != 0);
    return DPM_OK;
}

extern "C" int dpm_profile_read(const char *name, double *total_ms, int64_t *launches) {
    std::lock_guard<std::mutex> lk(g_pmu);
    double tot = 0.0;
    int64_t n = 0;
    for (auto &r : g_recs) {
        if (name && name[0] && !strstr(r.name, name)) continue;
        DPM_CUDA(cudaEventSynchronize(r.b));
        float ms = 0.f;
        DPM_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        tot += ms;
        ++n;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = n;
    return DPM_OK;
}

extern "C" int dpm_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_pmu);
    for (auto &r : g_recs) {
        cudaEventSynchronize(r.b);
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    return DPM_OK;
}

extern "C" int dpm_ctx_create(int device, dpm_ctx **out) {
    if (!out) { set_error("out is NULL"); return DPM_EINVAL; }
    *out = nullptr;
    int n = 0;
    DPM_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) { set_error("device %d not present (%d devices)", device, n); return DPM_EINVAL; }
    DPM_CUDA(cudaSetDevice(device));
    dpm_ctx *c = new (std::nothrow) dpm_ctx();
    if (!c) { set_error("out of host memory"); return DPM_ENOMEM; }
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    *out = c;
    return DPM_OK;
}

extern "C" int dpm_ctx_destroy(dpm_ctx *ctx) {
    delete ctx;
    return DPM_OK;
}

extern "C" int dpm_classify(dpm_ctx *ctx, const dpm_geom *geom, int N, double lo, double hi,
                            uint8_t *labels, int32_t *gin_idx, int64_t gin_cap, int32_t *gex_idx,
                            int64_t gex_cap, int64_t *n_gin, int64_t *n_gex, cudaStream_t s) {
    if (!ctx || !geom) { set_error("ctx/geom is NULL"); return DPM_EINVAL; }
    GridIndex gi;
    DPM_RET(build_grid_index(*geom, N, lo, hi, gi, s));
    if (n_gin) *n_gin = gi.n_gin;
    if (n_gex) *n_gex = gi.n_gex;
    if (gin_idx && gin_cap < gi.n_gin) { set_error("gin_cap %lld < |gamma_in| %lld", (long long)gin_cap, (long long)gi.n_gin); return DPM_EINVAL; }
    if (gex_idx && gex_cap < gi.n_gex) { set_error("gex_cap %lld < |gamma_ex| %lld", (long long)gex_cap, (long long)gi.n_gex); return DPM_EINVAL; }
    size_t n3 = (size_t)N * N * N;
    if (labels) DPM_CUDA(cudaMemcpyAsync(labels, gi.labels.p, n3, cudaMemcpyDeviceToDevice, s));
    if (gin_idx && gi.n_gin)
        DPM_CUDA(cudaMemcpyAsync(gin_idx, gi.gin.p, sizeof(int) * gi.n_gin, cudaMemcpyDeviceToDevice, s));
    if (gex_idx && gi.n_gex)
        DPM_CUDA(cudaMemcpyAsync(gex_idx, gi.gex.p, sizeof(int) * gi.n_gex, cudaMemcpyDeviceToDevice, s));
    DPM_CUDA(cudaStreamSynchronize(s));  // gi's buffers are freed on return
    return DPM_OK;
}

extern "C" int dpm_aux_solve_batched(dpm_ctx *ctx, int N, double h, double sigma, int B,
                                     const void *q, void *u, int precision, cudaStream_t s) {
    if (!ctx || !q || !u) { set_error("ctx/q/u is NULL"); return DPM_EINVAL; }
    if (!prec_ok(precision)) { set_error("unknown precision %d", precision); return DPM_EINVAL; }
    if (N < 2 || N > 256 || B < 1 || !(h > 0) || !(sigma >= 0)) {
        set_error("aux solve: need 2<=N<=256, B>=1, h>0, sigma>=0 (N=%d B=%d h=%g sigma=%g)", N, B, h, sigma);
        return DPM_EINVAL;
    }
    if (precision == DPM_PREC_TC32 && !tc_supported(N)) {
        set_error("tensor-core solve does not support N=%d", N);
        return DPM_EUNSUPPORTED;
    }
    if (precision == DPM_PREC_FFT32 && !fft_supported(N)) {
        set_error("FFT-style solve does not support N=%d", N);
        return DPM_EUNSUPPORTED;
    }
    ApParams p;
    p.N = N;
    p.h = h;
    p.sigma = sigma;
    p.mask_f = 0;
    p.mask_out = 0;
    size_t n3 = (size_t)N * N * N;
    if (precision == DPM_PREC_FP64) {
        std::vector<ApRhs<double>> r(B);
        for (int b = 0; b < B; ++b)
            r[b] = {static_cast<const double *>(q) + b * n3, nullptr,
                    static_cast<double *>(u) + b * n3, nullptr, 0, 0};
        return run_ap<double>(precision, p, r, ctx->work, ctx->rhs_desc, s);
    }
    std::vector<ApRhs<float>> r(B);
    for (int b = 0; b < B; ++b)
        r[b] = {static_cast<const float *>(q) + b * n3, nullptr, static_cast<float *>(u) + b * n3,
                nullptr, 0, 0};
    return run_ap<float>(precision, p, r, ctx->work, ctx->rhs_desc, s);
}

// ---------------------------------------------------------------------------
// BEP
// ---------------------------------------------------------------------------
namespace {

template <class T> int bep_setup(dpm_bep *b, cudaStream_t s) {
    DPM_RET(build_gamma_geom(b->geom, b->gi, b->K, b->gg, s));
    const int64_t ng = b->gi.n_gamma, m = b->gi.n_gin;
    DPM_RET(b->psi.alloc(sizeof(T) * b->ncol * ng));
    DPM_RET(b->psi_in.alloc(sizeof(double) * b->ncol * m));
    DPM_RET(make_basis_densities<T>(b->gg, b->gi, b->beta, b->psi.as<T>(), b->psi_in.as<double>(), s));
    DPM_RET(b->trace.alloc(sizeof(T) * (b->ncol + 4) * m));
    DPM_RET(b->dens.alloc(sizeof(T) * 4 * ng));
    DPM_RET(b->coef.alloc(sizeof(double) * 4 * b->ncol));
    DPM_RET(b->zero.alloc(sizeof(double) * b->ncol));
    DPM_CUDA(cudaMemsetAsync(b->zero.p, 0, sizeof(double) * b->ncol, s));
    b->lsq.m = (int)m;
    b->lsq.n = b->ncol;
    DPM_RET(b->lsq.A.alloc(sizeof(double) * m * b->ncol));
    if (m < b->ncol) {
        set_error("|gamma_in| = %lld is smaller than the %d BEP columns: refine the grid or lower K",
                  (long long)m, b->ncol);
        return DPM_EINVAL;
    }
    return DPM_OK;
}

ApParams base_params(const dpm_bep *b, double sigma) {
    ApParams p;
    p.N = b->N;
    p.h = b->gi.h;
    p.sigma = sigma;
    ap_params_from_index(p, b->gi);
    return p;
}

// Columns of eq. BEP_recast plus `extra` right-hand sides in the same batch.
// Shell pairs of the basis columns for the tensor-core N = 128 solver (the
// basis densities depend on the geometry only), computed on first use; null
// where they do not apply (the solver then gathers q from the densities).
template <class T>
int bep_shell_pre(dpm_bep *b, const float2 **out, cudaStream_t s) {
    *out = nullptr;
    if constexpr (sizeof(T) == sizeof(float)) {
        if (b->prec != DPM_PREC_TC32 || b->N != 128 || b->gi.n_shell <= 0) return DPM_OK;
        if (!b->shpre.p) {
            DPM_RET(b->shpre.alloc(sizeof(float2) * (size_t)b->ncol * b->gi.n_shell));
            DPM_RET(tc_shell_pre(b->gi.n_shell, b->gi.shell_nb.as<int>(), b->psi.as<float>(), b->gi.n_gamma,
                                 b->ncol, b->shpre.as<float2>(), s));
        }
        *out = b->shpre.as<float2>();
    }
    return DPM_OK;
}

template <class T>
int bep_assemble(dpm_bep *b, double sigma, std::vector<ApRhs<T>> extra, double fscale,
                 cudaStream_t s) {
    const int64_t ng = b->gi.n_gamma, m = b->gi.n_gin;
    std::vector<ApRhs<T>> rhs;
    rhs.reserve(b->ncol + extra.size());
    const float2 *pre = nullptr;
    DPM_RET(bep_shell_pre<T>(b, &pre, s));
    for (int k = 0; k < b->ncol; ++k)
        rhs.push_back({nullptr, b->psi.as<T>() + k * ng, nullptr, b->trace.as<T>() + k * m, 0, 0,
                       pre ? pre + (size_t)k * b->gi.n_shell : nullptr});
    for (auto &e : extra) rhs.push_back(e);
    ApParams p = base_params(b, sigma);
    p.fscale = fscale;
    DPM_RET(run_ap<T>(b->prec, p, rhs, b->work, b->desc, s));
    DPM_RET(assemble_bep<T>(b->psi_in.as<double>(), b->trace.as<T>(), b->lsq.A.as<double>(), m,
                            b->ncol, nullptr, s));
    DPM_RET(lsq_factor(b->lsq, nullptr, s));
    b->sigma = sigma;
    b->factored = true;
    return DPM_OK;
}

template <class T>
int bep_solve(dpm_bep *b, const void *fv, const double *neumann, void *uv, double *coeffs,
              cudaStream_t s) {
    const T *f = static_cast<const T *>(fv);
    T *u = static_cast<T *>(uv);
    const int64_t ng = b->gi.n_gamma, m = b->gi.n_gin;
    T *tr0 = b->trace.as<T>() + (int64_t)b->ncol * m;
    T *tr1 = tr0 + m;
    T *bvec = tr1 + m;
    T *dens0 = b->dens.as<T>(), *dens1 = dens0 + ng;
    double *C = b->coef.as<double>();
    std::vector<ApRhs<T>> rhs;
    rhs.push_back({f, nullptr, nullptr, tr0, 0, 0});
    if (neumann) {
        // density d*g_N (the known term of the extension)
        DPM_RET(extend_density<T>(b->gg, ng, 0, b->zero.as<double>(), 0, neumann, dens1, (int)ng, 1, 0, s));
        rhs.push_back({nullptr, dens1, nullptr, tr1, 0, 0});
    }
    ApParams p = base_params(b, b->sigma);
    DPM_RET(run_ap<T>(b->prec, p, rhs, b->work, b->desc, s));
    const T *bb = tr0;
    if (neumann) {
        k_neumann_rhs<T><<<(unsigned)((m + 255) / 256), 256, 0, s>>>((int)m, tr0, dens1,
                                                                    b->gi.gin_pos.as<int>(), tr1, bvec);
        DPM_LAUNCHED();
        bb = bvec;
    }
    DPM_RET(lsq_apply<T>(b->lsq, bb, (int)m, C, 1, s));
    DPM_RET(extend_density<T>(b->gg, ng, b->beta, C, b->ncol, neumann, dens0, (int)ng, 1, 0, s));
    std::vector<ApRhs<T>> rhs2;
    rhs2.push_back({f, dens0, u, nullptr, 0, 0});
    DPM_RET(run_ap<T>(b->prec, p, rhs2, b->work, b->desc, s));
    if (coeffs) DPM_CUDA(cudaMemcpyAsync(coeffs, C, sizeof(double) * b->ncol, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

template <class T>
int bep_solve_batched(dpm_bep *b, int nreq, const void *const *fv, const double *const *neumann,
                      void *const *uv, double *const *coeffs, cudaStream_t s) {
    const int64_t ng = b->gi.n_gamma, m = b->gi.n_gin;
    // per-batch buffers: traces [2*nreq][m], b vectors [nreq][m], densities [2*nreq][ng], C [nreq][ncol]
    const size_t need_tr = sizeof(T) * (size_t)(3 * nreq) * m;
    const size_t need_dn = sizeof(T) * (size_t)(2 * nreq) * ng;
    const size_t need_c = sizeof(double) * (size_t)nreq * b->ncol;
    DPM_RET(b->btrace.reserve(need_tr));
    DPM_RET(b->bdens.reserve(need_dn));
    DPM_RET(b->bcoef.reserve(need_c));
    T *tr = b->btrace.as<T>();           // [r]: particular trace, [nreq + r]: Neumann trace
    T *bv = tr + (size_t)2 * nreq * m;   // [r]: least-squares right-hand side
    T *dn = b->bdens.as<T>();            // [r]: u_gamma, [nreq + r]: d g_N
    double *C = b->bcoef.as<double>();
    std::vector<ApRhs<T>> rhs;
    for (int r = 0; r < nreq; ++r)
        rhs.push_back({static_cast<const T *>(fv[r]), nullptr, nullptr, tr + (size_t)r * m, 0, 0});
    for (int r = 0; r < nreq; ++r) {
        if (neumann && neumann[r]) {
            T *d1 = dn + (size_t)(nreq + r) * ng;
            DPM_RET(extend_density<T>(b->gg, ng, 0, b->zero.as<double>(), 0, neumann[r], d1, (int)ng, 1, 0, s));
            rhs.push_back({nullptr, d1, nullptr, tr + (size_t)(nreq + r) * m, 0, 0});
        }
    }
    ApParams p = base_params(b, b->sigma);
    DPM_RET(run_ap<T>(b->prec, p, rhs, b->work, b->desc, s));
    for (int r = 0; r < nreq; ++r) {
        T *dst = bv + (size_t)r * m;
        if (neumann && neumann[r]) {
            k_neumann_rhs<T><<<(unsigned)((m + 255) / 256), 256, 0, s>>>(
                (int)m, tr + (size_t)r * m, dn + (size_t)(nreq + r) * ng, b->gi.gin_pos.as<int>(),
                tr + (size_t)(nreq + r) * m, dst);
            DPM_LAUNCHED();
        } else {
            DPM_CUDA(cudaMemcpyAsync(dst, tr + (size_t)r * m, sizeof(T) * m, cudaMemcpyDeviceToDevice, s));
        }
    }
    DPM_RET(lsq_apply<T>(b->lsq, bv, (int)m, C, nreq, s));
    std::vector<ApRhs<T>> green;
    for (int r = 0; r < nreq; ++r) {
        T *d0 = dn + (size_t)r * ng;
        DPM_RET(extend_density<T>(b->gg, ng, b->beta, C + (size_t)r * b->ncol, b->ncol,
                                  neumann ? neumann[r] : nullptr, d0, (int)ng, 1, 0, s));
        green.push_back({static_cast<const T *>(fv[r]), d0, static_cast<T *>(uv[r]), nullptr, 0, 0});
    }
    DPM_RET(run_ap<T>(b->prec, p, green, b->work, b->desc, s));
    for (int r = 0; r < nreq; ++r)
        if (coeffs && coeffs[r])
            DPM_CUDA(cudaMemcpyAsync(coeffs[r], C + (size_t)r * b->ncol, sizeof(double) * b->ncol,
                                     cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

int bep_init(dpm_bep *b, dpm_ctx *ctx, const dpm_geom *geom, int N, double lo, double hi, int K,
             int beta, int precision, cudaStream_t s) {
    if (!ctx || !geom) { set_error("ctx/geom is NULL"); return DPM_EINVAL; }
    if (!prec_ok(precision)) { set_error("unknown precision %d", precision); return DPM_EINVAL; }
    if (beta != 0 && beta != 1) { set_error("beta must be 0 or 1"); return DPM_EINVAL; }
    if (N > 256) { set_error("N=%d > 256 not supported by the AP solver", N); return DPM_EINVAL; }
    if (precision == DPM_PREC_TC32 && !tc_supported(N)) {
        set_error("tensor-core solve does not support N=%d", N);
        return DPM_EUNSUPPORTED;
    }
    if (precision == DPM_PREC_FFT32 && !fft_supported(N)) {
        set_error("FFT-style solve does not support N=%d", N);
        return DPM_EUNSUPPORTED;
    }
    b->ctx = ctx;
    b->geom = *geom;
    b->N = N; b->lo = lo; b->hi = hi; b->K = K; b->beta = beta; b->prec = precision;
    b->ncol = (beta + 1) * (K + 1) * (K + 1);
    DPM_RET(build_grid_index(*geom, N, lo, hi, b->gi, s));
    if (precision == DPM_PREC_FP64) return bep_setup<double>(b, s);
    return bep_setup<float>(b, s);
}

}  // namespace

extern "C" int dpm_bep_build(dpm_ctx *ctx, const dpm_geom *geom, int N, double lo, double hi,
                             double sigma, int K, int beta, int precision, dpm_bep **out,
                             cudaStream_t s) {
    if (!out) { set_error("out is NULL"); return DPM_EINVAL; }
    *out = nullptr;
    if (!(sigma > 0)) { set_error("sigma must be positive"); return DPM_EINVAL; }
    dpm_bep *b = new (std::nothrow) dpm_bep();
    if (!b) { set_error("out of host memory"); return DPM_ENOMEM; }
    int r = bep_init(b, ctx, geom, N, lo, hi, K, beta, precision, s);
    if (r == DPM_OK) {
        if (precision == DPM_PREC_FP64) r = bep_assemble<double>(b, sigma, {}, 1.0, s);
        else r = bep_assemble<float>(b, sigma, {}, 1.0, s);
    }
    if (r == DPM_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_error("BEP build: %s", cudaGetErrorString(e)); r = DPM_ECUDA; }
    }
    if (r == DPM_OK && precision == DPM_PREC_TC32) r = tc_status_check();
    if (r != DPM_OK) { delete b; return r; }
    *out = b;
    return DPM_OK;
}

extern "C" int dpm_bep_get_info(const dpm_bep *b, dpm_bep_info *info) {
    if (!b || !info) { set_error("bep/info is NULL"); return DPM_EINVAL; }
    info->N = b->N; info->lo = b->lo; info->hi = b->hi; info->h = b->gi.h; info->sigma = b->sigma;
    info->K = b->K; info->beta = b->beta; info->ncol = b->ncol; info->precision = b->prec;
    info->n_mplus = b->gi.n_mplus; info->n_gin = b->gi.n_gin; info->n_gex = b->gi.n_gex;
    info->n_gamma = b->gi.n_gamma; info->n_shell = b->gi.n_shell;
    return DPM_OK;
}

extern "C" int dpm_bep_matrix(const dpm_bep *b, double *A, cudaStream_t s) {
    if (!b || !A) { set_error("bep/A is NULL"); return DPM_EINVAL; }
    const double *A0 = lsq_matrix(b->lsq);  // unfactored
    DPM_CUDA(cudaMemcpyAsync(A, A0, sizeof(double) * b->gi.n_gin * b->ncol, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

extern "C" int dpm_bep_gamma_geometry(const dpm_bep *b, int32_t *gamma_idx, double *foot,
                                      double *normal, double *dist, cudaStream_t s) {
    if (!b) { set_error("bep is NULL"); return DPM_EINVAL; }
    int64_t n = b->gi.n_gamma;
    if (gamma_idx) DPM_CUDA(cudaMemcpyAsync(gamma_idx, b->gi.gamma.p, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    if (foot) DPM_CUDA(cudaMemcpyAsync(foot, b->gg.foot.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
    if (normal) DPM_CUDA(cudaMemcpyAsync(normal, b->gg.normal.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
    if (dist) DPM_CUDA(cudaMemcpyAsync(dist, b->gg.dist.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

extern "C" int dpm_bep_destroy(dpm_bep *b) {
    delete b;
    return DPM_OK;
}

extern "C" int dpm_solve(dpm_bep *b, const void *f, const double *neumann, void *u, double *coeffs,
                         cudaStream_t s) {
    if (!b || !f || !u) { set_error("bep/f/u is NULL"); return DPM_EINVAL; }
    if (b->prec == DPM_PREC_FP64) return bep_solve<double>(b, f, neumann, u, coeffs, s);
    return bep_solve<float>(b, f, neumann, u, coeffs, s);
}

extern "C" int dpm_solve_batched(dpm_bep *b, int nreq, const void *const *f,
                                 const double *const *neumann, void *const *u,
                                 double *const *coeffs, cudaStream_t s) {
    if (!b || !f || !u) { set_error("bep/f/u is NULL"); return DPM_EINVAL; }
    if (nreq < 1 || nreq > kLsqMaxRhs) { set_error("nreq=%d outside [1, %d]", nreq, kLsqMaxRhs); return DPM_EINVAL; }
    for (int r = 0; r < nreq; ++r)
        if (!f[r] || !u[r]) { set_error("request %d: f/u is NULL", r); return DPM_EINVAL; }
    if (b->prec == DPM_PREC_FP64) return bep_solve_batched<double>(b, nreq, f, neumann, u, coeffs, s);
    return bep_solve_batched<float>(b, nreq, f, neumann, u, coeffs, s);
}

namespace {
size_t bep_bytes(const dpm_bep &b) {
    const GridIndex &g = b.gi;
    const GammaGeom &q = b.gg;
    const LsqFactor &l = b.lsq;
    return g.labels.bytes + g.gin.bytes + g.gex.bytes + g.gamma.bytes + g.shell.bytes +
           g.shell_nb.bytes + g.rp_gin.bytes + g.rp_shell.bytes + g.gin_pos.bytes + g.gex_pos.bytes +
           q.foot.bytes + q.normal.bytes + q.dist.bytes + q.phi.bytes + q.phi32.bytes + l.A.bytes +
           l.tau.bytes + l.X.bytes + l.work.bytes + b.psi.bytes + b.shpre.bytes + b.psi_in.bytes + b.trace.bytes +
           b.dens.bytes + b.coef.bytes + b.zero.bytes + b.desc.bytes + b.work.bytes + b.btrace.bytes +
           b.bdens.bytes + b.bcoef.bytes;
}
}  // namespace

extern "C" int dpm_bep_device_bytes(const dpm_bep *b, int64_t *bytes) {
    if (!b || !bytes) { set_error("bep/bytes is NULL"); return DPM_EINVAL; }
    *bytes = (int64_t)bep_bytes(*b);
    return DPM_OK;
}

extern "C" int dpm_bep_reserve(dpm_bep *b, int max_nreq) {
    if (!b) { set_error("bep is NULL"); return DPM_EINVAL; }
    if (max_nreq < 1 || max_nreq > kLsqMaxRhs) {
        set_error("max_nreq=%d outside [1, %d]", max_nreq, kLsqMaxRhs);
        return DPM_EINVAL;
    }
    DPM_CUDA(cudaSetDevice(b->ctx->device));
    const size_t T = b->prec == DPM_PREC_FP64 ? sizeof(double) : sizeof(float);
    const int64_t ng = b->gi.n_gamma, m = b->gi.n_gin;
    const int B = 2 * max_nreq;  // particular + Neumann, or Green's formula
    const size_t cube = (size_t)b->N * b->N * b->N * T * ap_cubes_per_rhs(b->prec, b->N);
    const size_t cb = std::max<size_t>(1, std::min<size_t>(B, kWorkCap / cube));
    size_t extra = 0;
    if (b->prec == DPM_PREC_TC32) {
        ApParams p = base_params(b, b->sigma);
        extra = tc_scratch_elems(p, (int)cb) * sizeof(float);
    }
    // Every buffer a solve of up to max_nreq requests touches; the build
    // workspace shrinks to that size (an exact re-allocation).
    DPM_RET(b->work.alloc(cb * cube + extra));
    DPM_RET(b->desc.reserve(sizeof(ApRhs<double>) * B));
    DPM_RET(b->btrace.reserve(T * (size_t)(3 * max_nreq) * m));
    DPM_RET(b->bdens.reserve(T * (size_t)(2 * max_nreq) * ng));
    DPM_RET(b->bcoef.reserve(sizeof(double) * (size_t)max_nreq * b->ncol));
    if (b->prec != DPM_PREC_FP64) {
        // makes the FP32 extension table now rather than on the first solve
        DPM_RET(extend_density<float>(b->gg, ng, 0, b->zero.as<double>(), 0, nullptr,
                                      b->bdens.as<float>(), (int)ng, 1, 0, 0));
    }
    DPM_CUDA(cudaDeviceSynchronize());
    return DPM_OK;
}

// ---------------------------------------------------------------------------
// PKS
// ---------------------------------------------------------------------------
namespace {

template <class T> int pks_alloc(dpm_pks *k, cudaStream_t s) {
    size_t n3 = (size_t)k->prm.N * k->prm.N * k->prm.N;
    DPM_RET(k->rho.alloc(sizeof(T) * n3));
    DPM_RET(k->c.alloc(sizeof(T) * n3));
    DPM_RET(k->frho.alloc(sizeof(T) * n3));
    DPM_RET(k->fc.alloc(sizeof(T) * n3));
    DPM_RET(k->gmax.alloc(sizeof(unsigned long long) * 4));
    DPM_RET(k->diag_part.alloc(sizeof(double) * 6 * pks_diag_blocks(k->prm.N)));
    DPM_RET(k->diag_out.alloc(sizeof(double) * 8));
    DPM_CUDA(cudaMemsetAsync(k->diag_out.p, 0, sizeof(double) * 8, s));
    return DPM_OK;
}

template <class T> int pks_step_one(dpm_pks *k, cudaStream_t s) {
    dpm_bep *b = &k->bep;
    const dpm_pks_params &P = k->prm;
    const int N = P.N;
    const double h = b->gi.h;
    double dt = P.dt_max;
    if (P.dt_mode == 1) {
        double gm[3];
        DPM_RET(pks_cfl<T>(N, b->gi.labels.as<uint8_t>(), k->c.as<T>(), k->gmax.as<unsigned long long>(), s));
        DPM_CUDA(cudaMemcpyAsync(gm, k->gmax.p, sizeof(gm), cudaMemcpyDeviceToHost, s));
        DPM_CUDA(cudaStreamSynchronize(s));
        for (int ax = 0; ax < 3; ++ax) {
            const double g = gm[ax];
            double gmaxv = (double)g / h;  // max |grad_h c| along ax
            if (gmaxv > 0) dt = std::min(dt, h / (6.0 * P.chi * gmaxv));
        }
        if (k->step > 0) dt = std::min(dt, k->dt_prev);
    }
    if (!(dt > 0) || !std::isfinite(dt)) { set_error("time step is not positive/finite (dt=%g)", dt); return DPM_ENUMERIC; }
    const bool rebuild = !b->factored || P.rebuild || dt < k->dt_prev;
    const double sigma = 1.0 / dt;
    const int64_t m = b->gi.n_gin, ng = b->gi.n_gamma;
    T *frho = k->frho.as<T>(), *fc = k->fc.as<T>();
    DPM_RET(pks_flux<T>(N, h, P.chi, dt, nullptr, b->gi.labels.as<uint8_t>(), k->rho.as<T>(),
                        k->c.as<T>(), frho, fc, s));
    T *tr0 = b->trace.as<T>() + (int64_t)b->ncol * m;
    T *tr1 = tr0 + m;
    std::vector<ApRhs<T>> part = {{frho, nullptr, nullptr, tr0, 0, 0},
                                  {fc, nullptr, nullptr, tr1, 0, 0}};
    if (rebuild) {
        DPM_RET(bep_assemble<T>(b, sigma, part, sigma, s));
    } else {
        ApParams p = base_params(b, sigma);
        p.fscale = sigma;  // L_{h,dt} u = f  <=>  (1/dt - Lap_h) u = f/dt
        DPM_RET(run_ap<T>(b->prec, p, part, b->work, b->desc, s));
    }
    double *C = b->coef.as<double>();
    DPM_RET(lsq_apply<T>(b->lsq, tr0, (int)m, C, 2, s));
    T *dens = b->dens.as<T>();
    DPM_RET(extend_density<T>(b->gg, ng, b->beta, C, b->ncol, nullptr, dens, (int)ng, 2, P.clamp, s));
    std::vector<ApRhs<T>> green = {{frho, dens, k->rho.as<T>(), nullptr, 0, 0},
                                   {fc, dens + ng, k->c.as<T>(), nullptr, 0, 0}};
    ApParams p = base_params(b, sigma);
    p.fscale = sigma;
    DPM_RET(run_ap<T>(b->prec, p, green, b->work, b->desc, s));
    DPM_RET(pks_diag<T>(N, b->gi.lo, h, b->gi.labels.as<uint8_t>(), k->rho.as<T>(), k->c.as<T>(),
                        k->diag_part.as<double>(), k->diag_out.as<double>(), s));
    k->t += dt;
    k->dt_prev = dt;
    k->step += 1;
    k->last_rebuilt = rebuild ? 1 : 0;
    return DPM_OK;
}

// One PKS step with dt, sigma and the time kept on the device: no host
// synchronisation, no allocation and no host copy, so it can be captured in
// a CUDA graph.  Same kernels and arithmetic as pks_step_one.  The BEP is
// rebuilt on every step with rebuild = 1, never with a fixed dt (dt_mode 0),
// and with the CFL dt (dt_mode 1) when dt decreases (Step 4b): a conditional
// graph node that a kernel switches from the step's dt.
template <class T> int pks_step_dev(dpm_pks *k, cudaStream_t s) {
    dpm_bep *b = &k->bep;
    const dpm_pks_params &P = k->prm;
    const int N = P.N;
    const double h = b->gi.h;
    StepScalars *sc = k->scal.as<StepScalars>();
    const uint8_t *lab = b->gi.labels.as<uint8_t>();
    if (P.dt_mode == 1)
        DPM_RET(pks_cfl<T>(N, lab, k->c.as<T>(), k->gmax.as<unsigned long long>(), s));
    DPM_RET(pks_step_dt(k->gmax.as<unsigned long long>(), h, P.chi, P.dt_max, P.dt_mode, sc, s));
    T *frho = k->frho.as<T>(), *fc = k->fc.as<T>();
    DPM_RET(pks_flux<T>(N, h, P.chi, 0.0, &sc->dt, lab, k->rho.as<T>(), k->c.as<T>(), frho, fc, s));
    const bool cond = P.dt_mode == 1 && !P.rebuild;  // Step 4b decided on the device
    const bool rebuild = P.rebuild != 0;
    ApParams p = base_params(b, 0.0);
    p.sigma_dev = &sc->sigma;
    p.fscale_dev = &sc->sigma;  // L_{h,dt} u = f  <=>  (1/dt - Lap_h) u = f/dt
    const int64_t m = b->gi.n_gin, ng = b->gi.n_gamma;
    const ApRhs<T> *rb = k->desc_rb.as<ApRhs<T>>();
    auto with_rebuild = [&](cudaStream_t st) -> int {
        DPM_RET(run_ap_dev<T>(b->prec, p, rb, b->ncol + 2, b->work, st));
        DPM_RET(assemble_bep<T>(b->psi_in.as<double>(), b->trace.as<T>(), b->lsq.A.as<double>(), m,
                                b->ncol, nullptr, st));
        return lsq_factor_async(b->lsq, st);
    };
    auto particular_only = [&](cudaStream_t st) -> int {
        return run_ap_dev<T>(b->prec, p, rb + b->ncol, 2, b->work, st);
    };
    if (cond) DPM_RET(step_branch(sc, s, k->aux, with_rebuild, particular_only));
    else if (rebuild) DPM_RET(with_rebuild(s));
    else DPM_RET(particular_only(s));
    double *C = b->coef.as<double>();
    T *tr0 = b->trace.as<T>() + (int64_t)b->ncol * m;
    DPM_RET(lsq_apply<T>(b->lsq, tr0, (int)m, C, 2, s));
    T *dens = b->dens.as<T>();
    DPM_RET(extend_density<T>(b->gg, ng, b->beta, C, b->ncol, nullptr, dens, (int)ng, 2, P.clamp, s));
    DPM_RET(run_ap_dev<T>(b->prec, p, k->desc_green.as<ApRhs<T>>(), 2, b->work, s));
    DPM_RET(pks_diag<T>(N, b->gi.lo, h, lab, k->rho.as<T>(), k->c.as<T>(), k->diag_part.as<double>(),
                        k->diag_out.as<double>(), s));
    DPM_RET(pks_step_end(sc, cond ? -1 : (rebuild ? 1 : 0), s));
    return DPM_OK;
}

// Descriptors of the device step's three batched solves, uploaded once.
template <class T> int pks_dev_setup(dpm_pks *k, cudaStream_t s) {
    dpm_bep *b = &k->bep;
    const int64_t m = b->gi.n_gin, ng = b->gi.n_gamma;
    T *frho = k->frho.as<T>(), *fc = k->fc.as<T>();
    T *tr0 = b->trace.as<T>() + (int64_t)b->ncol * m, *tr1 = tr0 + m;
    T *dens = b->dens.as<T>();
    std::vector<ApRhs<T>> rb;
    const float2 *pre = nullptr;
    DPM_RET(bep_shell_pre<T>(b, &pre, s));
    for (int c = 0; c < b->ncol; ++c)
        rb.push_back({nullptr, b->psi.as<T>() + c * ng, nullptr, b->trace.as<T>() + c * m, 0, 0,
                      pre ? pre + (size_t)c * b->gi.n_shell : nullptr});
    rb.push_back({frho, nullptr, nullptr, tr0, 0, 0});
    rb.push_back({fc, nullptr, nullptr, tr1, 0, 0});
    std::vector<ApRhs<T>> gr = {{frho, dens, k->rho.as<T>(), nullptr, 0, 0},
                                {fc, dens + ng, k->c.as<T>(), nullptr, 0, 0}};
    DPM_RET(k->desc_rb.reserve(sizeof(ApRhs<T>) * rb.size()));
    DPM_RET(k->desc_green.reserve(sizeof(ApRhs<T>) * gr.size()));
    DPM_CUDA(cudaMemcpyAsync(k->desc_rb.p, rb.data(), sizeof(ApRhs<T>) * rb.size(), cudaMemcpyHostToDevice, s));
    DPM_CUDA(cudaMemcpyAsync(k->desc_green.p, gr.data(), sizeof(ApRhs<T>) * gr.size(), cudaMemcpyHostToDevice, s));
    // buffers every solve of the step touches (the eager step sizes them the same way)
    const size_t cube = (size_t)b->N * b->N * b->N * sizeof(T) * ap_cubes_per_rhs(b->prec, b->N);
    const int B = b->ncol + 2;
    const size_t cb = std::max<size_t>(1, std::min<size_t>(B, kWorkCap / cube));
    size_t extra = 0;
    if (b->prec == DPM_PREC_TC32) {
        ApParams p = base_params(b, 0.0);
        extra = tc_scratch_elems(p, (int)cb) * sizeof(float);
    }
    DPM_RET(b->work.reserve(cb * cube + extra));
    if (!k->scal.p) {
        DPM_RET(k->scal.alloc(sizeof(StepScalars)));
    }
    StepScalars h{};
    h.t = k->t;
    h.dt_prev = k->dt_prev;
    h.step = k->step;
    h.rebuilt = k->last_rebuilt;
    // a factor for sigma = 1/dt_prev exists: Step 4b rebuilds only when dt decreases
    h.need_build = (b->factored && k->dt_prev > 0 && b->sigma == 1.0 / k->dt_prev) ? 0 : 1;
    DPM_CUDA(cudaMemcpyAsync(k->scal.p, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    DPM_CUDA(cudaStreamSynchronize(s));
    return DPM_OK;
}

int pks_dev_step(dpm_pks *k, cudaStream_t s) {
    return k->prm.precision == DPM_PREC_FP64 ? pks_step_dev<double>(k, s) : pks_step_dev<float>(k, s);
}

// Host copy of the device step's scalars (after graph steps).
int pks_dev_pull(dpm_pks *k, cudaStream_t s, int *bad) {
    StepScalars h{};
    DPM_CUDA(cudaMemcpyAsync(&h, k->scal.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    DPM_CUDA(cudaStreamSynchronize(s));
    k->t = h.t;
    k->dt_prev = h.dt;
    k->step = h.step;
    k->last_rebuilt = h.rebuilt;
    if (bad) *bad = h.bad;
    return DPM_OK;
}

// Advance one step by replaying the captured graph (capturing it first).
int pks_graph_step(dpm_pks *k, cudaStream_t s) {
    if (!k->gexec) {
        if (!k->dev_warm) {
            // an uncaptured step sizes every workspace the captured one uses
            DPM_RET(pks_dev_step(k, s));
            k->dev_warm = true;
            return DPM_OK;
        }
        if (!k->cap) DPM_CUDA(cudaStreamCreateWithFlags(&k->cap, cudaStreamNonBlocking));
        // order the capture stream after the caller's work (capture records only)
        DPM_CUDA(cudaStreamSynchronize(s));
        cudaGraph_t g = nullptr;
        DPM_CUDA(cudaStreamBeginCapture(k->cap, cudaStreamCaptureModeRelaxed));
        const long long l0 = g_launches.load();
        const int r = pks_dev_step(k, k->cap);
        const cudaError_t e = cudaStreamEndCapture(k->cap, &g);
        k->gkernels = g_launches.load() - l0;
        g_launches.fetch_sub(k->gkernels);  // counted when replayed
        if (r != DPM_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        DPM_CUDA(e);
        const cudaError_t ie = cudaGraphInstantiate(&k->gexec, g, 0);
        cudaGraphDestroy(g);
        DPM_CUDA(ie);
    }
    DPM_CUDA(cudaGraphLaunch(k->gexec, s));
    g_launches.fetch_add(k->gkernels);
    return DPM_OK;
}

}  // namespace

extern "C" int dpm_pks_create(dpm_ctx *ctx, const dpm_pks_params *prm, const dpm_gaussian *rho0,
                              const dpm_gaussian *c0, dpm_pks **out, cudaStream_t s) {
    if (!out || !prm) { set_error("out/params is NULL"); return DPM_EINVAL; }
    *out = nullptr;
    if (!(prm->dt_max > 0) || !(prm->chi >= 0) || (prm->dt_mode != 0 && prm->dt_mode != 1)) {
        set_error("PKS params: need dt_max > 0, chi >= 0, dt_mode in {0,1}");
        return DPM_EINVAL;
    }
    dpm_pks *k = new (std::nothrow) dpm_pks();
    if (!k) { set_error("out of host memory"); return DPM_ENOMEM; }
    k->ctx = ctx;
    k->prm = *prm;
    int r = bep_init(&k->bep, ctx, &prm->geom, prm->N, prm->lo, prm->hi, prm->K, prm->beta,
                     prm->precision, s);
    if (r == DPM_OK) {
        dpm_gaussian z{};
        const dpm_gaussian &g0 = rho0 ? *rho0 : z, &g1 = c0 ? *c0 : z;
        if (prm->precision == DPM_PREC_FP64) {
            r = pks_alloc<double>(k, s);
            if (r == DPM_OK) r = pks_init<double>(k->bep.gi, k->bep.gg, g0, g1, k->rho.as<double>(), k->c.as<double>(), s);
        } else {
            r = pks_alloc<float>(k, s);
            if (r == DPM_OK) r = pks_init<float>(k->bep.gi, k->bep.gg, g0, g1, k->rho.as<float>(), k->c.as<float>(), s);
        }
    }
    if (r == DPM_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_error("PKS create: %s", cudaGetErrorString(e)); r = DPM_ECUDA; }
    }
    if (r != DPM_OK) { delete k; return r; }
    *out = k;
    return DPM_OK;
}

extern "C" int dpm_pks_set_state(dpm_pks *k, const void *rho, const void *c, cudaStream_t s) {
    if (!k || !rho || !c) { set_error("pks/rho/c is NULL"); return DPM_EINVAL; }
    const uint8_t *lab = k->bep.gi.labels.as<uint8_t>();
    if (k->prm.precision == DPM_PREC_FP64) {
        DPM_RET(mask_copy<double>(k->prm.N, lab, static_cast<const double *>(rho), k->rho.as<double>(), s));
        DPM_RET(mask_copy<double>(k->prm.N, lab, static_cast<const double *>(c), k->c.as<double>(), s));
    } else {
        DPM_RET(mask_copy<float>(k->prm.N, lab, static_cast<const float *>(rho), k->rho.as<float>(), s));
        DPM_RET(mask_copy<float>(k->prm.N, lab, static_cast<const float *>(c), k->c.as<float>(), s));
    }
    return DPM_OK;
}

extern "C" int dpm_pks_set_graph(dpm_pks *k, int on, cudaStream_t s) {
    if (!k) { set_error("pks is NULL"); return DPM_EINVAL; }
    const dpm_pks_params &P = k->prm;
    if (on) {
        if (k->graph_on) return DPM_OK;
        DPM_CUDA(cudaSetDevice(k->ctx->device));
        dpm_bep *b = &k->bep;
        if (P.dt_mode == 0 && !P.rebuild && (!b->factored || b->sigma != 1.0 / P.dt_max)) {
            // the fixed-dt step solves against the BEP of sigma = 1/dt_max
            const double sg = 1.0 / P.dt_max;
            if (P.precision == DPM_PREC_FP64) DPM_RET(bep_assemble<double>(b, sg, {}, sg, s));
            else DPM_RET(bep_assemble<float>(b, sg, {}, sg, s));
        }
        if (P.precision == DPM_PREC_FP64) DPM_RET(pks_dev_setup<double>(k, s));
        else DPM_RET(pks_dev_setup<float>(k, s));
        k->graph_on = 1;
        return DPM_OK;
    }
    if (!k->graph_on) return DPM_OK;
    int bad = 0;
    DPM_RET(pks_dev_pull(k, s, &bad));
    if (k->gexec) {
        cudaGraphExecDestroy(k->gexec);
        k->gexec = nullptr;
    }
    k->graph_on = 0;
    k->dev_warm = false;
    k->bep.factored = true;
    k->bep.sigma = 1.0 / k->dt_prev;
    return DPM_OK;
}

extern "C" int dpm_pks_step(dpm_pks *k, int nsteps, dpm_pks_stats *stats, cudaStream_t s) {
    if (!k || nsteps < 0) { set_error("pks is NULL or nsteps < 0"); return DPM_EINVAL; }
    for (int i = 0; i < nsteps; ++i) {
        if (k->graph_on) DPM_RET(pks_graph_step(k, s));
        else if (k->prm.precision == DPM_PREC_FP64) DPM_RET(pks_step_one<double>(k, s));
        else DPM_RET(pks_step_one<float>(k, s));
    }
    if (stats && k->graph_on) {
        int bad = 0;
        DPM_RET(pks_dev_pull(k, s, &bad));
        if (bad) { set_error("time step was not positive/finite on the device"); return DPM_ENUMERIC; }
        if (k->last_rebuilt) DPM_RET(lsq_status(k->bep.lsq, s));
    }
    if (stats) {
        double d[6];
        DPM_CUDA(cudaMemcpyAsync(d, k->diag_out.p, sizeof(d), cudaMemcpyDeviceToHost, s));
        DPM_CUDA(cudaStreamSynchronize(s));
        stats->t = k->t;
        stats->dt = k->dt_prev;
        stats->step = k->step;
        stats->rebuilt = k->last_rebuilt;
        stats->mass = d[0];
        stats->max_rho = d[1];
        stats->min_rho = d[2];
        stats->min_c = d[3];
        stats->m2 = d[4];
        stats->free_energy = d[5];
        if (k->prm.precision == DPM_PREC_TC32) DPM_RET(tc_status_check());
        if (!std::isfinite(d[0]) || !std::isfinite(d[5])) {
            set_error("PKS state became non-finite at step %lld", (long long)k->step);
            return DPM_ENUMERIC;
        }
    }
    return DPM_OK;
}

extern "C" int dpm_pks_get_state(dpm_pks *k, void *rho, void *c, cudaStream_t s) {
    if (!k) { set_error("pks is NULL"); return DPM_EINVAL; }
    size_t n3 = (size_t)k->prm.N * k->prm.N * k->prm.N * elem_size(k->prm.precision);
    if (rho) DPM_CUDA(cudaMemcpyAsync(rho, k->rho.p, n3, cudaMemcpyDeviceToDevice, s));
    if (c) DPM_CUDA(cudaMemcpyAsync(c, k->c.p, n3, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

extern "C" int dpm_pks_device_bytes(const dpm_pks *k, int64_t *bytes) {
    if (!k || !bytes) { set_error("pks/bytes is NULL"); return DPM_EINVAL; }
    *bytes = (int64_t)(bep_bytes(k->bep) + k->rho.bytes + k->c.bytes + k->frho.bytes + k->fc.bytes +
                       k->gmax.bytes + k->diag_part.bytes + k->diag_out.bytes);
    return DPM_OK;
}

extern "C" int dpm_pks_destroy(dpm_pks *k) {
    delete k;
    return DPM_OK;
}

// ---------------------------------------------------------------------------
// Domain decomposition, Case 1 (Section 3): Omega_1 = ball |x - c| < r1 on its
// own grid, Omega_2 = shell r1 < |x - c| < r2 on another; the series on Z are
// shared by both sub-domains (interface conditions), the Gamma series belong to
// Omega_2, and the reduced BEPs of both (eqs. reduced_DD1_BEP1,
// reduced_DD1_BEP2) are stacked into one least-squares problem.
// ---------------------------------------------------------------------------
namespace {
struct DDSub {
    int N = 0, prec = 0, ncol_l = 0;
    double lo = 0, hi = 0;
    dpm_geom geom{};
    GridIndex gi;
    GammaGeom gg;
    DevBuf surf, psi, psi_in, trace, dens, work, desc;
    DevBuf rho, c, frho, fc, gmax, diag_part, diag_out;  // time-loop state
};
}  // namespace

struct dpm_dd {
    dpm_ctx *ctx = nullptr;
    dpm_dd_params prm{};
    DDSub sub[2];
    int nz = 0, ng = 0, ncol = 0, storage = 0;  // storage: DPM_PREC_FP64 (double) or float
    double sigma = 0;
    bool factored = false;
    LsqFactor lsq;
    DevBuf coef, bvec;
    DevBuf gwork, gitems;  // grouped SIMT solves of both sub-domains
};

struct dpm_dd_pks {
    dpm_dd dd;
    double chi = 0, dt_max = 0;
    int dt_mode = 0, rebuild = 0, clamp = 1;
    double t = 0, dt_prev = 0;
    int64_t step = 0;
    int last_rebuilt = 0;
    // device-resident steps replayed as a CUDA graph (dpm_dd_pks_set_graph):
    // batch 0 the BEP columns + the particular solutions, 1 the particular
    // solutions, 2 Green's formula
    GraphStepper gs;
    PreparedBatch batch[3];
    std::vector<SubSolve> subs;
};

namespace {

int dd_sub_prec(int requested, int N) {
    if (requested == DPM_PREC_TC32) return tc_supported(N) ? DPM_PREC_TC32 : DPM_PREC_FP32;
    if (requested == DPM_PREC_FFT32)
        return fft_supported(N) ? DPM_PREC_FFT32 : tc_supported(N) ? DPM_PREC_TC32 : DPM_PREC_FP32;
    return requested;
}

ApParams dd_params(const DDSub &sd, double sigma) {
    ApParams p;
    p.N = sd.N;
    p.h = sd.gi.h;
    p.sigma = sigma;
    ap_params_from_index(p, sd.gi);
    return p;
}

// The right-hand sides of the two sub-domains: one grouped set of SIMT launches
// when both grids use the SIMT solver (their N may differ; DPM_DD_GROUP=0 turns
// this off), else one batched solve per sub-domain.
template <class T>
int dd_run_pair(int prec0, const ApParams &p0, const std::vector<ApRhs<T>> &r0, DevBuf &w0, DevBuf &d0,
                int prec1, const ApParams &p1, const std::vector<ApRhs<T>> &r1, DevBuf &w1, DevBuf &d1,
                DevBuf &gw, DevBuf &gd, cudaStream_t s) {
    const char *env = getenv("DPM_DD_GROUP");
    const bool simt0 = prec0 == DPM_PREC_FP32 || prec0 == DPM_PREC_FP64;
    const bool simt1 = prec1 == DPM_PREC_FP32 || prec1 == DPM_PREC_FP64;
    if (!(simt0 && simt1) || (env && env[0] == '0') || r0.empty() || r1.empty()) {
        DPM_RET(run_ap<T>(prec0, p0, r0, w0, d0, s));
        return run_ap<T>(prec1, p1, r1, w1, d1, s);
    }
    std::vector<ApParams> probs = {p0, p1};
    std::vector<ApRhs<T>> rhs(r0);
    rhs.insert(rhs.end(), r1.begin(), r1.end());
    std::vector<int> prob_of(r0.size(), 0);
    prob_of.resize(rhs.size(), 1);
    return ap_solve_simt_group<T>(probs, rhs, prob_of, gw, gd, s);
}

template <class T> int dd_init(dpm_dd *d, dpm_ctx *ctx, const dpm_dd_params &P, cudaStream_t s) {
    d->ctx = ctx;
    d->prm = P;
    d->storage = P.precision == DPM_PREC_FP64 ? DPM_PREC_FP64 : DPM_PREC_FP32;
    d->nz = (P.KZ + 1) * (P.KZ + 1);
    d->ng = (P.KG + 1) * (P.KG + 1);
    d->ncol = 3 * d->nz + 2 * d->ng;
    for (int l = 0; l < 2; ++l) {
        DDSub &sd = d->sub[l];
        sd.geom.kind = l == 0 ? 0 : 2;
        for (int t = 0; t < 3; ++t) sd.geom.center[t] = P.center[t];
        sd.geom.axes[0] = l == 0 ? P.r1 : P.r2;
        sd.geom.axes[1] = l == 0 ? P.r1 : P.r1;
        sd.geom.axes[2] = l == 0 ? P.r1 : 0.0;
        sd.N = l == 0 ? P.N1 : P.N2;
        sd.lo = l == 0 ? P.lo1 : P.lo2;
        sd.hi = l == 0 ? P.hi1 : P.hi2;
        sd.prec = dd_sub_prec(P.precision, sd.N);
        DPM_RET(build_grid_index(sd.geom, sd.N, sd.lo, sd.hi, sd.gi, s));
        const int K = l == 0 ? P.KZ : std::max(P.KZ, P.KG);
        DPM_RET(build_gamma_geom(sd.geom, sd.gi, K, sd.gg, s));
        const int64_t n = sd.gi.n_gamma, m = sd.gi.n_gin;
        DPM_RET(sd.surf.alloc(std::max<int64_t>(n, 1)));
        DPM_RET(dd_surface_flags(n, sd.gg.foot.as<double>(), P.center, l == 0 ? 2.0 * P.r1 : 0.5 * (P.r1 + P.r2),
                                 sd.surf.as<uint8_t>(), s));
        sd.ncol_l = l == 0 ? 3 * d->nz : d->ncol;
        DPM_RET(sd.psi.alloc(sizeof(T) * sd.ncol_l * n));
        DPM_RET(sd.psi_in.alloc(sizeof(double) * sd.ncol_l * m));
        DPM_RET(dd_columns<T>(n, m, sd.gg.nsh, d->nz, d->ng, sd.ncol_l, sd.gg.phi.as<double>(),
                              sd.gg.dist.as<double>(), sd.surf.as<uint8_t>(), sd.gi.gin_pos.as<int>(),
                              sd.psi.as<T>(), sd.psi_in.as<double>(), s));
        DPM_RET(sd.trace.alloc(sizeof(T) * (sd.ncol_l + 4) * m));
        DPM_RET(sd.dens.alloc(sizeof(T) * 4 * n));
    }
    const int64_t m = d->sub[0].gi.n_gin + d->sub[1].gi.n_gin;
    if (m < d->ncol) {
        set_error("%lld BEP rows for %d unknowns: refine the grids or lower KZ/KG", (long long)m, d->ncol);
        return DPM_EINVAL;
    }
    d->lsq.m = (int)m;
    d->lsq.n = d->ncol;
    DPM_RET(d->lsq.A.alloc(sizeof(double) * m * d->ncol));
    DPM_RET(d->coef.alloc(sizeof(double) * 4 * d->ncol));
    DPM_RET(d->bvec.alloc(sizeof(T) * 4 * m));
    return DPM_OK;
}

// Batched solves of every column density of both sub-domains (plus `extra`
// right-hand sides per sub-domain in the same batches), the stacked BEP and
// its factorisation.
template <class T>
int dd_build_bep(dpm_dd *d, double sigma, const std::vector<ApRhs<T>> *extra, double fscale,
                 cudaStream_t s) {
    std::vector<ApRhs<T>> rhs[2];
    ApParams prm[2];
    for (int l = 0; l < 2; ++l) {
        DDSub &sd = d->sub[l];
        const int64_t n = sd.gi.n_gamma, m = sd.gi.n_gin;
        for (int k = 0; k < sd.ncol_l; ++k)
            rhs[l].push_back({nullptr, sd.psi.as<T>() + k * n, nullptr, sd.trace.as<T>() + k * m, 0, 0});
        if (extra)
            for (auto &e : extra[l]) rhs[l].push_back(e);
        prm[l] = dd_params(sd, sigma);
        prm[l].fscale = fscale;
    }
    DPM_RET(dd_run_pair<T>(d->sub[0].prec, prm[0], rhs[0], d->sub[0].work, d->sub[0].desc, d->sub[1].prec, prm[1],
                           rhs[1], d->sub[1].work, d->sub[1].desc, d->gwork, d->gitems, s));
    DPM_RET(dd_assemble<T>(d->sub[0].gi.n_gin, d->sub[1].gi.n_gin, 3 * d->nz, d->ncol,
                           d->sub[0].psi_in.as<double>(), d->sub[0].trace.as<T>(),
                           d->sub[1].psi_in.as<double>(), d->sub[1].trace.as<T>(), d->lsq.A.as<double>(), s));
    DPM_RET(lsq_factor(d->lsq, nullptr, s));
    d->sigma = sigma;
    d->factored = true;
    return DPM_OK;
}

template <class T>
int dd_solve(dpm_dd *d, const void *f1v, const void *f2v, const double *gn, void *u1v, void *u2v,
             double *coeffs, cudaStream_t s) {
    DDSub &a = d->sub[0], &b = d->sub[1];
    const int64_t m1 = a.gi.n_gin, m2 = b.gi.n_gin, n1 = a.gi.n_gamma, n2 = b.gi.n_gamma;
    const T *f[2] = {static_cast<const T *>(f1v), static_cast<const T *>(f2v)};
    T *u[2] = {static_cast<T *>(u1v), static_cast<T *>(u2v)};
    T *tr1 = a.trace.as<T>() + (int64_t)a.ncol_l * m1;
    T *tr2 = b.trace.as<T>() + (int64_t)b.ncol_l * m2, *trv = tr2 + m2;
    T *v = b.dens.as<T>() + n2;
    if (gn) DPM_RET(dd_neumann_density<T>(n2, b.gg.dist.as<double>(), b.surf.as<uint8_t>(), gn, v, s));
    {
        std::vector<ApRhs<T>> r1 = {{f[0], nullptr, nullptr, tr1, 0, 0}};
        std::vector<ApRhs<T>> r2 = {{f[1], nullptr, nullptr, tr2, 0, 0}};
        if (gn) r2.push_back({nullptr, v, nullptr, trv, 0, 0});
        DPM_RET(dd_run_pair<T>(a.prec, dd_params(a, d->sigma), r1, a.work, a.desc, b.prec, dd_params(b, d->sigma),
                               r2, b.work, b.desc, d->gwork, d->gitems, s));
    }
    T *bv = d->bvec.as<T>();
    DPM_RET(dd_rhs<T>(m1, m2, tr1, tr2, gn ? v : nullptr, b.gi.gin_pos.as<int>(), trv, bv, s));
    double *C = d->coef.as<double>();
    DPM_RET(lsq_apply<T>(d->lsq, bv, (int)(m1 + m2), C, 1, s));
    std::vector<ApRhs<T>> g[2];
    for (int l = 0; l < 2; ++l) {
        DDSub &sd = d->sub[l];
        T *dn = sd.dens.as<T>();
        DPM_RET(dd_extend<T>(sd.gi.n_gamma, sd.gg.nsh, d->nz, d->ng, sd.gg.phi.as<double>(),
                             sd.gg.dist.as<double>(), sd.surf.as<uint8_t>(), C, d->ncol,
                             l == 1 ? gn : nullptr, dn, (int)sd.gi.n_gamma, 1, 0, s));
        g[l] = {{f[l], dn, u[l], nullptr, 0, 0}};
    }
    DPM_RET(dd_run_pair<T>(a.prec, dd_params(a, d->sigma), g[0], a.work, a.desc, b.prec, dd_params(b, d->sigma),
                           g[1], b.work, b.desc, d->gwork, d->gitems, s));
    (void)n1;
    if (coeffs) DPM_CUDA(cudaMemcpyAsync(coeffs, C, sizeof(double) * d->ncol, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

int dd_check(const dpm_dd_params *P) {
    if (!P) { set_error("params is NULL"); return DPM_EINVAL; }
    if (!(P->r1 > 0 && P->r2 > P->r1)) { set_error("need 0 < r1 < r2"); return DPM_EINVAL; }
    if (P->KZ < 0 || P->KG < 0 || P->KZ > 16 || P->KG > 16) { set_error("KZ, KG in [0, 16]"); return DPM_EINVAL; }
    if (!prec_ok(P->precision)) { set_error("unknown precision %d", P->precision); return DPM_EINVAL; }
    if (P->N1 > 256 || P->N2 > 256) { set_error("N1, N2 <= 256"); return DPM_EINVAL; }
    return DPM_OK;
}

}  // namespace

extern "C" int dpm_dd_build(dpm_ctx *ctx, const dpm_dd_params *P, double sigma, dpm_dd **out,
                            cudaStream_t s) {
    if (!ctx || !out) { set_error("ctx/out is NULL"); return DPM_EINVAL; }
    *out = nullptr;
    DPM_RET(dd_check(P));
    if (!(sigma >= 0)) { set_error("sigma must be >= 0"); return DPM_EINVAL; }
    DPM_CUDA(cudaSetDevice(ctx->device));
    dpm_dd *d = new (std::nothrow) dpm_dd();
    if (!d) { set_error("out of host memory"); return DPM_ENOMEM; }
    int r;
    if (P->precision == DPM_PREC_FP64) {
        r = dd_init<double>(d, ctx, *P, s);
        if (r == DPM_OK) r = dd_build_bep<double>(d, sigma, nullptr, 1.0, s);
    } else {
        r = dd_init<float>(d, ctx, *P, s);
        if (r == DPM_OK) r = dd_build_bep<float>(d, sigma, nullptr, 1.0, s);
    }
    if (r != DPM_OK) { delete d; return r; }
    *out = d;
    return DPM_OK;
}

extern "C" int dpm_dd_get_info(const dpm_dd *d, dpm_dd_info *info) {
    if (!d || !info) { set_error("dd/info is NULL"); return DPM_EINVAL; }
    for (int l = 0; l < 2; ++l) {
        info->N[l] = d->sub[l].N;
        info->h[l] = d->sub[l].gi.h;
        info->precision[l] = d->sub[l].prec;
        info->n_mplus[l] = d->sub[l].gi.n_mplus;
        info->n_gin[l] = d->sub[l].gi.n_gin;
        info->n_gamma[l] = d->sub[l].gi.n_gamma;
    }
    info->nz = d->nz;
    info->ng = d->ng;
    info->ncol = d->ncol;
    info->sigma = d->sigma;
    return DPM_OK;
}

extern "C" int dpm_dd_matrix(dpm_dd *d, double *A, cudaStream_t s) {
    if (!d || !A) { set_error("dd/A is NULL"); return DPM_EINVAL; }
    DPM_CUDA(cudaMemcpyAsync(A, d->lsq.A.p, sizeof(double) * (size_t)d->lsq.m * d->ncol,
                             cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

extern "C" int dpm_dd_solve(dpm_dd *d, const void *f1, const void *f2, const double *neumann2,
                            void *u1, void *u2, double *coeffs, cudaStream_t s) {
    if (!d || !f1 || !f2 || !u1 || !u2) { set_error("dd/f/u is NULL"); return DPM_EINVAL; }
    if (d->storage == DPM_PREC_FP64) return dd_solve<double>(d, f1, f2, neumann2, u1, u2, coeffs, s);
    return dd_solve<float>(d, f1, f2, neumann2, u1, u2, coeffs, s);
}

extern "C" int dpm_dd_destroy(dpm_dd *d) {
    delete d;
    return DPM_OK;
}

// ---- time loop on the two sub-domains ------------------------------------------------
namespace {

template <class T> int dd_pks_alloc(dpm_dd_pks *k, const dpm_gaussian &g0, const dpm_gaussian &g1,
                                    cudaStream_t s) {
    for (int l = 0; l < 2; ++l) {
        DDSub &sd = k->dd.sub[l];
        const size_t n3 = (size_t)sd.N * sd.N * sd.N;
        DPM_RET(sd.rho.alloc(sizeof(T) * n3));
        DPM_RET(sd.c.alloc(sizeof(T) * n3));
        DPM_RET(sd.frho.alloc(sizeof(T) * n3));
        DPM_RET(sd.fc.alloc(sizeof(T) * n3));
        DPM_RET(sd.gmax.alloc(sizeof(unsigned long long) * 4));
        DPM_RET(sd.diag_part.alloc(sizeof(double) * 6 * pks_diag_blocks(sd.N)));
        DPM_RET(sd.diag_out.alloc(sizeof(double) * 8));
        DPM_CUDA(cudaMemsetAsync(sd.diag_out.p, 0, sizeof(double) * 8, s));
        DPM_RET(pks_init<T>(sd.gi, sd.gg, g0, g1, sd.rho.as<T>(), sd.c.as<T>(), s));
    }
    return DPM_OK;
}

// Steps 3-7 on both sub-domains: dt from the smaller CFL bound of the two grids,
// the stacked BEP rebuilt when dt decreases (or always with rebuild = 1), one
// least squares for the particular traces of both, extensions and Green's
// formula per sub-domain.
template <class T> int dd_pks_step(dpm_dd_pks *k, cudaStream_t s) {
    dpm_dd *d = &k->dd;
    double dt = k->dt_max;
    if (k->dt_mode == 1) {
        for (int l = 0; l < 2; ++l) {
            DDSub &sd = d->sub[l];
            DPM_RET(pks_cfl<T>(sd.N, sd.gi.labels.as<uint8_t>(), sd.c.as<T>(), sd.gmax.as<unsigned long long>(), s));
        }
        double gm[2][3];
        for (int l = 0; l < 2; ++l)
            DPM_CUDA(cudaMemcpyAsync(gm[l], d->sub[l].gmax.p, sizeof(gm[l]), cudaMemcpyDeviceToHost, s));
        DPM_CUDA(cudaStreamSynchronize(s));
        for (int l = 0; l < 2; ++l) {
            const double h = d->sub[l].gi.h;
            for (int ax = 0; ax < 3; ++ax) {
                const double gmaxv = gm[l][ax] / h;
                if (gmaxv > 0) dt = std::min(dt, h / (6.0 * k->chi * gmaxv));
            }
        }
        if (k->step > 0) dt = std::min(dt, k->dt_prev);
    }
    if (!(dt > 0) || !std::isfinite(dt)) { set_error("time step is not positive/finite (dt=%g)", dt); return DPM_ENUMERIC; }
    const bool rebuild = !d->factored || k->rebuild || dt < k->dt_prev;
    const double sigma = 1.0 / dt;
    std::vector<ApRhs<T>> part[2];
    T *trp[2];
    for (int l = 0; l < 2; ++l) {
        DDSub &sd = d->sub[l];
        const int64_t m = sd.gi.n_gin;
        DPM_RET(pks_flux<T>(sd.N, sd.gi.h, k->chi, dt, nullptr, sd.gi.labels.as<uint8_t>(), sd.rho.as<T>(),
                            sd.c.as<T>(), sd.frho.as<T>(), sd.fc.as<T>(), s));
        trp[l] = sd.trace.as<T>() + (int64_t)sd.ncol_l * m;
        part[l] = {{sd.frho.as<T>(), nullptr, nullptr, trp[l], 0, 0},
                   {sd.fc.as<T>(), nullptr, nullptr, trp[l] + m, 0, 0}};
    }
    if (rebuild) {
        DPM_RET(dd_build_bep<T>(d, sigma, part, sigma, s));
    } else {
        ApParams p0 = dd_params(d->sub[0], sigma), p1 = dd_params(d->sub[1], sigma);
        p0.fscale = p1.fscale = sigma;  // L_{h,dt} u = f  <=>  (1/dt - Lap_h) u = f/dt
        DPM_RET(dd_run_pair<T>(d->sub[0].prec, p0, part[0], d->sub[0].work, d->sub[0].desc, d->sub[1].prec, p1,
                               part[1], d->sub[1].work, d->sub[1].desc, d->gwork, d->gitems, s));
    }
    const int64_t m1 = d->sub[0].gi.n_gin, m2 = d->sub[1].gi.n_gin, m = m1 + m2;
    T *bv = d->bvec.as<T>();
    for (int f = 0; f < 2; ++f)
        DPM_RET(dd_rhs<T>(m1, m2, trp[0] + f * m1, trp[1] + f * m2, nullptr, nullptr, nullptr, bv + f * m, s));
    double *C = d->coef.as<double>();
    DPM_RET(lsq_apply<T>(d->lsq, bv, (int)m, C, 2, s));
    std::vector<ApRhs<T>> g[2];
    ApParams pg[2];
    for (int l = 0; l < 2; ++l) {
        DDSub &sd = d->sub[l];
        const int64_t n = sd.gi.n_gamma;
        T *dn = sd.dens.as<T>();
        DPM_RET(dd_extend<T>(n, sd.gg.nsh, d->nz, d->ng, sd.gg.phi.as<double>(), sd.gg.dist.as<double>(),
                             sd.surf.as<uint8_t>(), C, d->ncol, nullptr, dn, (int)n, 2, k->clamp, s));
        g[l] = {{sd.frho.as<T>(), dn, sd.rho.as<T>(), nullptr, 0, 0},
                {sd.fc.as<T>(), dn + n, sd.c.as<T>(), nullptr, 0, 0}};
        pg[l] = dd_params(sd, sigma);
        pg[l].fscale = sigma;
    }
    DPM_RET(dd_run_pair<T>(d->sub[0].prec, pg[0], g[0], d->sub[0].work, d->sub[0].desc, d->sub[1].prec, pg[1],
                           g[1], d->sub[1].work, d->sub[1].desc, d->gwork, d->gitems, s));
    for (int l = 0; l < 2; ++l) {
        DDSub &sd = d->sub[l];
        DPM_RET(pks_diag<T>(sd.N, sd.gi.lo, sd.gi.h, sd.gi.labels.as<uint8_t>(), sd.rho.as<T>(), sd.c.as<T>(),
                            sd.diag_part.as<double>(), sd.diag_out.as<double>(), s));
    }
    k->t += dt;
    k->dt_prev = dt;
    k->step += 1;
    k->last_rebuilt = rebuild ? 1 : 0;
    return DPM_OK;
}

}  // namespace

namespace {

// The device-resident Case 1 step (no host synchronisation, allocation or
// copy: capturable).  Same kernels and arithmetic as dd_pks_step, with dt and
// sigma on the device; the stacked BEP rebuilt every step with rebuild = 1,
// never with dt_mode 0, and when dt decreases (a conditional graph node) with
// the CFL dt otherwise.
template <class T> int dd_dev_setup(dpm_dd_pks *k, cudaStream_t s) {
    dpm_dd *d = &k->dd;
    const int need = (d->factored && k->dt_prev > 0 && d->sigma == 1.0 / k->dt_prev) ? 0 : 1;
    DPM_RET(k->gs.push(k->t, k->dt_prev, k->step, k->last_rebuilt, need, s));
    const StepScalars *sc = k->gs.sc();
    k->subs.assign(2, SubSolve{});
    std::vector<std::vector<std::vector<ApRhs<T>>>> rhs(3, std::vector<std::vector<ApRhs<T>>>(2));
    const bool rebuild = k->dt_mode == 1 || k->rebuild;  // batch 0 is needed
    for (int l = 0; l < 2; ++l) {
        DDSub &sd = d->sub[l];
        ApParams p = dd_params(sd, 0.0);
        p.sigma_dev = &sc->sigma;
        p.fscale_dev = &sc->sigma;  // L_{h,dt} u = f  <=>  (1/dt - Lap_h) u = f/dt
        k->subs[l] = {sd.prec, p, &sd.work};
        const int64_t n = sd.gi.n_gamma, m = sd.gi.n_gin;
        T *trp = sd.trace.as<T>() + (int64_t)sd.ncol_l * m, *dn = sd.dens.as<T>();
        std::vector<ApRhs<T>> part = {{sd.frho.as<T>(), nullptr, nullptr, trp, 0, 0},
                                      {sd.fc.as<T>(), nullptr, nullptr, trp + m, 0, 0}};
        if (rebuild) {
            for (int j = 0; j < sd.ncol_l; ++j)
                rhs[0][l].push_back({nullptr, sd.psi.as<T>() + j * n, nullptr, sd.trace.as<T>() + j * m, 0, 0});
            for (auto &e : part) rhs[0][l].push_back(e);
        }
        rhs[1][l] = part;
        rhs[2][l] = {{sd.frho.as<T>(), dn, sd.rho.as<T>(), nullptr, 0, 0},
                     {sd.fc.as<T>(), dn + n, sd.c.as<T>(), nullptr, 0, 0}};
    }
    return prepare_batches<T>(k->subs, rhs, k->batch, d->gwork, s);
}

template <class T> int dd_step_dev(dpm_dd_pks *k, cudaStream_t s) {
    dpm_dd *d = &k->dd;
    StepScalars *sc = k->gs.sc();
    StepGrids g;
    g.n = 2;
    for (int l = 0; l < 2; ++l) {
        DDSub &sd = d->sub[l];
        if (k->dt_mode == 1)
            DPM_RET(pks_cfl<T>(sd.N, sd.gi.labels.as<uint8_t>(), sd.c.as<T>(), sd.gmax.as<unsigned long long>(), s));
        g.gmax[l] = sd.gmax.as<unsigned long long>();
        g.h[l] = sd.gi.h;
    }
    DPM_RET(pks_step_dt_grids(g, k->chi, k->dt_max, k->dt_mode, sc, s));
    T *trp[2];
    for (int l = 0; l < 2; ++l) {
        DDSub &sd = d->sub[l];
        DPM_RET(pks_flux<T>(sd.N, sd.gi.h, k->chi, 0.0, &sc->dt, sd.gi.labels.as<uint8_t>(), sd.rho.as<T>(),
                            sd.c.as<T>(), sd.frho.as<T>(), sd.fc.as<T>(), s));
        trp[l] = sd.trace.as<T>() + (int64_t)sd.ncol_l * sd.gi.n_gin;
    }
    const bool cond = k->dt_mode == 1 && !k->rebuild;  // Step 4b decided on the device
    const bool rebuild = k->rebuild != 0;
    auto with_rebuild = [&](cudaStream_t st) -> int {
        DPM_RET(run_prepared<T>(k->batch[0], k->subs, st));
        DPM_RET(dd_assemble<T>(d->sub[0].gi.n_gin, d->sub[1].gi.n_gin, 3 * d->nz, d->ncol,
                               d->sub[0].psi_in.as<double>(), d->sub[0].trace.as<T>(),
                               d->sub[1].psi_in.as<double>(), d->sub[1].trace.as<T>(), d->lsq.A.as<double>(), st));
        return lsq_factor_async(d->lsq, st);
    };
    auto particular_only = [&](cudaStream_t st) -> int { return run_prepared<T>(k->batch[1], k->subs, st); };
    if (cond) DPM_RET(step_branch(sc, s, k->gs.aux, with_rebuild, particular_only));
    else if (rebuild) DPM_RET(with_rebuild(s));
    else DPM_RET(particular_only(s));
    const int64_t m1 = d->sub[0].gi.n_gin, m2 = d->sub[1].gi.n_gin, m = m1 + m2;
    T *bv = d->bvec.as<T>();
    for (int f = 0; f < 2; ++f)
        DPM_RET(dd_rhs<T>(m1, m2, trp[0] + f * m1, trp[1] + f * m2, nullptr, nullptr, nullptr, bv + f * m, s));
    double *C = d->coef.as<double>();
    DPM_RET(lsq_apply<T>(d->lsq, bv, (int)m, C, 2, s));
    for (int l = 0; l < 2; ++l) {
        DDSub &sd = d->sub[l];
        const int64_t n = sd.gi.n_gamma;
        DPM_RET(dd_extend<T>(n, sd.gg.nsh, d->nz, d->ng, sd.gg.phi.as<double>(), sd.gg.dist.as<double>(),
                             sd.surf.as<uint8_t>(), C, d->ncol, nullptr, sd.dens.as<T>(), (int)n, 2, k->clamp, s));
    }
    DPM_RET(run_prepared<T>(k->batch[2], k->subs, s));
    for (int l = 0; l < 2; ++l) {
        DDSub &sd = d->sub[l];
        DPM_RET(pks_diag<T>(sd.N, sd.gi.lo, sd.gi.h, sd.gi.labels.as<uint8_t>(), sd.rho.as<T>(), sd.c.as<T>(),
                            sd.diag_part.as<double>(), sd.diag_out.as<double>(), s));
    }
    DPM_RET(pks_step_end(sc, cond ? -1 : (rebuild ? 1 : 0), s));
    return DPM_OK;
}

}  // namespace

extern "C" int dpm_dd_pks_set_graph(dpm_dd_pks *k, int on, cudaStream_t s) {
    if (!k) { set_error("pks is NULL"); return DPM_EINVAL; }
    dpm_dd *d = &k->dd;
    const bool f64 = d->storage == DPM_PREC_FP64;
    if (on) {
        if (k->gs.on) return DPM_OK;
        DPM_CUDA(cudaSetDevice(d->ctx->device));
        if (k->dt_mode == 0 && !k->rebuild && (!d->factored || d->sigma != 1.0 / k->dt_max)) {
            // the fixed-dt step solves against the stacked BEP of sigma = 1/dt_max
            const double sg = 1.0 / k->dt_max;
            if (f64) DPM_RET(dd_build_bep<double>(d, sg, nullptr, sg, s));
            else DPM_RET(dd_build_bep<float>(d, sg, nullptr, sg, s));
        }
        if (f64) DPM_RET(dd_dev_setup<double>(k, s));
        else DPM_RET(dd_dev_setup<float>(k, s));
        k->gs.on = 1;
        return DPM_OK;
    }
    if (!k->gs.on) return DPM_OK;
    int bad = 0;
    DPM_RET(k->gs.pull(k->t, k->dt_prev, k->step, k->last_rebuilt, &bad, s));
    k->gs.stop();
    d->factored = true;
    d->sigma = 1.0 / k->dt_prev;
    return DPM_OK;
}

extern "C" int dpm_dd_pks_create(dpm_ctx *ctx, const dpm_dd_params *P, double chi, double dt_max,
                                 int dt_mode, int rebuild, int clamp, const dpm_gaussian *rho0,
                                 const dpm_gaussian *c0, dpm_dd_pks **out, cudaStream_t s) {
    if (!ctx || !out) { set_error("ctx/out is NULL"); return DPM_EINVAL; }
    *out = nullptr;
    DPM_RET(dd_check(P));
    if (!(dt_max > 0) || !(chi >= 0) || (dt_mode != 0 && dt_mode != 1)) {
        set_error("need dt_max > 0, chi >= 0, dt_mode in {0,1}");
        return DPM_EINVAL;
    }
    DPM_CUDA(cudaSetDevice(ctx->device));
    dpm_dd_pks *k = new (std::nothrow) dpm_dd_pks();
    if (!k) { set_error("out of host memory"); return DPM_ENOMEM; }
    k->chi = chi;
    k->dt_max = dt_max;
    k->dt_mode = dt_mode;
    k->rebuild = rebuild;
    k->clamp = clamp;
    dpm_gaussian z{};
    const dpm_gaussian &g0 = rho0 ? *rho0 : z, &g1 = c0 ? *c0 : z;
    int r;
    if (P->precision == DPM_PREC_FP64) {
        r = dd_init<double>(&k->dd, ctx, *P, s);
        if (r == DPM_OK) r = dd_pks_alloc<double>(k, g0, g1, s);
    } else {
        r = dd_init<float>(&k->dd, ctx, *P, s);
        if (r == DPM_OK) r = dd_pks_alloc<float>(k, g0, g1, s);
    }
    if (r == DPM_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_error("%s", cudaGetErrorString(e)); r = DPM_ECUDA; }
    }
    if (r != DPM_OK) { delete k; return r; }
    *out = k;
    return DPM_OK;
}

extern "C" int dpm_dd_pks_step(dpm_dd_pks *k, int nsteps, dpm_pks_stats *stats, cudaStream_t s) {
    if (!k || nsteps < 0) { set_error("pks is NULL or nsteps < 0"); return DPM_EINVAL; }
    const bool f64 = k->dd.storage == DPM_PREC_FP64;
    for (int i = 0; i < nsteps; ++i) {
        if (k->gs.on)
            DPM_RET(k->gs.step([&](cudaStream_t st) { return f64 ? dd_step_dev<double>(k, st) : dd_step_dev<float>(k, st); }, s));
        else if (f64) DPM_RET(dd_pks_step<double>(k, s));
        else DPM_RET(dd_pks_step<float>(k, s));
    }
    if (stats && k->gs.on) {
        int bad = 0;
        DPM_RET(k->gs.pull(k->t, k->dt_prev, k->step, k->last_rebuilt, &bad, s));
        if (bad) { set_error("time step was not positive/finite on the device"); return DPM_ENUMERIC; }
        if (k->last_rebuilt) DPM_RET(lsq_status(k->dd.lsq, s));
    }
    if (stats) {
        double d[2][6];
        for (int l = 0; l < 2; ++l)
            DPM_CUDA(cudaMemcpyAsync(d[l], k->dd.sub[l].diag_out.p, sizeof(d[l]), cudaMemcpyDeviceToHost, s));
        DPM_CUDA(cudaStreamSynchronize(s));
        stats->t = k->t;
        stats->dt = k->dt_prev;
        stats->step = k->step;
        stats->rebuilt = k->last_rebuilt;
        stats->mass = d[0][0] + d[1][0];
        stats->max_rho = std::max(d[0][1], d[1][1]);
        stats->min_rho = std::min(d[0][2], d[1][2]);
        stats->min_c = std::min(d[0][3], d[1][3]);
        stats->m2 = d[0][4] + d[1][4];
        stats->free_energy = d[0][5] + d[1][5];
        if (k->dd.prm.precision == DPM_PREC_TC32) DPM_RET(tc_status_check());
        if (!std::isfinite(stats->mass) || !std::isfinite(stats->free_energy)) {
            set_error("PKS state became non-finite at step %lld", (long long)k->step);
            return DPM_ENUMERIC;
        }
    }
    return DPM_OK;
}

extern "C" int dpm_dd_pks_get_state(dpm_dd_pks *k, int l, void *rho, void *c, cudaStream_t s) {
    if (!k || l < 0 || l > 1) { set_error("pks is NULL or sub-domain index not 0/1"); return DPM_EINVAL; }
    const DDSub &sd = k->dd.sub[l];
    const size_t n3 = (size_t)sd.N * sd.N * sd.N * elem_size(k->dd.storage);
    if (rho) DPM_CUDA(cudaMemcpyAsync(rho, sd.rho.p, n3, cudaMemcpyDeviceToDevice, s));
    if (c) DPM_CUDA(cudaMemcpyAsync(c, sd.c.p, n3, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

extern "C" int dpm_dd_pks_destroy(dpm_dd_pks *k) {
    delete k;
    return DPM_OK;
}

// ---------------------------------------------------------------------------
// Domain decomposition, Case 2 (Section 3): the interface Z (a sphere about
// center + (0, 0, zoff)) meets Gamma.  Omega_1 = Omega inside Z, Omega_2 =
// Omega outside Z, each on its own grid in its own frame; the grid boundary of
// each splits into Gamma nodes, Z nodes and the wedge layer carrying both
// (eq. reduced_DD2_BEP); the Z and Gamma zonal series are shared by both
// sub-domains and the stacked reduced BEPs solved in the least-squares sense.
// ---------------------------------------------------------------------------
namespace {
struct DD2Sub {
    int N = 0, prec = 0;
    double lo = 0, hi = 0, origin[3] = {0, 0, 0};
    dpm_geom geom{};
    GridIndex gi;
    int64_t n_rows = 0, n_wedge = 0;
    DevBuf flags, dG, dZ, cosG, cosZ, footG, footZ, YG, YZ;
    DevBuf row_i, row_e, row_s;
    DevBuf psi, own, trace, dens, vG, work, desc;
    GammaGeom init_geom;                                   // foot points for the initial data
    DevBuf rho, c, frho, fc, gmax, diag_part, diag_out;    // time-loop state
};
}  // namespace

struct dpm_dd2 {
    dpm_ctx *ctx = nullptr;
    dpm_dd2_params prm{};
    DD2Sub sub[2];
    int ncol = 0, storage = 0;
    double sigma = 0;
    bool factored = false;
    LsqFactor lsq;
    DevBuf coef, bvec;
    DevBuf gwork, gitems;  // grouped SIMT solves of both sub-domains
};

struct dpm_dd2_pks {
    dpm_dd2 dd;
    double chi = 0, dt_max = 0;
    int dt_mode = 0, rebuild = 0, clamp = 1;
    double t = 0, dt_prev = 0;
    int64_t step = 0;
    int last_rebuilt = 0;
    // device-resident steps replayed as a CUDA graph (dpm_dd2_pks_set_graph)
    GraphStepper gs;
    PreparedBatch batch[3];
    std::vector<SubSolve> subs;
};

namespace {

ApParams dd2_ap(const DD2Sub &sd, double sigma) {
    ApParams p;
    p.N = sd.N;
    p.h = sd.gi.h;
    p.sigma = sigma;
    ap_params_from_index(p, sd.gi);
    return p;
}

// Unknown series on Gamma: 2 (u and d^2u/dn^2, the default) or 1 (u only).
int dd2_gamma_series(const dpm_dd2_params &P) { return P.gamma_series == 1 ? 1 : 2; }

int dd2_check(const dpm_dd2_params *P) {
    if (!P) { set_error("params is NULL"); return DPM_EINVAL; }
    if (!(P->R > 0 && P->rz > 0)) { set_error("need R > 0, rz > 0"); return DPM_EINVAL; }
    const double az = std::fabs(P->zoff);
    if (!(az > std::fabs(P->R - P->rz) && az < P->R + P->rz)) {
        set_error("Case 2 needs |R - rz| < |zoff| < R + rz (Z must cut Gamma)");
        return DPM_EINVAL;
    }
    if (P->MZ < 1 || P->MZ > 64 || P->MG < 1 || P->MG > 1024) {
        set_error("MZ in [1, 64], MG in [1, 1024]");
        return DPM_EINVAL;
    }
    if (P->gamma_series < 0 || P->gamma_series > 2) {
        set_error("gamma_series must be 0 (default: 2), 1 or 2 (got %d)", P->gamma_series);
        return DPM_EINVAL;
    }
    if (!prec_ok(P->precision)) { set_error("unknown precision %d", P->precision); return DPM_EINVAL; }
    if (P->N1 > 256 || P->N2 > 256) { set_error("N1, N2 <= 256"); return DPM_EINVAL; }
    return DPM_OK;
}

template <class T> int dd2_init(dpm_dd2 *d, dpm_ctx *ctx, const dpm_dd2_params &P, cudaStream_t s) {
    d->ctx = ctx;
    d->prm = P;
    d->storage = P.precision == DPM_PREC_FP64 ? DPM_PREC_FP64 : DPM_PREC_FP32;
    const int MZ = P.MZ, MG = P.MG;
    d->ncol = 3 * MZ + dd2_gamma_series(P) * MG;
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = d->sub[l];
        const double *org = l == 0 ? P.origin1 : P.origin2;
        for (int t = 0; t < 3; ++t) sd.origin[t] = org[t];
        sd.geom.kind = l == 0 ? 3 : 4;
        for (int t = 0; t < 3; ++t) sd.geom.center[t] = P.center[t] - org[t];
        sd.geom.axes[0] = P.R;
        sd.geom.axes[1] = P.rz;
        sd.geom.axes[2] = P.zoff;
        sd.N = l == 0 ? P.N1 : P.N2;
        sd.lo = l == 0 ? P.lo1 : P.lo2;
        sd.hi = l == 0 ? P.hi1 : P.hi2;
        sd.prec = dd_sub_prec(P.precision, sd.N);
        DPM_RET(build_grid_index(sd.geom, sd.N, sd.lo, sd.hi, sd.gi, s));
        const int64_t n = sd.gi.n_gamma, g = sd.gi.n_gin;
        const int64_t n3 = (int64_t)sd.N * sd.N * sd.N;
        // the grid-boundary sets of the whole sphere and of the ball inside Z
        const double c0[3] = {sd.geom.center[0], sd.geom.center[1], sd.geom.center[2]};
        const double cz[3] = {c0[0], c0[1], c0[2] + P.zoff};
        dpm_geom go{}, gb{};
        go.kind = gb.kind = 0;
        for (int t = 0; t < 3; ++t) {
            go.center[t] = c0[t];
            gb.center[t] = cz[t];
            go.axes[t] = P.R;
            gb.axes[t] = P.rz;
        }
        DevBuf lab_o, lab_b;
        DPM_RET(lab_o.alloc(n3));
        DPM_RET(lab_b.alloc(n3));
        DPM_RET(classify_labels(go, sd.N, sd.lo, sd.hi, lab_o.as<uint8_t>(), s));
        DPM_RET(classify_labels(gb, sd.N, sd.lo, sd.hi, lab_b.as<uint8_t>(), s));
        const int64_t n1 = std::max<int64_t>(n, 1);
        DPM_RET(sd.flags.alloc(n1));
        DPM_RET(sd.dG.alloc(sizeof(double) * n1));
        DPM_RET(sd.dZ.alloc(sizeof(double) * n1));
        DPM_RET(sd.cosG.alloc(sizeof(double) * n1));
        DPM_RET(sd.cosZ.alloc(sizeof(double) * n1));
        DPM_RET(sd.footG.alloc(sizeof(double) * 3 * n1));
        DPM_RET(sd.footZ.alloc(sizeof(double) * 3 * n1));
        DPM_RET(dd2_split(sd.gi, lab_o.as<uint8_t>(), lab_b.as<uint8_t>(), c0, P.R, cz, P.rz,
                          sd.flags.as<uint8_t>(), sd.dG.as<double>(), sd.dZ.as<double>(), sd.cosG.as<double>(),
                          sd.cosZ.as<double>(), sd.footG.as<double>(), sd.footZ.as<double>(), s));
        DPM_RET(sd.YG.alloc(sizeof(double) * MG * n1));
        DPM_RET(sd.YZ.alloc(sizeof(double) * MZ * n1));
        // Z inside Omega spans cos theta_Z in [-1, c*] (zoff > 0) or [c*, 1], c* the
        // cosine at the circle Z n Gamma: (R^2 - zoff^2 - rz^2)/(2 zoff rz)
        const double cstar = (P.R * P.R - P.zoff * P.zoff - P.rz * P.rz) / (2.0 * P.zoff * P.rz);
        const double za = P.zoff > 0 ? -1.0 : cstar, zb = P.zoff > 0 ? cstar : 1.0;
        DPM_RET(dd2_zonal(n, MG, sd.cosG.as<double>(), -1.0, 1.0, sd.YG.as<double>(), s));
        DPM_RET(dd2_zonal(n, MZ, sd.cosZ.as<double>(), za, zb, sd.YZ.as<double>(), s));
        // BEP rows: gamma_in nodes in ascending order, a Gamma row before a Z row
        std::vector<uint8_t> hf(n);
        std::vector<int> hpos(g);
        if (n) DPM_CUDA(cudaMemcpyAsync(hf.data(), sd.flags.p, n, cudaMemcpyDeviceToHost, s));
        if (g) DPM_CUDA(cudaMemcpyAsync(hpos.data(), sd.gi.gin_pos.p, sizeof(int) * g, cudaMemcpyDeviceToHost, s));
        DPM_CUDA(cudaStreamSynchronize(s));
        std::vector<int> ri, re;
        std::vector<uint8_t> rs;
        sd.n_wedge = 0;
        for (int64_t e = 0; e < n; ++e) sd.n_wedge += hf[e] == 3;
        for (int64_t i = 0; i < g; ++i) {
            const int e = hpos[i];
            if (hf[e] & 1) { ri.push_back((int)i); re.push_back(e); rs.push_back(0); }
            if (hf[e] & 2) { ri.push_back((int)i); re.push_back(e); rs.push_back(1); }
        }
        sd.n_rows = (int64_t)ri.size();
        const int64_t m1 = std::max<int64_t>(sd.n_rows, 1);
        DPM_RET(sd.row_i.alloc(sizeof(int) * m1));
        DPM_RET(sd.row_e.alloc(sizeof(int) * m1));
        DPM_RET(sd.row_s.alloc(m1));
        if (sd.n_rows) {
            DPM_CUDA(cudaMemcpyAsync(sd.row_i.p, ri.data(), sizeof(int) * sd.n_rows, cudaMemcpyHostToDevice, s));
            DPM_CUDA(cudaMemcpyAsync(sd.row_e.p, re.data(), sizeof(int) * sd.n_rows, cudaMemcpyHostToDevice, s));
            DPM_CUDA(cudaMemcpyAsync(sd.row_s.p, rs.data(), sd.n_rows, cudaMemcpyHostToDevice, s));
        }
        DPM_RET(sd.psi.alloc(sizeof(T) * d->ncol * n1));
        DPM_RET(sd.own.alloc(sizeof(double) * d->ncol * m1));
        DPM_RET(dd2_columns<T>(n, sd.n_rows, MZ, MG, dd2_gamma_series(P), sd.flags.as<uint8_t>(), sd.dG.as<double>(), sd.dZ.as<double>(),
                               sd.YG.as<double>(), sd.YZ.as<double>(), sd.row_e.as<int>(), sd.row_s.as<uint8_t>(),
                               sd.psi.as<T>(), sd.own.as<double>(), s));
        DPM_RET(sd.trace.alloc(sizeof(T) * (d->ncol + 4) * std::max<int64_t>(g, 1)));
        DPM_RET(sd.dens.alloc(sizeof(T) * 4 * n1));
        DPM_RET(sd.vG.alloc(sizeof(double) * n1));
        DPM_CUDA(cudaStreamSynchronize(s));  // host vectors and label buffers go out of scope
    }
    const int64_t m = d->sub[0].n_rows + d->sub[1].n_rows;
    if (m < d->ncol) {
        set_error("%lld BEP rows for %d unknowns: refine the grids or lower MZ/MG", (long long)m, d->ncol);
        return DPM_EINVAL;
    }
    d->lsq.m = (int)m;
    d->lsq.n = d->ncol;
    // the partial-sphere series make kappa^2 too large for the FP32 Gram
    d->lsq.method = LsqFactor::kEquilibrated64;
    DPM_RET(d->lsq.A.alloc(sizeof(double) * m * d->ncol));
    DPM_RET(d->coef.alloc(sizeof(double) * 4 * d->ncol));
    DPM_RET(d->bvec.alloc(sizeof(T) * 4 * m));
    return DPM_OK;
}

template <class T>
int dd2_build_bep(dpm_dd2 *d, double sigma, const std::vector<ApRhs<T>> *extra, double fscale, cudaStream_t s) {
    std::vector<ApRhs<T>> rhs[2];
    ApParams prm[2];
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = d->sub[l];
        const int64_t n = sd.gi.n_gamma, g = sd.gi.n_gin;
        for (int k = 0; k < d->ncol; ++k)
            rhs[l].push_back({nullptr, sd.psi.as<T>() + k * n, nullptr, sd.trace.as<T>() + k * g, 0, 0});
        if (extra)
            for (auto &e : extra[l]) rhs[l].push_back(e);
        prm[l] = dd2_ap(sd, sigma);
        prm[l].fscale = fscale;
    }
    DPM_RET(dd_run_pair<T>(d->sub[0].prec, prm[0], rhs[0], d->sub[0].work, d->sub[0].desc, d->sub[1].prec, prm[1],
                           rhs[1], d->sub[1].work, d->sub[1].desc, d->gwork, d->gitems, s));
    const DD2Sub &a = d->sub[0], &b = d->sub[1];
    DPM_RET(dd2_assemble<T>(a.n_rows, b.n_rows, d->ncol, a.own.as<double>(), a.trace.as<T>(), a.gi.n_gin,
                            a.row_i.as<int>(), b.own.as<double>(), b.trace.as<T>(), b.gi.n_gin, b.row_i.as<int>(),
                            d->lsq.A.as<double>(), s));
    DPM_RET(lsq_factor(d->lsq, nullptr, s));
    d->sigma = sigma;
    d->factored = true;
    return DPM_OK;
}

template <class T>
int dd2_solve(dpm_dd2 *d, const void *f1v, const void *f2v, const double *gn1, const double *gn2, void *u1v,
              void *u2v, double *coeffs, cudaStream_t s) {
    const T *f[2] = {static_cast<const T *>(f1v), static_cast<const T *>(f2v)};
    T *u[2] = {static_cast<T *>(u1v), static_cast<T *>(u2v)};
    const double *gn[2] = {gn1, gn2};
    T *bv = d->bvec.as<T>();
    int64_t off = 0;
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = d->sub[l];
        const int64_t n = sd.gi.n_gamma, g = sd.gi.n_gin;
        T *trp = sd.trace.as<T>() + (int64_t)d->ncol * g, *trv = trp + g;
        T *veff = sd.dens.as<T>() + n;
        std::vector<ApRhs<T>> r = {{f[l], nullptr, nullptr, trp, 0, 0}};
        if (gn[l]) {
            DPM_RET(dd2_neumann<T>(n, sd.flags.as<uint8_t>(), sd.dG.as<double>(), gn[l], sd.vG.as<double>(), veff, s));
            r.push_back({nullptr, veff, nullptr, trv, 0, 0});
        }
        DPM_RET(run_ap<T>(sd.prec, dd2_ap(sd, d->sigma), r, sd.work, sd.desc, s));
        DPM_RET(dd2_rhs<T>(sd.n_rows, sd.row_i.as<int>(), sd.row_e.as<int>(), sd.row_s.as<uint8_t>(), trp,
                           gn[l] ? sd.vG.as<double>() : nullptr, trv, bv + off, s));
        off += sd.n_rows;
    }
    double *C = d->coef.as<double>();
    DPM_RET(lsq_apply<T>(d->lsq, bv, (int)off, C, 1, s));
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = d->sub[l];
        const int64_t n = sd.gi.n_gamma;
        T *dn = sd.dens.as<T>();
        DPM_RET(dd2_extend<T>(n, d->prm.MZ, d->prm.MG, dd2_gamma_series(d->prm), sd.flags.as<uint8_t>(), sd.dG.as<double>(), sd.dZ.as<double>(),
                              sd.YG.as<double>(), sd.YZ.as<double>(), C, d->ncol, gn[l], dn, (int)n, 1, 0, s));
        std::vector<ApRhs<T>> gr = {{f[l], dn, u[l], nullptr, 0, 0}};
        DPM_RET(run_ap<T>(sd.prec, dd2_ap(sd, d->sigma), gr, sd.work, sd.desc, s));
    }
    if (coeffs) DPM_CUDA(cudaMemcpyAsync(coeffs, C, sizeof(double) * d->ncol, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

}  // namespace

extern "C" int dpm_dd2_build(dpm_ctx *ctx, const dpm_dd2_params *P, double sigma, dpm_dd2 **out,
                             cudaStream_t s) {
    if (!ctx || !out) { set_error("ctx/out is NULL"); return DPM_EINVAL; }
    *out = nullptr;
    DPM_RET(dd2_check(P));
    if (!(sigma > 0)) { set_error("sigma must be > 0"); return DPM_EINVAL; }
    DPM_CUDA(cudaSetDevice(ctx->device));
    dpm_dd2 *d = new (std::nothrow) dpm_dd2();
    if (!d) { set_error("out of host memory"); return DPM_ENOMEM; }
    int r;
    if (P->precision == DPM_PREC_FP64) {
        r = dd2_init<double>(d, ctx, *P, s);
        if (r == DPM_OK) r = dd2_build_bep<double>(d, sigma, nullptr, 1.0, s);
    } else {
        r = dd2_init<float>(d, ctx, *P, s);
        if (r == DPM_OK) r = dd2_build_bep<float>(d, sigma, nullptr, 1.0, s);
    }
    if (r == DPM_OK && P->precision == DPM_PREC_TC32) r = tc_status_check();
    if (r != DPM_OK) { delete d; return r; }
    *out = d;
    return DPM_OK;
}

extern "C" int dpm_dd2_get_info(const dpm_dd2 *d, dpm_dd2_info *info) {
    if (!d || !info) { set_error("dd/info is NULL"); return DPM_EINVAL; }
    for (int l = 0; l < 2; ++l) {
        const DD2Sub &sd = d->sub[l];
        info->N[l] = sd.N;
        info->h[l] = sd.gi.h;
        info->precision[l] = sd.prec;
        info->n_mplus[l] = sd.gi.n_mplus;
        info->n_gin[l] = sd.gi.n_gin;
        info->n_gamma[l] = sd.gi.n_gamma;
        info->n_rows[l] = sd.n_rows;
        info->n_wedge[l] = sd.n_wedge;
    }
    info->ncol = d->ncol;
    info->sigma = d->sigma;
    return DPM_OK;
}

extern "C" int dpm_dd2_matrix(dpm_dd2 *d, double *A, cudaStream_t s) {
    if (!d || !A) { set_error("dd/A is NULL"); return DPM_EINVAL; }
    const size_t bytes = sizeof(double) * (size_t)d->lsq.m * d->ncol;
    DPM_CUDA(cudaMemcpyAsync(A, d->lsq.A.p, bytes, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

extern "C" int dpm_dd2_gamma(dpm_dd2 *d, int l, int32_t *gamma_idx, uint8_t *flags, double *foot_gamma,
                             cudaStream_t s) {
    if (!d || l < 0 || l > 1) { set_error("dd is NULL or sub-domain index not 0/1"); return DPM_EINVAL; }
    const DD2Sub &sd = d->sub[l];
    const size_t n = (size_t)sd.gi.n_gamma;
    if (gamma_idx) DPM_CUDA(cudaMemcpyAsync(gamma_idx, sd.gi.gamma.p, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    if (flags) DPM_CUDA(cudaMemcpyAsync(flags, sd.flags.p, n, cudaMemcpyDeviceToDevice, s));
    if (foot_gamma)
        DPM_CUDA(cudaMemcpyAsync(foot_gamma, sd.footG.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

extern "C" int dpm_dd2_solve(dpm_dd2 *d, const void *f1, const void *f2, const double *neumann1,
                             const double *neumann2, void *u1, void *u2, double *coeffs, cudaStream_t s) {
    if (!d || !f1 || !f2 || !u1 || !u2) { set_error("dd/f/u is NULL"); return DPM_EINVAL; }
    int r = d->storage == DPM_PREC_FP64 ? dd2_solve<double>(d, f1, f2, neumann1, neumann2, u1, u2, coeffs, s)
                                        : dd2_solve<float>(d, f1, f2, neumann1, neumann2, u1, u2, coeffs, s);
    if (r == DPM_OK && d->prm.precision == DPM_PREC_TC32) r = tc_status_check();
    return r;
}

extern "C" int dpm_dd2_destroy(dpm_dd2 *d) {
    delete d;
    return DPM_OK;
}

// ---- time loop on the two sub-domains of Case 2 --------------------------------------
namespace {

template <class T> int dd2_pks_alloc(dpm_dd2_pks *k, const dpm_gaussian &g0, const dpm_gaussian &g1, cudaStream_t s) {
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = k->dd.sub[l];
        const size_t n3 = (size_t)sd.N * sd.N * sd.N;
        DPM_RET(sd.rho.alloc(sizeof(T) * n3));
        DPM_RET(sd.c.alloc(sizeof(T) * n3));
        DPM_RET(sd.frho.alloc(sizeof(T) * n3));
        DPM_RET(sd.fc.alloc(sizeof(T) * n3));
        DPM_RET(sd.gmax.alloc(sizeof(unsigned long long) * 4));
        DPM_RET(sd.diag_part.alloc(sizeof(double) * 6 * pks_diag_blocks(sd.N)));
        DPM_RET(sd.diag_out.alloc(sizeof(double) * 8));
        DPM_CUDA(cudaMemsetAsync(sd.diag_out.p, 0, sizeof(double) * 8, s));
        const int64_t n = sd.gi.n_gamma;
        DPM_RET(sd.init_geom.foot.alloc(sizeof(double) * 3 * std::max<int64_t>(n, 1)));
        DPM_RET(dd2_init_foot(n, sd.flags.as<uint8_t>(), sd.footG.as<double>(), sd.footZ.as<double>(),
                              sd.init_geom.foot.as<double>(), s));
        dpm_gaussian a = g0, b = g1;  // centres in the local frame
        for (int t = 0; t < 3; ++t) {
            a.center[t] -= sd.origin[t];
            b.center[t] -= sd.origin[t];
        }
        DPM_RET(pks_init<T>(sd.gi, sd.init_geom, a, b, sd.rho.as<T>(), sd.c.as<T>(), s));
    }
    return DPM_OK;
}

template <class T> int dd2_pks_step(dpm_dd2_pks *k, cudaStream_t s) {
    dpm_dd2 *d = &k->dd;
    double dt = k->dt_max;
    if (k->dt_mode == 1) {
        for (int l = 0; l < 2; ++l) {
            DD2Sub &sd = d->sub[l];
            DPM_RET(pks_cfl<T>(sd.N, sd.gi.labels.as<uint8_t>(), sd.c.as<T>(), sd.gmax.as<unsigned long long>(), s));
        }
        double gm[2][3];
        for (int l = 0; l < 2; ++l)
            DPM_CUDA(cudaMemcpyAsync(gm[l], d->sub[l].gmax.p, sizeof(gm[l]), cudaMemcpyDeviceToHost, s));
        DPM_CUDA(cudaStreamSynchronize(s));
        for (int l = 0; l < 2; ++l) {
            const double h = d->sub[l].gi.h;
            for (int ax = 0; ax < 3; ++ax) {
                const double gmaxv = gm[l][ax] / h;
                if (gmaxv > 0) dt = std::min(dt, h / (6.0 * k->chi * gmaxv));
            }
        }
        if (k->step > 0) dt = std::min(dt, k->dt_prev);
    }
    if (!(dt > 0) || !std::isfinite(dt)) { set_error("time step is not positive/finite (dt=%g)", dt); return DPM_ENUMERIC; }
    const bool rebuild = !d->factored || k->rebuild || dt < k->dt_prev;
    const double sigma = 1.0 / dt;
    std::vector<ApRhs<T>> part[2];
    T *trp[2];
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = d->sub[l];
        const int64_t g = sd.gi.n_gin;
        DPM_RET(pks_flux<T>(sd.N, sd.gi.h, k->chi, dt, nullptr, sd.gi.labels.as<uint8_t>(), sd.rho.as<T>(),
                            sd.c.as<T>(), sd.frho.as<T>(), sd.fc.as<T>(), s));
        trp[l] = sd.trace.as<T>() + (int64_t)d->ncol * g;
        part[l] = {{sd.frho.as<T>(), nullptr, nullptr, trp[l], 0, 0},
                   {sd.fc.as<T>(), nullptr, nullptr, trp[l] + g, 0, 0}};
    }
    if (rebuild) {
        DPM_RET(dd2_build_bep<T>(d, sigma, part, sigma, s));
    } else {
        ApParams p0 = dd2_ap(d->sub[0], sigma), p1 = dd2_ap(d->sub[1], sigma);
        p0.fscale = p1.fscale = sigma;  // L_{h,dt} u = f  <=>  (1/dt - Lap_h) u = f/dt
        DPM_RET(dd_run_pair<T>(d->sub[0].prec, p0, part[0], d->sub[0].work, d->sub[0].desc, d->sub[1].prec, p1,
                               part[1], d->sub[1].work, d->sub[1].desc, d->gwork, d->gitems, s));
    }
    const int64_t m = d->sub[0].n_rows + d->sub[1].n_rows;
    T *bv = d->bvec.as<T>();
    for (int f = 0; f < 2; ++f) {
        int64_t off = 0;
        for (int l = 0; l < 2; ++l) {
            DD2Sub &sd = d->sub[l];
            DPM_RET(dd2_rhs<T>(sd.n_rows, sd.row_i.as<int>(), sd.row_e.as<int>(), sd.row_s.as<uint8_t>(),
                               trp[l] + f * sd.gi.n_gin, nullptr, nullptr, bv + f * m + off, s));
            off += sd.n_rows;
        }
    }
    double *C = d->coef.as<double>();
    DPM_RET(lsq_apply<T>(d->lsq, bv, (int)m, C, 2, s));
    std::vector<ApRhs<T>> g[2];
    ApParams pg[2];
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = d->sub[l];
        const int64_t n = sd.gi.n_gamma;
        T *dn = sd.dens.as<T>();
        DPM_RET(dd2_extend<T>(n, d->prm.MZ, d->prm.MG, dd2_gamma_series(d->prm), sd.flags.as<uint8_t>(), sd.dG.as<double>(), sd.dZ.as<double>(),
                              sd.YG.as<double>(), sd.YZ.as<double>(), C, d->ncol, nullptr, dn, (int)n, 2, k->clamp, s));
        g[l] = {{sd.frho.as<T>(), dn, sd.rho.as<T>(), nullptr, 0, 0},
                {sd.fc.as<T>(), dn + n, sd.c.as<T>(), nullptr, 0, 0}};
        pg[l] = dd2_ap(sd, sigma);
        pg[l].fscale = sigma;
    }
    DPM_RET(dd_run_pair<T>(d->sub[0].prec, pg[0], g[0], d->sub[0].work, d->sub[0].desc, d->sub[1].prec, pg[1],
                           g[1], d->sub[1].work, d->sub[1].desc, d->gwork, d->gitems, s));
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = d->sub[l];
        DPM_RET(pks_diag<T>(sd.N, sd.gi.lo, sd.gi.h, sd.gi.labels.as<uint8_t>(), sd.rho.as<T>(), sd.c.as<T>(),
                            sd.diag_part.as<double>(), sd.diag_out.as<double>(), s, sd.origin));
    }
    k->t += dt;
    k->dt_prev = dt;
    k->step += 1;
    k->last_rebuilt = rebuild ? 1 : 0;
    return DPM_OK;
}

}  // namespace

namespace {

// The device-resident Case 2 step, as dd_step_dev for Case 1 (same kernels and
// arithmetic as dd2_pks_step; dt and sigma on the device).
template <class T> int dd2_dev_setup(dpm_dd2_pks *k, cudaStream_t s) {
    dpm_dd2 *d = &k->dd;
    const int need = (d->factored && k->dt_prev > 0 && d->sigma == 1.0 / k->dt_prev) ? 0 : 1;
    DPM_RET(k->gs.push(k->t, k->dt_prev, k->step, k->last_rebuilt, need, s));
    const StepScalars *sc = k->gs.sc();
    k->subs.assign(2, SubSolve{});
    std::vector<std::vector<std::vector<ApRhs<T>>>> rhs(3, std::vector<std::vector<ApRhs<T>>>(2));
    const bool rebuild = k->dt_mode == 1 || k->rebuild;  // batch 0 is needed
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = d->sub[l];
        ApParams p = dd2_ap(sd, 0.0);
        p.sigma_dev = &sc->sigma;
        p.fscale_dev = &sc->sigma;  // L_{h,dt} u = f  <=>  (1/dt - Lap_h) u = f/dt
        k->subs[l] = {sd.prec, p, &sd.work};
        const int64_t n = sd.gi.n_gamma, g = sd.gi.n_gin;
        T *trp = sd.trace.as<T>() + (int64_t)d->ncol * g, *dn = sd.dens.as<T>();
        std::vector<ApRhs<T>> part = {{sd.frho.as<T>(), nullptr, nullptr, trp, 0, 0},
                                      {sd.fc.as<T>(), nullptr, nullptr, trp + g, 0, 0}};
        if (rebuild) {
            for (int j = 0; j < d->ncol; ++j)
                rhs[0][l].push_back({nullptr, sd.psi.as<T>() + j * n, nullptr, sd.trace.as<T>() + j * g, 0, 0});
            for (auto &e : part) rhs[0][l].push_back(e);
        }
        rhs[1][l] = part;
        rhs[2][l] = {{sd.frho.as<T>(), dn, sd.rho.as<T>(), nullptr, 0, 0},
                     {sd.fc.as<T>(), dn + n, sd.c.as<T>(), nullptr, 0, 0}};
    }
    return prepare_batches<T>(k->subs, rhs, k->batch, d->gwork, s);
}

template <class T> int dd2_step_dev(dpm_dd2_pks *k, cudaStream_t s) {
    dpm_dd2 *d = &k->dd;
    StepScalars *sc = k->gs.sc();
    StepGrids gr;
    gr.n = 2;
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = d->sub[l];
        if (k->dt_mode == 1)
            DPM_RET(pks_cfl<T>(sd.N, sd.gi.labels.as<uint8_t>(), sd.c.as<T>(), sd.gmax.as<unsigned long long>(), s));
        gr.gmax[l] = sd.gmax.as<unsigned long long>();
        gr.h[l] = sd.gi.h;
    }
    DPM_RET(pks_step_dt_grids(gr, k->chi, k->dt_max, k->dt_mode, sc, s));
    T *trp[2];
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = d->sub[l];
        DPM_RET(pks_flux<T>(sd.N, sd.gi.h, k->chi, 0.0, &sc->dt, sd.gi.labels.as<uint8_t>(), sd.rho.as<T>(),
                            sd.c.as<T>(), sd.frho.as<T>(), sd.fc.as<T>(), s));
        trp[l] = sd.trace.as<T>() + (int64_t)d->ncol * sd.gi.n_gin;
    }
    const bool cond = k->dt_mode == 1 && !k->rebuild;  // Step 4b decided on the device
    const bool rebuild = k->rebuild != 0;
    auto with_rebuild = [&](cudaStream_t st) -> int {
        DPM_RET(run_prepared<T>(k->batch[0], k->subs, st));
        const DD2Sub &a = d->sub[0], &b = d->sub[1];
        DPM_RET(dd2_assemble<T>(a.n_rows, b.n_rows, d->ncol, a.own.as<double>(), a.trace.as<T>(), a.gi.n_gin,
                                a.row_i.as<int>(), b.own.as<double>(), b.trace.as<T>(), b.gi.n_gin,
                                b.row_i.as<int>(), d->lsq.A.as<double>(), st));
        return lsq_factor_async(d->lsq, st);
    };
    auto particular_only = [&](cudaStream_t st) -> int { return run_prepared<T>(k->batch[1], k->subs, st); };
    if (cond) DPM_RET(step_branch(sc, s, k->gs.aux, with_rebuild, particular_only));
    else if (rebuild) DPM_RET(with_rebuild(s));
    else DPM_RET(particular_only(s));
    const int64_t m = d->sub[0].n_rows + d->sub[1].n_rows;
    T *bv = d->bvec.as<T>();
    for (int f = 0; f < 2; ++f) {
        int64_t off = 0;
        for (int l = 0; l < 2; ++l) {
            DD2Sub &sd = d->sub[l];
            DPM_RET(dd2_rhs<T>(sd.n_rows, sd.row_i.as<int>(), sd.row_e.as<int>(), sd.row_s.as<uint8_t>(),
                               trp[l] + f * sd.gi.n_gin, nullptr, nullptr, bv + f * m + off, s));
            off += sd.n_rows;
        }
    }
    double *C = d->coef.as<double>();
    DPM_RET(lsq_apply<T>(d->lsq, bv, (int)m, C, 2, s));
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = d->sub[l];
        const int64_t n = sd.gi.n_gamma;
        DPM_RET(dd2_extend<T>(n, d->prm.MZ, d->prm.MG, dd2_gamma_series(d->prm), sd.flags.as<uint8_t>(),
                              sd.dG.as<double>(), sd.dZ.as<double>(), sd.YG.as<double>(), sd.YZ.as<double>(), C,
                              d->ncol, nullptr, sd.dens.as<T>(), (int)n, 2, k->clamp, s));
    }
    DPM_RET(run_prepared<T>(k->batch[2], k->subs, s));
    for (int l = 0; l < 2; ++l) {
        DD2Sub &sd = d->sub[l];
        DPM_RET(pks_diag<T>(sd.N, sd.gi.lo, sd.gi.h, sd.gi.labels.as<uint8_t>(), sd.rho.as<T>(), sd.c.as<T>(),
                            sd.diag_part.as<double>(), sd.diag_out.as<double>(), s, sd.origin));
    }
    DPM_RET(pks_step_end(sc, cond ? -1 : (rebuild ? 1 : 0), s));
    return DPM_OK;
}

}  // namespace

extern "C" int dpm_dd2_pks_set_graph(dpm_dd2_pks *k, int on, cudaStream_t s) {
    if (!k) { set_error("pks is NULL"); return DPM_EINVAL; }
    dpm_dd2 *d = &k->dd;
    const bool f64 = d->storage == DPM_PREC_FP64;
    if (on) {
        if (k->gs.on) return DPM_OK;
        DPM_CUDA(cudaSetDevice(d->ctx->device));
        if (k->dt_mode == 0 && !k->rebuild && (!d->factored || d->sigma != 1.0 / k->dt_max)) {
            // the fixed-dt step solves against the stacked BEP of sigma = 1/dt_max
            const double sg = 1.0 / k->dt_max;
            if (f64) DPM_RET(dd2_build_bep<double>(d, sg, nullptr, sg, s));
            else DPM_RET(dd2_build_bep<float>(d, sg, nullptr, sg, s));
        }
        if (f64) DPM_RET(dd2_dev_setup<double>(k, s));
        else DPM_RET(dd2_dev_setup<float>(k, s));
        k->gs.on = 1;
        return DPM_OK;
    }
    if (!k->gs.on) return DPM_OK;
    int bad = 0;
    DPM_RET(k->gs.pull(k->t, k->dt_prev, k->step, k->last_rebuilt, &bad, s));
    k->gs.stop();
    d->factored = true;
    d->sigma = 1.0 / k->dt_prev;
    return DPM_OK;
}

extern "C" int dpm_dd2_pks_create(dpm_ctx *ctx, const dpm_dd2_params *P, double chi, double dt_max, int dt_mode,
                                  int rebuild, int clamp, const dpm_gaussian *rho0, const dpm_gaussian *c0,
                                  dpm_dd2_pks **out, cudaStream_t s) {
    if (!ctx || !out) { set_error("ctx/out is NULL"); return DPM_EINVAL; }
    *out = nullptr;
    DPM_RET(dd2_check(P));
    if (!(dt_max > 0) || !(chi >= 0) || (dt_mode != 0 && dt_mode != 1)) {
        set_error("need dt_max > 0, chi >= 0, dt_mode in {0,1}");
        return DPM_EINVAL;
    }
    DPM_CUDA(cudaSetDevice(ctx->device));
    dpm_dd2_pks *k = new (std::nothrow) dpm_dd2_pks();
    if (!k) { set_error("out of host memory"); return DPM_ENOMEM; }
    k->chi = chi;
    k->dt_max = dt_max;
    k->dt_mode = dt_mode;
    k->rebuild = rebuild;
    k->clamp = clamp;
    dpm_gaussian z{};
    const dpm_gaussian &g0 = rho0 ? *rho0 : z, &g1 = c0 ? *c0 : z;
    int r;
    if (P->precision == DPM_PREC_FP64) {
        r = dd2_init<double>(&k->dd, ctx, *P, s);
        if (r == DPM_OK) r = dd2_pks_alloc<double>(k, g0, g1, s);
    } else {
        r = dd2_init<float>(&k->dd, ctx, *P, s);
        if (r == DPM_OK) r = dd2_pks_alloc<float>(k, g0, g1, s);
    }
    if (r == DPM_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_error("%s", cudaGetErrorString(e)); r = DPM_ECUDA; }
    }
    if (r != DPM_OK) { delete k; return r; }
    *out = k;
    return DPM_OK;
}

extern "C" int dpm_dd2_pks_step(dpm_dd2_pks *k, int nsteps, dpm_pks_stats *stats, cudaStream_t s) {
    if (!k || nsteps < 0) { set_error("pks is NULL or nsteps < 0"); return DPM_EINVAL; }
    const bool f64 = k->dd.storage == DPM_PREC_FP64;
    for (int i = 0; i < nsteps; ++i) {
        if (k->gs.on)
            DPM_RET(k->gs.step([&](cudaStream_t st) { return f64 ? dd2_step_dev<double>(k, st) : dd2_step_dev<float>(k, st); }, s));
        else if (f64) DPM_RET(dd2_pks_step<double>(k, s));
        else DPM_RET(dd2_pks_step<float>(k, s));
    }
    if (stats && k->gs.on) {
        int bad = 0;
        DPM_RET(k->gs.pull(k->t, k->dt_prev, k->step, k->last_rebuilt, &bad, s));
        if (bad) { set_error("time step was not positive/finite on the device"); return DPM_ENUMERIC; }
        if (k->last_rebuilt) DPM_RET(lsq_status(k->dd.lsq, s));
    }
    if (stats) {
        double dg[2][6];
        for (int l = 0; l < 2; ++l)
            DPM_CUDA(cudaMemcpyAsync(dg[l], k->dd.sub[l].diag_out.p, sizeof(dg[l]), cudaMemcpyDeviceToHost, s));
        DPM_CUDA(cudaStreamSynchronize(s));
        stats->t = k->t;
        stats->dt = k->dt_prev;
        stats->step = k->step;
        stats->rebuilt = k->last_rebuilt;
        stats->mass = dg[0][0] + dg[1][0];
        stats->max_rho = std::max(dg[0][1], dg[1][1]);
        stats->min_rho = std::min(dg[0][2], dg[1][2]);
        stats->min_c = std::min(dg[0][3], dg[1][3]);
        stats->m2 = dg[0][4] + dg[1][4];
        stats->free_energy = dg[0][5] + dg[1][5];
        if (k->dd.prm.precision == DPM_PREC_TC32) DPM_RET(tc_status_check());
        if (!std::isfinite(stats->mass) || !std::isfinite(stats->free_energy)) {
            set_error("PKS state became non-finite at step %lld", (long long)k->step);
            return DPM_ENUMERIC;
        }
    }
    return DPM_OK;
}

extern "C" int dpm_dd2_pks_get_state(dpm_dd2_pks *k, int l, void *rho, void *c, cudaStream_t s) {
    if (!k || l < 0 || l > 1) { set_error("pks is NULL or sub-domain index not 0/1"); return DPM_EINVAL; }
    const DD2Sub &sd = k->dd.sub[l];
    const size_t n3 = (size_t)sd.N * sd.N * sd.N * elem_size(k->dd.storage);
    if (rho) DPM_CUDA(cudaMemcpyAsync(rho, sd.rho.p, n3, cudaMemcpyDeviceToDevice, s));
    if (c) DPM_CUDA(cudaMemcpyAsync(c, sd.c.p, n3, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

extern "C" int dpm_dd2_pks_destroy(dpm_dd2_pks *k) {
    delete k;
    return DPM_OK;
}

// ---------------------------------------------------------------------------
// Layered domain decomposition: the ball and L - 1 concentric shells, each on
// its own grid; one shared 3-term series per interface, the 2-term series on
// Gamma; the stacked (block-banded) reduced BEPs in one least squares.
// ---------------------------------------------------------------------------
namespace {
struct MLSub {
    int N = 0, prec = 0, ncl = 0;
    double lo = 0, hi = 0;
    dpm_geom geom{};
    GridIndex gi;
    GammaGeom gg;
    DevBuf sphere, cols, psi, psi_in, trace, dens, work, desc;
    DevBuf rho, c, frho, fc, gmax, diag_part, diag_out;
};
}  // namespace

struct dpm_ml {
    dpm_ctx *ctx = nullptr;
    dpm_ml_params prm{};
    MLSub sub[DPM_ML_MAX];
    int L = 0;
    MlColumns cm{};
    int ncol = 0, storage = 0;
    double sigma = 0;
    bool factored = false;
    LsqFactor lsq;
    DevBuf coef, bvec, gwork, gitems;
};

struct dpm_ml_pks {
    dpm_ml ml;
    double chi = 0, dt_max = 0;
    int dt_mode = 0, rebuild = 0, clamp = 1;
    double t = 0, dt_prev = 0;
    int64_t step = 0;
    int last_rebuilt = 0;
    // device-resident steps replayed as a CUDA graph (dpm_ml_pks_set_graph):
    // batch 0 the BEP columns + the particular solutions, 1 the particular
    // solutions, 2 Green's formula
    GraphStepper gs;
    PreparedBatch batch[3];
    std::vector<SubSolve> subs;
};

namespace {

int ml_check(const dpm_ml_params *P) {
    if (!P) { set_error("params is NULL"); return DPM_EINVAL; }
    if (P->L < 2 || P->L > DPM_ML_MAX) { set_error("L must be in [2, %d]", DPM_ML_MAX); return DPM_EINVAL; }
    for (int l = 0; l < P->L; ++l) {
        if (!(P->radii[l] > (l ? P->radii[l - 1] : 0.0))) { set_error("radii must increase from > 0"); return DPM_EINVAL; }
        if (P->N[l] < 6 || P->N[l] > 256) { set_error("N[%d] = %d outside [6, 256]", l, P->N[l]); return DPM_EINVAL; }
        if (l < P->L - 1 && (P->K[l] < 0 || P->K[l] > 16)) { set_error("K in [0, 16]"); return DPM_EINVAL; }
    }
    if (P->KG < 0 || P->KG > 16) { set_error("KG in [0, 16]"); return DPM_EINVAL; }
    if (!prec_ok(P->precision)) { set_error("unknown precision %d", P->precision); return DPM_EINVAL; }
    return DPM_OK;
}

ApParams ml_ap(const MLSub &sd, double sigma) {
    ApParams p;
    p.N = sd.N;
    p.h = sd.gi.h;
    p.sigma = sigma;
    ap_params_from_index(p, sd.gi);
    return p;
}

// One batched solve per sub-domain, the SIMT grids' right-hand sides in one
// grouped set of launches (DPM_DD_GROUP=0: one batch each).
template <class T>
int ml_run(dpm_ml *d, const std::vector<ApParams> &prm, const std::vector<std::vector<ApRhs<T>>> &rhs, cudaStream_t s) {
    const char *env = getenv("DPM_DD_GROUP");
    const bool group = !(env && env[0] == '0');
    std::vector<ApParams> gp;
    std::vector<ApRhs<T>> gr;
    std::vector<int> gof;
    for (size_t l = 0; l < d->L; ++l) {
        MLSub &sd = d->sub[l];
        if (rhs[l].empty()) continue;
        const bool simt = sd.prec == DPM_PREC_FP32 || sd.prec == DPM_PREC_FP64;
        if (group && simt) {
            gp.push_back(prm[l]);
            gr.insert(gr.end(), rhs[l].begin(), rhs[l].end());
            gof.resize(gr.size(), (int)gp.size() - 1);
        } else {
            DPM_RET(run_ap<T>(sd.prec, prm[l], rhs[l], sd.work, sd.desc, s));
        }
    }
    if (!gr.empty()) DPM_RET(ap_solve_simt_group<T>(gp, gr, gof, d->gwork, d->gitems, s));
    return DPM_OK;
}

// Extension operator (eq. extension_operator) onto sub-domain l's grid boundary: its
// spheres' series, in FP32 sums for FP32 storage (the FP32 harmonic table is
// built on first use), FP64 otherwise; densities at dens + q n, q < nr.
template <class T>
int ml_extend_sub(dpm_ml *d, int l, const double *C, const double *gn, T *dens, int nr, int clamp, cudaStream_t s) {
    MLSub &sd = d->sub[l];
    const int64_t n = sd.gi.n_gamma;
    const float *phit = nullptr;
    if (sizeof(T) == 4) {
        DPM_RET(gamma_phi32(sd.gg, n, s));
        phit = sd.gg.phi32.as<float>();
    }
    return ml_extend<T>(n, sd.gg.nsh, d->cm, sd.sphere.as<uint8_t>(), sd.gg.dist.as<double>(), sd.gg.phi.as<double>(),
                        phit, l == 0 ? 1 : l, l + 1, C, d->ncol, gn, dens, (int)n, nr, clamp, s);
}

template <class T> int ml_init(dpm_ml *d, dpm_ctx *ctx, const dpm_ml_params &P, cudaStream_t s) {
    d->ctx = ctx;
    d->prm = P;
    d->storage = P.precision == DPM_PREC_FP64 ? DPM_PREC_FP64 : DPM_PREC_FP32;
    const int L = P.L;
    MlColumns &cm = d->cm;
    cm.L = L;
    cm.off[0] = 0;
    int Kmax = P.KG;
    for (int m = 1; m <= L; ++m) {
        const int K = m < L ? P.K[m - 1] : P.KG;
        Kmax = std::max(Kmax, K);
        cm.n[m - 1] = (K + 1) * (K + 1);
        cm.off[m] = cm.off[m - 1] + (m < L ? 3 : 2) * cm.n[m - 1];
    }
    d->ncol = cm.off[L];
    d->L = L;
    int64_t mtot = 0;
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        sd.geom.kind = l == 0 ? 0 : 2;
        for (int t = 0; t < 3; ++t) sd.geom.center[t] = P.center[t];
        sd.geom.axes[0] = P.radii[l];
        sd.geom.axes[1] = l == 0 ? P.radii[0] : P.radii[l - 1];
        sd.geom.axes[2] = l == 0 ? P.radii[0] : 0.0;
        sd.N = P.N[l];
        sd.lo = P.lo[l];
        sd.hi = P.hi[l];
        sd.prec = dd_sub_prec(P.precision, sd.N);
        DPM_RET(build_grid_index(sd.geom, sd.N, sd.lo, sd.hi, sd.gi, s));
        DPM_RET(build_gamma_geom(sd.geom, sd.gi, Kmax, sd.gg, s));
        const int64_t n = sd.gi.n_gamma, m = sd.gi.n_gin;
        DPM_RET(sd.sphere.alloc(std::max<int64_t>(n, 1)));
        const double rmid = l == 0 ? 2.0 * P.radii[0] : 0.5 * (P.radii[l - 1] + P.radii[l]);
        DPM_RET(ml_sphere_flags(n, sd.gg.foot.as<double>(), P.center, rmid, l, l == 0 ? 1 : 0, sd.sphere.as<uint8_t>(), s));
        // the columns of this sub-domain's spheres: 1 for the ball, l and l + 1 for shell l
        std::vector<int> cols;
        const int m0 = l == 0 ? 1 : l, m1 = l + 1;
        for (int q = m0; q <= m1; ++q)
            for (int k = cm.off[q - 1]; k < cm.off[q]; ++k) cols.push_back(k);
        sd.ncl = (int)cols.size();
        DPM_RET(sd.cols.alloc(sizeof(int) * sd.ncl));
        DPM_CUDA(cudaMemcpyAsync(sd.cols.p, cols.data(), sizeof(int) * sd.ncl, cudaMemcpyHostToDevice, s));
        DPM_RET(sd.psi.alloc(sizeof(T) * sd.ncl * std::max<int64_t>(n, 1)));
        DPM_RET(sd.psi_in.alloc(sizeof(double) * sd.ncl * std::max<int64_t>(m, 1)));
        DPM_RET(ml_columns<T>(n, m, sd.gg.nsh, cm, sd.ncl, sd.cols.as<int>(), sd.sphere.as<uint8_t>(),
                              sd.gg.dist.as<double>(), sd.gg.phi.as<double>(), sd.gi.gin_pos.as<int>(), sd.psi.as<T>(),
                              sd.psi_in.as<double>(), s));
        DPM_RET(sd.trace.alloc(sizeof(T) * (sd.ncl + 4) * std::max<int64_t>(m, 1)));
        DPM_RET(sd.dens.alloc(sizeof(T) * 4 * std::max<int64_t>(n, 1)));
        DPM_CUDA(cudaStreamSynchronize(s));  // `cols` goes out of scope
        mtot += m;
    }
    if (mtot < d->ncol) {
        set_error("%lld BEP rows for %d unknowns: refine the grids or lower K", (long long)mtot, d->ncol);
        return DPM_EINVAL;
    }
    d->lsq.m = (int)mtot;
    d->lsq.n = d->ncol;
    DPM_RET(d->lsq.A.alloc(sizeof(double) * mtot * d->ncol));
    DPM_RET(d->coef.alloc(sizeof(double) * 4 * d->ncol));
    DPM_RET(d->bvec.alloc(sizeof(T) * 4 * mtot));
    // the stacked matrix is block-banded: sub-domain l's rows meet only the
    // series of its own spheres (the ball: sphere 1; shell l: spheres l, l + 1)
    std::vector<int64_t> row0(1, 0);
    std::vector<int> c0, c1;
    for (int l = 0; l < L; ++l) {
        const int m0 = l == 0 ? 1 : l, m1 = l + 1;
        row0.push_back(row0.back() + d->sub[l].gi.n_gin);
        c0.push_back(cm.off[m0 - 1]);
        c1.push_back(cm.off[m1]);
    }
    DPM_RET(lsq_set_band(d->lsq, row0, c0, c1, s));
    return DPM_OK;
}

template <class T>
int ml_build_bep(dpm_ml *d, double sigma, const std::vector<std::vector<ApRhs<T>>> *extra, double fscale, cudaStream_t s) {
    const int L = (int)d->L;
    std::vector<ApParams> prm(L);
    std::vector<std::vector<ApRhs<T>>> rhs(L);
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        const int64_t n = sd.gi.n_gamma, m = sd.gi.n_gin;
        for (int j = 0; j < sd.ncl; ++j)
            rhs[l].push_back({nullptr, sd.psi.as<T>() + j * n, nullptr, sd.trace.as<T>() + j * m, 0, 0});
        if (extra)
            for (auto &e : (*extra)[l]) rhs[l].push_back(e);
        prm[l] = ml_ap(sd, sigma);
        prm[l].fscale = fscale;
    }
    DPM_RET(ml_run<T>(d, prm, rhs, s));
    const int64_t mtot = d->lsq.m;
    DPM_CUDA(cudaMemsetAsync(d->lsq.A.p, 0, sizeof(double) * mtot * d->ncol, s));
    int64_t row0 = 0;
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        DPM_RET(ml_assemble<T>(sd.gi.n_gin, sd.ncl, mtot, row0, sd.cols.as<int>(), sd.psi_in.as<double>(),
                               sd.trace.as<T>(), d->lsq.A.as<double>(), s));
        row0 += sd.gi.n_gin;
    }
    DPM_RET(lsq_factor(d->lsq, nullptr, s));
    d->sigma = sigma;
    d->factored = true;
    return DPM_OK;
}

template <class T>
int ml_solve(dpm_ml *d, const void *const *fv, const double *gn, void *const *uv, double *coeffs, cudaStream_t s) {
    const int L = (int)d->L;
    std::vector<ApParams> prm(L);
    std::vector<std::vector<ApRhs<T>>> rhs(L);
    MLSub &last = d->sub[L - 1];
    T *v = last.dens.as<T>() + last.gi.n_gamma;
    if (gn) DPM_RET(ml_neumann<T>(last.gi.n_gamma, L, last.sphere.as<uint8_t>(), last.gg.dist.as<double>(), gn, v, s));
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        const int64_t m = sd.gi.n_gin;
        T *trp = sd.trace.as<T>() + (int64_t)sd.ncl * m;
        rhs[l].push_back({static_cast<const T *>(fv[l]), nullptr, nullptr, trp, 0, 0});
        if (l == L - 1 && gn) rhs[l].push_back({nullptr, v, nullptr, trp + m, 0, 0});
        prm[l] = ml_ap(sd, d->sigma);
    }
    DPM_RET(ml_run<T>(d, prm, rhs, s));
    T *bv = d->bvec.as<T>();
    int64_t row0 = 0;
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        const int64_t m = sd.gi.n_gin;
        T *trp = sd.trace.as<T>() + (int64_t)sd.ncl * m;
        const bool nm = l == L - 1 && gn;
        DPM_RET(ml_rhs<T>(m, trp, nm ? v : nullptr, sd.gi.gin_pos.as<int>(), trp + m, bv + row0, s));
        row0 += m;
    }
    double *C = d->coef.as<double>();
    DPM_RET(lsq_apply<T>(d->lsq, bv, (int)row0, C, 1, s));
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        DPM_RET(ml_extend_sub<T>(d, l, C, l == L - 1 ? gn : nullptr, sd.dens.as<T>(), 1, 0, s));
        rhs[l] = {{static_cast<const T *>(fv[l]), sd.dens.as<T>(), static_cast<T *>(uv[l]), nullptr, 0, 0}};
    }
    DPM_RET(ml_run<T>(d, prm, rhs, s));
    if (coeffs) DPM_CUDA(cudaMemcpyAsync(coeffs, C, sizeof(double) * d->ncol, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

}  // namespace

extern "C" int dpm_ml_build(dpm_ctx *ctx, const dpm_ml_params *P, double sigma, dpm_ml **out, cudaStream_t s) {
    if (!ctx || !out) { set_error("ctx/out is NULL"); return DPM_EINVAL; }
    *out = nullptr;
    DPM_RET(ml_check(P));
    if (!(sigma > 0)) { set_error("sigma must be > 0"); return DPM_EINVAL; }
    DPM_CUDA(cudaSetDevice(ctx->device));
    dpm_ml *d = new (std::nothrow) dpm_ml();
    if (!d) { set_error("out of host memory"); return DPM_ENOMEM; }
    int r;
    if (P->precision == DPM_PREC_FP64) {
        r = ml_init<double>(d, ctx, *P, s);
        if (r == DPM_OK) r = ml_build_bep<double>(d, sigma, nullptr, 1.0, s);
    } else {
        r = ml_init<float>(d, ctx, *P, s);
        if (r == DPM_OK) r = ml_build_bep<float>(d, sigma, nullptr, 1.0, s);
    }
    if (r == DPM_OK && P->precision == DPM_PREC_TC32) r = tc_status_check();
    if (r != DPM_OK) { delete d; return r; }
    *out = d;
    return DPM_OK;
}

extern "C" int dpm_ml_get_info(const dpm_ml *d, dpm_ml_info *info) {
    if (!d || !info) { set_error("ml/info is NULL"); return DPM_EINVAL; }
    *info = dpm_ml_info{};
    info->L = (int)d->L;
    for (size_t l = 0; l < d->L; ++l) {
        const MLSub &sd = d->sub[l];
        info->N[l] = sd.N;
        info->h[l] = sd.gi.h;
        info->precision[l] = sd.prec;
        info->n_mplus[l] = sd.gi.n_mplus;
        info->n_gin[l] = sd.gi.n_gin;
        info->n_gamma[l] = sd.gi.n_gamma;
    }
    info->ncol = d->ncol;
    info->sigma = d->sigma;
    return DPM_OK;
}

extern "C" int dpm_ml_matrix(dpm_ml *d, double *A, cudaStream_t s) {
    if (!d || !A) { set_error("ml/A is NULL"); return DPM_EINVAL; }
    DPM_CUDA(cudaMemcpyAsync(A, d->lsq.A.p, sizeof(double) * (size_t)d->lsq.m * d->ncol, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

extern "C" int dpm_ml_solve(dpm_ml *d, const void *const *f, const double *neumann, void *const *u, double *coeffs,
                            cudaStream_t s) {
    if (!d || !f || !u) { set_error("ml/f/u is NULL"); return DPM_EINVAL; }
    for (size_t l = 0; l < d->L; ++l)
        if (!f[l] || !u[l]) { set_error("f[%zu]/u[%zu] is NULL", l, l); return DPM_EINVAL; }
    int r = d->storage == DPM_PREC_FP64 ? ml_solve<double>(d, f, neumann, u, coeffs, s)
                                        : ml_solve<float>(d, f, neumann, u, coeffs, s);
    if (r == DPM_OK && d->prm.precision == DPM_PREC_TC32) r = tc_status_check();
    return r;
}

extern "C" int dpm_ml_destroy(dpm_ml *d) {
    delete d;
    return DPM_OK;
}

namespace {

template <class T> int ml_pks_alloc(dpm_ml_pks *k, const dpm_gaussian &g0, const dpm_gaussian &g1, cudaStream_t s) {
    for (int l = 0; l < k->ml.L; ++l) {
        MLSub &sd = k->ml.sub[l];
        const size_t n3 = (size_t)sd.N * sd.N * sd.N;
        DPM_RET(sd.rho.alloc(sizeof(T) * n3));
        DPM_RET(sd.c.alloc(sizeof(T) * n3));
        DPM_RET(sd.frho.alloc(sizeof(T) * n3));
        DPM_RET(sd.fc.alloc(sizeof(T) * n3));
        DPM_RET(sd.gmax.alloc(sizeof(unsigned long long) * 4));
        DPM_RET(sd.diag_part.alloc(sizeof(double) * 6 * pks_diag_blocks(sd.N)));
        DPM_RET(sd.diag_out.alloc(sizeof(double) * 8));
        DPM_CUDA(cudaMemsetAsync(sd.diag_out.p, 0, sizeof(double) * 8, s));
        DPM_RET(pks_init<T>(sd.gi, sd.gg, g0, g1, sd.rho.as<T>(), sd.c.as<T>(), s));
    }
    return DPM_OK;
}

template <class T> int ml_pks_step(dpm_ml_pks *k, cudaStream_t s) {
    dpm_ml *d = &k->ml;
    const int L = (int)d->L;
    double dt = k->dt_max;
    if (k->dt_mode == 1) {
        std::vector<double> gm(3 * L);
        for (int l = 0; l < L; ++l) {
            MLSub &sd = d->sub[l];
            DPM_RET(pks_cfl<T>(sd.N, sd.gi.labels.as<uint8_t>(), sd.c.as<T>(), sd.gmax.as<unsigned long long>(), s));
            DPM_CUDA(cudaMemcpyAsync(gm.data() + 3 * l, sd.gmax.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
        DPM_CUDA(cudaStreamSynchronize(s));
        for (int l = 0; l < L; ++l) {
            const double h = d->sub[l].gi.h;
            for (int ax = 0; ax < 3; ++ax) {
                const double gmaxv = gm[3 * l + ax] / h;
                if (gmaxv > 0) dt = std::min(dt, h / (6.0 * k->chi * gmaxv));
            }
        }
        if (k->step > 0) dt = std::min(dt, k->dt_prev);
    }
    if (!(dt > 0) || !std::isfinite(dt)) { set_error("time step is not positive/finite (dt=%g)", dt); return DPM_ENUMERIC; }
    const bool rebuild = !d->factored || k->rebuild || dt < k->dt_prev;
    const double sigma = 1.0 / dt;
    std::vector<std::vector<ApRhs<T>>> part(L);
    std::vector<ApParams> prm(L);
    std::vector<T *> trp(L);
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        const int64_t m = sd.gi.n_gin;
        DPM_RET(pks_flux<T>(sd.N, sd.gi.h, k->chi, dt, nullptr, sd.gi.labels.as<uint8_t>(), sd.rho.as<T>(), sd.c.as<T>(),
                            sd.frho.as<T>(), sd.fc.as<T>(), s));
        trp[l] = sd.trace.as<T>() + (int64_t)sd.ncl * m;
        part[l] = {{sd.frho.as<T>(), nullptr, nullptr, trp[l], 0, 0}, {sd.fc.as<T>(), nullptr, nullptr, trp[l] + m, 0, 0}};
        prm[l] = ml_ap(sd, sigma);
        prm[l].fscale = sigma;  // L_{h,dt} u = f  <=>  (1/dt - Lap_h) u = f/dt
    }
    if (rebuild) DPM_RET(ml_build_bep<T>(d, sigma, &part, sigma, s));
    else DPM_RET(ml_run<T>(d, prm, part, s));
    const int64_t mtot = d->lsq.m;
    T *bv = d->bvec.as<T>();
    for (int f = 0; f < 2; ++f) {
        int64_t row0 = 0;
        for (int l = 0; l < L; ++l) {
            MLSub &sd = d->sub[l];
            const int64_t m = sd.gi.n_gin;
            DPM_RET(ml_rhs<T>(m, trp[l] + f * m, nullptr, nullptr, nullptr, bv + f * mtot + row0, s));
            row0 += m;
        }
    }
    double *C = d->coef.as<double>();
    DPM_RET(lsq_apply<T>(d->lsq, bv, (int)mtot, C, 2, s));
    std::vector<std::vector<ApRhs<T>>> g(L);
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        const int64_t n = sd.gi.n_gamma;
        T *dn = sd.dens.as<T>();
        DPM_RET(ml_extend_sub<T>(d, l, C, nullptr, dn, 2, k->clamp, s));
        g[l] = {{sd.frho.as<T>(), dn, sd.rho.as<T>(), nullptr, 0, 0}, {sd.fc.as<T>(), dn + n, sd.c.as<T>(), nullptr, 0, 0}};
    }
    DPM_RET(ml_run<T>(d, prm, g, s));
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        DPM_RET(pks_diag<T>(sd.N, sd.gi.lo, sd.gi.h, sd.gi.labels.as<uint8_t>(), sd.rho.as<T>(), sd.c.as<T>(),
                            sd.diag_part.as<double>(), sd.diag_out.as<double>(), s));
    }
    k->t += dt;
    k->dt_prev = dt;
    k->step += 1;
    k->last_rebuilt = rebuild ? 1 : 0;
    return DPM_OK;
}

// The device-resident layered step (no host synchronisation, allocation or
// copy: capturable).  Same kernels and arithmetic as ml_pks_step, with dt and
// sigma on the device; the stacked BEP is rebuilt on every step unless dt is
// fixed (dt_mode 0 without rebuild).
template <class T> std::vector<ApRhs<T>> ml_part_rhs(MLSub &sd) {
    const int64_t m = sd.gi.n_gin;
    T *trp = sd.trace.as<T>() + (int64_t)sd.ncl * m;
    return {{sd.frho.as<T>(), nullptr, nullptr, trp, 0, 0}, {sd.fc.as<T>(), nullptr, nullptr, trp + m, 0, 0}};
}

template <class T> std::vector<ApRhs<T>> ml_green_rhs(MLSub &sd) {
    const int64_t n = sd.gi.n_gamma;
    T *dn = sd.dens.as<T>();
    return {{sd.frho.as<T>(), dn, sd.rho.as<T>(), nullptr, 0, 0}, {sd.fc.as<T>(), dn + n, sd.c.as<T>(), nullptr, 0, 0}};
}

ApParams ml_ap_dev(const MLSub &sd, const StepScalars *sc) {
    ApParams p = ml_ap(sd, 0.0);
    p.sigma_dev = &sc->sigma;
    p.fscale_dev = &sc->sigma;  // L_{h,dt} u = f  <=>  (1/dt - Lap_h) u = f/dt
    return p;
}

template <class T> int ml_dev_setup(dpm_ml_pks *k, cudaStream_t s) {
    dpm_ml *d = &k->ml;
    const int L = (int)d->L;
    const int need = (d->factored && k->dt_prev > 0 && d->sigma == 1.0 / k->dt_prev) ? 0 : 1;
    DPM_RET(k->gs.push(k->t, k->dt_prev, k->step, k->last_rebuilt, need, s));
    const StepScalars *sc = k->gs.sc();
    k->subs.assign(L, SubSolve{});
    for (int l = 0; l < L; ++l) k->subs[l] = {d->sub[l].prec, ml_ap_dev(d->sub[l], sc), &d->sub[l].work};
    const bool rebuild = k->dt_mode == 1 || k->rebuild;  // batch 0 is needed
    std::vector<std::vector<std::vector<ApRhs<T>>>> rhs(3, std::vector<std::vector<ApRhs<T>>>(L));
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        const int64_t n = sd.gi.n_gamma, m = sd.gi.n_gin;
        if (rebuild) {
            for (int j = 0; j < sd.ncl; ++j)
                rhs[0][l].push_back({nullptr, sd.psi.as<T>() + j * n, nullptr, sd.trace.as<T>() + j * m, 0, 0});
            for (auto &e : ml_part_rhs<T>(sd)) rhs[0][l].push_back(e);
        }
        rhs[1][l] = ml_part_rhs<T>(sd);
        rhs[2][l] = ml_green_rhs<T>(sd);
    }
    return prepare_batches<T>(k->subs, rhs, k->batch, d->gwork, s);
}

template <class T> int ml_run_batch(dpm_ml_pks *k, int kb, cudaStream_t s) {
    return run_prepared<T>(k->batch[kb], k->subs, s);
}

template <class T> int ml_step_dev(dpm_ml_pks *k, cudaStream_t s) {
    dpm_ml *d = &k->ml;
    const int L = (int)d->L;
    StepScalars *sc = k->gs.sc();
    StepGrids g;
    g.n = L;
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        if (k->dt_mode == 1)
            DPM_RET(pks_cfl<T>(sd.N, sd.gi.labels.as<uint8_t>(), sd.c.as<T>(), sd.gmax.as<unsigned long long>(), s));
        g.gmax[l] = sd.gmax.as<unsigned long long>();
        g.h[l] = sd.gi.h;
    }
    DPM_RET(pks_step_dt_grids(g, k->chi, k->dt_max, k->dt_mode, sc, s));
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        DPM_RET(pks_flux<T>(sd.N, sd.gi.h, k->chi, 0.0, &sc->dt, sd.gi.labels.as<uint8_t>(), sd.rho.as<T>(),
                            sd.c.as<T>(), sd.frho.as<T>(), sd.fc.as<T>(), s));
    }
    const bool cond = k->dt_mode == 1 && !k->rebuild;  // Step 4b decided on the device
    const bool rebuild = k->rebuild != 0;
    const int64_t mtot = d->lsq.m;
    auto with_rebuild = [&](cudaStream_t st) -> int {
        DPM_RET(ml_run_batch<T>(k, 0, st));
        DPM_CUDA(cudaMemsetAsync(d->lsq.A.p, 0, sizeof(double) * mtot * d->ncol, st));
        int64_t row0 = 0;
        for (int l = 0; l < L; ++l) {
            MLSub &sd = d->sub[l];
            DPM_RET(ml_assemble<T>(sd.gi.n_gin, sd.ncl, mtot, row0, sd.cols.as<int>(), sd.psi_in.as<double>(),
                                   sd.trace.as<T>(), d->lsq.A.as<double>(), st));
            row0 += sd.gi.n_gin;
        }
        return lsq_factor_async(d->lsq, st);
    };
    auto particular_only = [&](cudaStream_t st) -> int { return ml_run_batch<T>(k, 1, st); };
    if (cond) DPM_RET(step_branch(sc, s, k->gs.aux, with_rebuild, particular_only));
    else if (rebuild) DPM_RET(with_rebuild(s));
    else DPM_RET(particular_only(s));
    T *bv = d->bvec.as<T>();
    for (int f = 0; f < 2; ++f) {
        int64_t row0 = 0;
        for (int l = 0; l < L; ++l) {
            MLSub &sd = d->sub[l];
            const int64_t m = sd.gi.n_gin;
            const T *trp = sd.trace.as<T>() + (int64_t)sd.ncl * m;
            DPM_RET(ml_rhs<T>(m, trp + f * m, nullptr, nullptr, nullptr, bv + f * mtot + row0, s));
            row0 += m;
        }
    }
    double *C = d->coef.as<double>();
    DPM_RET(lsq_apply<T>(d->lsq, bv, (int)mtot, C, 2, s));
    for (int l = 0; l < L; ++l) DPM_RET(ml_extend_sub<T>(d, l, C, nullptr, d->sub[l].dens.as<T>(), 2, k->clamp, s));
    DPM_RET(ml_run_batch<T>(k, 2, s));
    for (int l = 0; l < L; ++l) {
        MLSub &sd = d->sub[l];
        DPM_RET(pks_diag<T>(sd.N, sd.gi.lo, sd.gi.h, sd.gi.labels.as<uint8_t>(), sd.rho.as<T>(), sd.c.as<T>(),
                            sd.diag_part.as<double>(), sd.diag_out.as<double>(), s));
    }
    DPM_RET(pks_step_end(sc, cond ? -1 : (rebuild ? 1 : 0), s));
    return DPM_OK;
}

}  // namespace

extern "C" int dpm_ml_pks_set_graph(dpm_ml_pks *k, int on, cudaStream_t s) {
    if (!k) { set_error("pks is NULL"); return DPM_EINVAL; }
    dpm_ml *d = &k->ml;
    const bool f64 = d->storage == DPM_PREC_FP64;
    if (on) {
        if (k->gs.on) return DPM_OK;
        DPM_CUDA(cudaSetDevice(d->ctx->device));
        if (k->dt_mode == 0 && !k->rebuild && (!d->factored || d->sigma != 1.0 / k->dt_max)) {
            // the fixed-dt step solves against the stacked BEP of sigma = 1/dt_max
            const double sg = 1.0 / k->dt_max;
            if (f64) DPM_RET(ml_build_bep<double>(d, sg, nullptr, sg, s));
            else DPM_RET(ml_build_bep<float>(d, sg, nullptr, sg, s));
        }
        if (f64) DPM_RET(ml_dev_setup<double>(k, s));
        else DPM_RET(ml_dev_setup<float>(k, s));
        k->gs.on = 1;
        return DPM_OK;
    }
    if (!k->gs.on) return DPM_OK;
    int bad = 0;
    DPM_RET(k->gs.pull(k->t, k->dt_prev, k->step, k->last_rebuilt, &bad, s));
    k->gs.stop();
    d->factored = true;
    d->sigma = 1.0 / k->dt_prev;
    return DPM_OK;
}

extern "C" int dpm_ml_pks_create(dpm_ctx *ctx, const dpm_ml_params *P, double chi, double dt_max, int dt_mode, int rebuild,
                                 int clamp, const dpm_gaussian *rho0, const dpm_gaussian *c0, dpm_ml_pks **out,
                                 cudaStream_t s) {
    if (!ctx || !out) { set_error("ctx/out is NULL"); return DPM_EINVAL; }
    *out = nullptr;
    DPM_RET(ml_check(P));
    if (!(dt_max > 0) || !(chi >= 0) || (dt_mode != 0 && dt_mode != 1)) {
        set_error("need dt_max > 0, chi >= 0, dt_mode in {0,1}");
        return DPM_EINVAL;
    }
    DPM_CUDA(cudaSetDevice(ctx->device));
    dpm_ml_pks *k = new (std::nothrow) dpm_ml_pks();
    if (!k) { set_error("out of host memory"); return DPM_ENOMEM; }
    k->chi = chi;
    k->dt_max = dt_max;
    k->dt_mode = dt_mode;
    k->rebuild = rebuild;
    k->clamp = clamp;
    dpm_gaussian z{};
    const dpm_gaussian &g0 = rho0 ? *rho0 : z, &g1 = c0 ? *c0 : z;
    int r;
    if (P->precision == DPM_PREC_FP64) {
        r = ml_init<double>(&k->ml, ctx, *P, s);
        if (r == DPM_OK) r = ml_pks_alloc<double>(k, g0, g1, s);
    } else {
        r = ml_init<float>(&k->ml, ctx, *P, s);
        if (r == DPM_OK) r = ml_pks_alloc<float>(k, g0, g1, s);
    }
    if (r == DPM_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_error("%s", cudaGetErrorString(e)); r = DPM_ECUDA; }
    }
    if (r != DPM_OK) { delete k; return r; }
    *out = k;
    return DPM_OK;
}

extern "C" int dpm_ml_pks_step(dpm_ml_pks *k, int nsteps, dpm_pks_stats *stats, cudaStream_t s) {
    if (!k || nsteps < 0) { set_error("pks is NULL or nsteps < 0"); return DPM_EINVAL; }
    const bool f64 = k->ml.storage == DPM_PREC_FP64;
    for (int i = 0; i < nsteps; ++i) {
        if (k->gs.on)
            DPM_RET(k->gs.step([&](cudaStream_t st) { return f64 ? ml_step_dev<double>(k, st) : ml_step_dev<float>(k, st); }, s));
        else if (f64) DPM_RET(ml_pks_step<double>(k, s));
        else DPM_RET(ml_pks_step<float>(k, s));
    }
    if (stats && k->gs.on) {
        int bad = 0;
        DPM_RET(k->gs.pull(k->t, k->dt_prev, k->step, k->last_rebuilt, &bad, s));
        if (bad) { set_error("time step was not positive/finite on the device"); return DPM_ENUMERIC; }
        if (k->last_rebuilt) DPM_RET(lsq_status(k->ml.lsq, s));
    }
    if (stats) {
        const int L = (int)k->ml.L;
        std::vector<double> dg(6 * L);
        for (int l = 0; l < L; ++l)
            DPM_CUDA(cudaMemcpyAsync(dg.data() + 6 * l, k->ml.sub[l].diag_out.p, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
        DPM_CUDA(cudaStreamSynchronize(s));
        *stats = dpm_pks_stats{};
        stats->t = k->t;
        stats->dt = k->dt_prev;
        stats->step = k->step;
        stats->rebuilt = k->last_rebuilt;
        stats->max_rho = -INFINITY;
        stats->min_rho = INFINITY;
        stats->min_c = INFINITY;
        for (int l = 0; l < L; ++l) {
            stats->mass += dg[6 * l];
            stats->max_rho = std::max(stats->max_rho, dg[6 * l + 1]);
            stats->min_rho = std::min(stats->min_rho, dg[6 * l + 2]);
            stats->min_c = std::min(stats->min_c, dg[6 * l + 3]);
            stats->m2 += dg[6 * l + 4];
            stats->free_energy += dg[6 * l + 5];
        }
        if (k->ml.prm.precision == DPM_PREC_TC32) DPM_RET(tc_status_check());
        if (!std::isfinite(stats->mass) || !std::isfinite(stats->free_energy)) {
            set_error("PKS state became non-finite at step %lld", (long long)k->step);
            return DPM_ENUMERIC;
        }
    }
    return DPM_OK;
}

extern "C" int dpm_ml_pks_get_state(dpm_ml_pks *k, int l, void *rho, void *c, cudaStream_t s) {
    if (!k || l < 0 || l >= (int)k->ml.L) { set_error("pks is NULL or sub-domain index out of range"); return DPM_EINVAL; }
    const MLSub &sd = k->ml.sub[l];
    const size_t n3 = (size_t)sd.N * sd.N * sd.N * elem_size(k->ml.storage);
    if (rho) DPM_CUDA(cudaMemcpyAsync(rho, sd.rho.p, n3, cudaMemcpyDeviceToDevice, s));
    if (c) DPM_CUDA(cudaMemcpyAsync(c, sd.c.p, n3, cudaMemcpyDeviceToDevice, s));
    return DPM_OK;
}

extern "C" int dpm_ml_pks_destroy(dpm_ml_pks *k) {
    delete k;
    return DPM_OK;
}
