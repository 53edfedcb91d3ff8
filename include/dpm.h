/*
 * dpm.h -- C ABI of the GB300 (sm_103a) Difference Potentials Method library.
 *
 * The library implements the data-parallel hot path of the Difference
 * Potentials Method (DPM) for the 3D Patlak-Keller-Segel (PKS) chemotaxis
 * system of Epshteyn & Xia, "Efficient Numerical Algorithms based on
 * Difference Potentials for Chemotaxis Systems in 3D" (arXiv:1811.03557).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns int: DPM_OK (0) or a negative DPM_E* code.  On an
 *    error dpm_last_error() returns a message (thread-local, valid until the
 *    next call on the same thread).  No C++ exception crosses this boundary.
 *  - Grid: the auxiliary domain is the cube [lo, hi]^3 with N interior nodes
 *    per axis, x_j = lo + j*h, j = 1..N, h = (hi - lo)/(N + 1).  The nodes
 *    j = 0 and j = N+1 are the Dirichlet layer N^0 \ M^0 of the auxiliary
 *    problem and are never stored.
 *  - Arrays over the grid are C-ordered u[i][j][k] (i = x, j = y, k = z, k
 *    contiguous), linear index (i*N + j)*N + k, N^3 elements.
 *  - "device" pointers are CUDA device memory (or managed memory) owned by
 *    the caller; "host" pointers are ordinary host memory.  Handles
 *    (dpm_ctx, dpm_bep, dpm_pks) own their internal device workspaces and free
 *    them in the matching destroy call.
 *  - All device work is enqueued on the caller's stream; a call returns once
 *    the work is enqueued unless its comment says it synchronises (calls that
 *    return counts or statistics to host memory synchronise the stream).
 *  - A handle may be used by one host thread at a time.  Work on one handle
 *    issued to two streams without ordering between them races.
 */
#ifndef DPM_H_
#define DPM_H_

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define DPM_OK            0
#define DPM_EINVAL       -1   /* invalid argument, size or geometry          */
#define DPM_ENOMEM       -2   /* device allocation failed                     */
#define DPM_ETIMEOUT     -3   /* a bounded device wait gave up                */
#define DPM_ENUMERIC     -4   /* non-finite value or singular factorisation  */
#define DPM_EUNSUPPORTED -5   /* valid request the library does not serve    */
#define DPM_ECUDA        -6   /* a CUDA runtime call failed                   */

/* ---- arithmetic of the auxiliary-problem (AP) solve -------------------- */
#define DPM_PREC_FP32 0  /* FP32 SIMT folded DST-I, FP32 storage            */
#define DPM_PREC_FP64 1  /* FP64 SIMT DST-I, FP64 storage (comparator path) */
#define DPM_PREC_TC32 2  /* tcgen05 DST-I contractions (3-term f16 split,
                            FP32 accumulate), FP32 storage; N = 128, 256    */
#define DPM_PREC_FFT32 3 /* FFT-style FP32 DST-I: even/odd fold + Rader
                            convolutions by length-128 FFTs (N + 1 = 257 is
                            prime), three passes; FP32 storage; N = 256     */

/* ---- node label bits (one uint8 per node of M^0, Definition 2.1) ------- */
#define DPM_LBL_MPLUS 1  /* node of M^+ (strict interior of Omega)           */
#define DPM_LBL_GIN   2  /* node of gamma_in  = M^+ intersect gamma          */
#define DPM_LBL_GEX   4  /* node of gamma_ex  = M^- intersect gamma          */
#define DPM_LBL_SHELL 8  /* node of M^- where L[v_gamma] of a density on
                            gamma can be nonzero (gamma_ex and M^- neighbours
                            of gamma): the support of the right-hand side of
                            a difference potential, eq. rhs:difference_potentials */

typedef struct dpm_ctx dpm_ctx;
typedef struct dpm_bep dpm_bep;
typedef struct dpm_pks dpm_pks;

/* Domain Omega.  kind 0: sphere |x - center| < axes[0] (axes[1], axes[2]
 * ignored); kind 1: ellipsoid sum ((x_i - center_i)/axes_i)^2 < 1; kind 2:
 * spherical shell axes[1] < |x - center| < axes[0] (the sub-domain of the
 * domain decomposition; the forms of both spheres are tested as below);
 * kinds 3 and 4: the sphere |x - center| < axes[0] inside (3) or outside (4)
 * the sphere of radius axes[1] about center + (0, 0, axes[2]) (the sub-domains
 * of the domain decomposition whose interface meets Gamma).
 * Membership is decided in IEEE double with the fixed order
 * ((tx*tx + ty*ty) + tz*tz) < 1, t_i = (x_i - c_i)/a_i, so that the integer
 * point sets are reproducible bit for bit. */
typedef struct {
    int kind;
    double center[3];
    double axes[3];
} dpm_geom;

/* amp * exp(-alpha * ((x-x0)^2 + (y-y0)^2 + zscale*(z-z0)^2)): the form of the
 * paper's initial conditions (Section 4, Tests (A) and (B); Remark 2.3 (i)). */
typedef struct {
    double amp, alpha;
    double center[3];
    double zscale;
} dpm_gaussian;

typedef struct {
    int N;
    double lo, hi, h, sigma;
    int K, beta, ncol, precision;
    int64_t n_mplus, n_gin, n_gex, n_gamma, n_shell;
} dpm_bep_info;

typedef struct {
    dpm_geom geom;
    int N;
    double lo, hi;
    double chi;       /* chemotactic sensitivity (alpha = gamma_rho = gamma_c = 1) */
    double dt_max;    /* time step, or its upper bound in CFL mode              */
    int K, beta;      /* spherical-harmonic degree, extension terms - 2          */
    int precision;    /* DPM_PREC_*                                             */
    int dt_mode;      /* 0: dt = dt_max every step; 1: dt = min(dt_prev,
                         h/(6 chi max|grad_h c|), dt_max) (Step 3)              */
    int rebuild;      /* 0: rebuild the BEP only when dt decreases (Step 4b);
                         1: rebuild it on every step                           */
    int clamp;        /* 1: u_gamma <- max(u_gamma, 0) after the extension
                         (Theorem 2.4, condition 3)                             */
} dpm_pks_params;

typedef struct {
    double t, dt;
    int64_t step;
    int rebuilt;            /* the BEP was (re)assembled in this step         */
    double mass;            /* h^3 sum_{M+} rho                                */
    double max_rho;         /* eq. sd-norm:max                                 */
    double min_rho, min_c;  /* minima over N^+                                 */
    double m2;              /* second moment, eq. sd-norm:second-moment         */
    double free_energy;     /* eq. sd-norm:free-energy                          */
} dpm_pks_stats;

/* Message of the last failed call on this thread ("" if none). */
const char *dpm_last_error(void);

/* Create a context on CUDA device `device` (made current on the calling
 * thread).  The context holds scratch space shared by calls made through it. */
int dpm_ctx_create(int device, dpm_ctx **out);
int dpm_ctx_destroy(dpm_ctx *ctx);

/*
 * Node classification, Definition 2.1 (point sets M^+, M^-, N^+, N^-,
 * gamma = N^+ ^ N^-, gamma_in = M^+ ^ gamma, gamma_ex = M^- ^ gamma).
 *   labels   device uint8[N^3]: DPM_LBL_* bits per node (may be NULL).
 *   gin_idx  device int32[gin_cap]: ascending linear indices of gamma_in (may
 *            be NULL: count only).  gex_idx likewise for gamma_ex.
 *   n_gin, n_gex  host int64 out: the set sizes (this call synchronises).
 * Errors: DPM_EINVAL if N < 6, lo >= hi, a non-positive axis, Omega has no
 * node, a node of M^+ lies within 2 nodes of a cube face (then N^+ or the
 * potential's right-hand side would reach the Dirichlet layer), or a
 * capacity is smaller than the set.  Integer outputs are bit-exact with the
 * CPU oracle's.
 */
int dpm_classify(dpm_ctx *ctx, const dpm_geom *geom, int N, double lo, double hi,
                 uint8_t *labels, int32_t *gin_idx, int64_t gin_cap,
                 int32_t *gex_idx, int64_t gex_cap, int64_t *n_gin, int64_t *n_gex,
                 cudaStream_t stream);

/*
 * Batched Auxiliary Problem solve, Definition 2.4 with the shifted operator:
 *   (sigma - Lap_h) u_b = q_b on M^0,  u_b = 0 on N^0 \ M^0,   b = 0..B-1,
 * Lap_h the 7-point Laplacian (eq. stencil:7-point), diagonalised by the 3D
 * DST-I with eigenvalues sigma + (4/h^2) sum_axes sin^2(pi a/(2(N+1))).
 * (The paper's L_{h,dt} = I - dt Lap_h equals dt (sigma - Lap_h), sigma = 1/dt.)
 *   q, u  device arrays [B][N][N][N]: float for DPM_PREC_FP32/TC32/FFT32, double for
 *         DPM_PREC_FP64.  u may equal q (in place); otherwise they must not
 *         overlap.
 * Requires 2 <= N <= 256, h > 0, sigma >= 0, B >= 1.  DPM_PREC_TC32 requires
 * N = 128 or 256 (DPM_EUNSUPPORTED otherwise) and a 16-byte aligned q (its planes
 * are staged by bulk copies; DPM_EINVAL otherwise).  DPM_PREC_FFT32 requires
 * N = 256 (N + 1 = 257 prime: Rader's algorithm) and a 16-byte aligned q.
 * DPM_PREC_FP32 solves grids of N <= 32 in one pass with each cube in shared
 * memory (no workspace), larger ones in five passes over the workspace.
 * Scratch: the context's workspace, grown on demand.
 */
int dpm_aux_solve_batched(dpm_ctx *ctx, int N, double h, double sigma, int B,
                          const void *q, void *u, int precision, cudaStream_t stream);

/*
 * The same FP32 auxiliary solve as dpm_aux_solve_batched with DPM_PREC_FP32,
 * for callers that must not let a library allocate device memory: an
 * application whose own allocator owns every byte of the GPU, or a
 * latency-critical loop in which cudaMalloc/cudaFree (which may synchronise
 * the device and take an unbounded time) are not acceptable.  The paper has
 * no counterpart; this is an interface convenience.
 *   q, u  device float[B][N][N][N], owned by the caller (u may equal q).
 * All scratch -- the B*N^3 workspace, the sine table and the per-right-hand-
 * side descriptors -- lives in one fixed device array compiled into the
 * library (about 64 MiB, held by every GPU that loads the library until the
 * process exits).  The call allocates nothing.  Limits: 2 <= N <= 256,
 * 1 <= B <= 1024 and B*N^3 <= 16*2^20 (e.g. one N=256 cube, or 8 N=128
 * cubes); larger requests fail with DPM_EINVAL before any work is enqueued.
 * Runs on the calling thread's current CUDA device.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  Every call reuses the same
 * array, so calls that overlap on the GPU (e.g. on two unordered streams)
 * race and must be serialised by the caller.
 */
int dpm_aux_solve_batched_noalloc(int N, double h, double sigma, int B, const float *q,
                                  float *u, cudaStream_t stream);

/*
 * Tile width of the SIMT (DPM_PREC_FP32 / DPM_PREC_FP64) solver.  Each of its
 * five passes works on tiles of C grid lines (C = 16, 32 or 64; smaller tiles
 * give more CTAs per SM, larger ones more reuse of each sine-table load).  The
 * first solve on a device for a given N, precision and batch class (B <= 2,
 * B <= 16, larger) times every width whose shared memory fits on a problem of
 * that size with zero right-hand sides (same work as real data), keeps the
 * fastest and synchronises the stream once to read the timers; a solve issued
 * while its stream is being captured does not tune and uses the tuned width,
 * else 32.  Every output is summed in the same order for each width, so the
 * choice changes the run time only, never the result.  Environment: DPM_SIMT_TILE
 * = 16|32|64 forces a width; DPM_AUTOTUNE=0 keeps 32.  The no-alloc solve
 * always uses 32.  FP32 grids of N <= 32 take the one-pass solve and have no
 * tile width.
 * dpm_simt_tile writes to *tile the width tuned on the current device for
 * (N, precision, B), or 0 if none has been tuned (or none applies).
 */
int dpm_simt_tile(int N, int precision, int B, int *tile);

/*
 * Steps 1-2 of the main algorithm: classify the grid, project every node of
 * gamma on Gamma (foot point, signed distance d > 0 outside Omega along the
 * outward normal; Definition 2.6), evaluate the real orthonormal spherical
 * harmonics phi_nu, nu = l^2+l+m < (K+1)^2, at the foot point's polar and
 * azimuthal angles about the centre (eq. spectral_approximation_sd), assemble
 * the |gamma_in| x ncol BEP matrix of eq. BEP_recast,
 *   A[:, k] = Tr_{gamma_in} (I - P_{N+gamma}) psi_k,
 *   psi_k = phi_k (k < (K+1)^2),  psi_k = (d^2/2) phi_{k-(K+1)^2} (beta = 1),
 * ncol = (beta+1)(K+1)^2, with one AP per column solved in one batch, and
 * factor it for least squares (the R factor of its QR decomposition, kept
 * resident with A; solves refine in FP64).
 * K in [0, 16], beta in {0, 1}; sigma > 0.  Synchronises the stream.
 */
int dpm_bep_build(dpm_ctx *ctx, const dpm_geom *geom, int N, double lo, double hi,
                  double sigma, int K, int beta, int precision, dpm_bep **out,
                  cudaStream_t stream);
int dpm_bep_get_info(const dpm_bep *bep, dpm_bep_info *info);
/* Copy the BEP matrix to device double[n_gin * ncol], column-major. */
int dpm_bep_matrix(const dpm_bep *bep, double *A, cudaStream_t stream);
/* Copy the gamma geometry: ascending linear indices (int32[n_gamma]), foot
 * points and unit outward normals (double[n_gamma][3]) and signed distances
 * (double[n_gamma]).  Any pointer may be NULL.  All device pointers. */
int dpm_bep_gamma_geometry(const dpm_bep *bep, int32_t *gamma_idx, double *foot,
                           double *normal, double *dist, cudaStream_t stream);
int dpm_bep_destroy(dpm_bep *bep);

/*
 * Elliptic DPM solve of (sigma - Lap) u = f in Omega, du/dn = g_N on Gamma:
 * particular solution G f (eq. rhs:particular_solution), least squares of
 * the BEP for the spectral coefficients (Step 5, using the resident QR),
 * extension u_gamma = sum C0 phi + d g_N + beta (d^2/2) sum C2 phi
 * (eq. extension_operator), and the discrete generalised Green's formula
 * u = P_{N+gamma} u_gamma + G f on N^+ (eq. generalized_greens_formula).
 *   f        device [N^3] (float, or double for DPM_PREC_FP64), used on M^+.
 *   neumann  device double[n_gamma] g_N at the foot point of each node of
 *            gamma (ascending order), or NULL for zero Neumann data.
 *   u        device [N^3] out: the solution on N^+, 0 elsewhere.
 *   coeffs   device double[ncol] out (C0 then C2), or NULL.
 */
int dpm_solve(dpm_bep *bep, const void *f, const double *neumann, void *u,
              double *coeffs, cudaStream_t stream);

/*
 * dpm_solve for nreq independent right-hand sides against one resident BEP
 * (the batching primitive of a request loop): all particular solutions (and
 * Neumann terms) in one batched AP, the least squares for all of them, the
 * extensions, and all Green's-formula APs in a second batched AP.  Arguments
 * are host arrays of nreq device pointers with the meaning of dpm_solve's
 * (neumann[r] and coeffs[r] may be NULL; the arrays themselves may be NULL).
 * Every request's result is computed by the same per-request arithmetic as
 * dpm_solve, so it is identical whether solved alone or in a batch.
 * 1 <= nreq <= 64.
 */
int dpm_solve_batched(dpm_bep *bep, int nreq, const void *const *f, const double *const *neumann,
                      void *const *u, double *const *coeffs, cudaStream_t stream);

/*
 * Device bytes held by a BEP object (index lists, gamma geometry, columns,
 * the factor, and the solve workspaces as currently sized).  Host-side
 * query; no device work.
 */
int dpm_bep_device_bytes(const dpm_bep *bep, int64_t *bytes);

/*
 * Size every workspace a dpm_solve_batched call of up to max_nreq requests
 * touches, so that such solves allocate nothing, and shrink the build
 * workspace to that size (a later rebuild grows it again).  Synchronises the
 * device (it may free memory).  Not part of the method: it serves request
 * loops that keep many factorisations resident.  1 <= max_nreq <= 64.
 */
int dpm_bep_reserve(dpm_bep *bep, int max_nreq);

/*
 * PKS time stepping (Steps 3-7 of the main algorithm) on one domain.
 * create: builds the point sets and gamma geometry and sets rho^0, c^0 to the
 * given Gaussians at the nodes of M^+ and at the foot points of gamma_ex
 * (Remark 2.1, 2-term extension with zero Neumann data).  Synchronises.
 * set_state/get_state: device [N^3] arrays (float, or double for
 * DPM_PREC_FP64) holding the values on N^+ (other nodes ignored / zeroed).
 * step: advances nsteps steps; each step chooses dt (Step 3), forms the
 * upwind minmod flux and the IMEX right-hand sides (eqs. discrete_chemotaxis
 * to slope_limiter), rebuilds the BEP when dt_mode/rebuild ask for it (Step
 * 4b), solves the particular problems, the least squares and the extensions
 * (Steps 4a-5) and applies Green's formula (Steps 6-7) for rho and c.
 * If stats is not NULL the call synchronises and writes the statistics of
 * the last step (host struct).  DPM_ENUMERIC if a value became non-finite.
 */
int dpm_pks_create(dpm_ctx *ctx, const dpm_pks_params *params, const dpm_gaussian *rho0,
                   const dpm_gaussian *c0, dpm_pks **out, cudaStream_t stream);
int dpm_pks_set_state(dpm_pks *pks, const void *rho, const void *c, cudaStream_t stream);
int dpm_pks_step(dpm_pks *pks, int nsteps, dpm_pks_stats *stats, cudaStream_t stream);

/*
 * Graph stepping (on != 0): later dpm_pks_step calls keep dt, sigma and the
 * time in device memory (Step 3's dt computed by a kernel from the CFL
 * maxima), so a step needs no host synchronisation; the library captures one
 * step in a CUDA graph (on its own capture stream, after one uncaptured step
 * that sizes the workspaces) and replays it on `stream` for each step.  Same
 * kernels and arithmetic as the default stepping, so the results are the
 * same.  The BEP is rebuilt every step with rebuild = 1, never with dt_mode 0
 * (the BEP of sigma = 1/dt_max), and with dt_mode 1 and rebuild = 0 only when
 * dt decreases (Step 4b): a conditional (if/else) graph node whose condition
 * a kernel sets from the step's dt.  on = 0 returns to the default stepping
 * (synchronises to read the time back).  The pivot status of the
 * factorisations is checked when statistics are requested.
 */
int dpm_pks_set_graph(dpm_pks *pks, int on, cudaStream_t stream);
int dpm_pks_get_state(dpm_pks *pks, void *rho, void *c, cudaStream_t stream);
/* Device bytes held by a PKS run (its BEP, the two fields and scratch). */
int dpm_pks_device_bytes(const dpm_pks *pks, int64_t *bytes);

int dpm_pks_destroy(dpm_pks *pks);

/* ---- diagnostics (no counterpart in the paper) -------------------------
 * dpm_launch_count: number of CUDA kernels this library has launched in this
 * process (all threads), for checking that work ran on the GPU.
 * dpm_profile_enable(1): from now on each kernel launch of the library is
 * bracketed by CUDA events recorded on the stream it is launched on (adds a
 * little host overhead); 0 stops recording.  dpm_profile_read: synchronises
 * on the recorded events and returns, for kernels whose name contains
 * `name` (NULL or "" = all), the summed device time in ms and the number of
 * launches.  dpm_profile_reset drops all records. */
int64_t dpm_launch_count(void);
int dpm_profile_enable(int on);
int dpm_profile_read(const char *name, double *total_ms, int64_t *launches);
int dpm_profile_reset(void);

/* ---- domain decomposition, Case 1 (Section 3) ---------------------------------
 * Omega_1 = ball |x - center| < r1 on an N1^3 grid of [lo1, hi1]^3, Omega_2 =
 * shell r1 < |x - center| < r2 on an N2^3 grid of [lo2, hi2]^3 (classified as
 * dpm_geom kind 2 with axes = (r2, r1, -); its grid boundary splits into the
 * nodes whose foot point lies on the interface Z (|x - c| = r1) and those on
 * Gamma (|x - c| = r2)).  Unknowns: three real spherical-harmonic series of
 * degree KZ on Z -- u, du/dnu, d2u/dnu2 with nu = (x - c)/|x - c| -- shared by
 * both sub-domains (the interface conditions, eq. interface_condition), and
 * two of degree KG on Gamma -- u, d2u/dn2 (du/dn is the Neumann data).  The
 * reduced BEPs of both sub-domains (eqs. reduced_DD1_BEP1, reduced_DD1_BEP2)
 * are stacked (rows: gamma_in of Omega_1, then of Omega_2; columns: the Z
 * coefficients (3 (KZ+1)^2, term-major) then the Gamma ones (2 (KG+1)^2)) and
 * solved in the least-squares sense; each sub-domain then applies Green's
 * formula on its own grid.  precision applies per sub-domain: DPM_PREC_TC32
 * falls back to DPM_PREC_FP32 on a grid whose N has no tensor-core solver;
 * DPM_PREC_FFT32 uses the FFT-style solver where N has one, else the
 * tensor-core solver where N has one, else DPM_PREC_FP32. */
typedef struct dpm_dd dpm_dd;
typedef struct dpm_dd_pks dpm_dd_pks;

typedef struct {
    double center[3];
    double r1, r2;        /* interface and outer radius, 0 < r1 < r2 */
    int N1;
    double lo1, hi1;      /* grid of the ball */
    int N2;
    double lo2, hi2;      /* grid of the shell */
    int KZ, KG;           /* harmonic degrees on Z and Gamma, 0..16 */
    int precision;
} dpm_dd_params;

typedef struct {
    int N[2];
    double h[2];
    int precision[2];
    int64_t n_mplus[2], n_gin[2], n_gamma[2];
    int nz, ng, ncol;
    double sigma;
} dpm_dd_info;

/* Steps 1-2 for both sub-domains at shift sigma (synchronises). */
int dpm_dd_build(dpm_ctx *ctx, const dpm_dd_params *params, double sigma, dpm_dd **out,
                 cudaStream_t stream);
int dpm_dd_get_info(const dpm_dd *dd, dpm_dd_info *info);
/* The stacked BEP matrix: device double[(n_gin[0] + n_gin[1]) * ncol], column-major. */
int dpm_dd_matrix(dpm_dd *dd, double *A, cudaStream_t stream);
/*
 * (sigma - Lap) u = f on Omega_1 + Omega_2 with du/dn = g_N on Gamma: f1 / f2
 * device [N1^3] / [N2^3] (float, or double for DPM_PREC_FP64) used on M^+ of
 * each sub-domain; neumann2 device double[n_gamma[1]] (values at the grid
 * boundary nodes of the shell, in ascending node order; only its Gamma nodes
 * are read) or NULL for zero; u1 / u2 device outputs valid on N^+ of each
 * sub-domain (zero elsewhere); coeffs device double[ncol] or NULL.
 */
int dpm_dd_solve(dpm_dd *dd, const void *f1, const void *f2, const double *neumann2, void *u1,
                 void *u2, double *coeffs, cudaStream_t stream);
int dpm_dd_destroy(dpm_dd *dd);

/*
 * PKS time stepping on the two sub-domains (Steps 3-7 with the coupled BEP;
 * zero Neumann data on Gamma): dt = min(dt_max, the CFL bounds of both grids,
 * dt_prev) in dt_mode 1 (dt_max in dt_mode 0); the stacked BEP is rebuilt
 * when dt decreases or on every step with rebuild = 1; clamp: u_gamma >= 0.
 * rho0/c0 set the state on M^+ of each sub-domain and at the foot points of its
 * exterior grid-boundary nodes.  Statistics combine both sub-domains (sums of
 * mass, second moment and free energy; max / min over both).
 */
int dpm_dd_pks_create(dpm_ctx *ctx, const dpm_dd_params *params, double chi, double dt_max,
                      int dt_mode, int rebuild, int clamp, const dpm_gaussian *rho0,
                      const dpm_gaussian *c0, dpm_dd_pks **out, cudaStream_t stream);
int dpm_dd_pks_step(dpm_dd_pks *pks, int nsteps, dpm_pks_stats *stats, cudaStream_t stream);
/* Graph stepping of the Case 1 loop, as dpm_ml_pks_set_graph (Steps 3-7 of the
 * main algorithm on both sub-domains, Section 3): dt on the device, the
 * batched solves of both grids prepared once, the step captured in one CUDA
 * graph and replayed; the stacked BEP rebuilt as dpm_pks_set_graph rebuilds it
 * (with dt_mode 1 and rebuild = 0 only when dt decreases).  Same kernels and
 * arithmetic as the default stepping.  With dt_mode 0 and no rebuild the BEP is
 * built when graph stepping starts, so the first step then reports rebuilt = 0.
 * on = 0 returns to the default stepping. */
int dpm_dd_pks_set_graph(dpm_dd_pks *pks, int on, cudaStream_t stream);
/* State of sub-domain l (0: ball, 1: shell) into device [N_l^3] arrays. */
int dpm_dd_pks_get_state(dpm_dd_pks *pks, int l, void *rho, void *c, cudaStream_t stream);
int dpm_dd_pks_destroy(dpm_dd_pks *pks);

/* ---- domain decomposition, Case 2 (Section 3: the interface meets Gamma) -----
 * Omega = sphere |x - center| < R; the interface Z is the sphere |x - c_Z| = rz,
 * c_Z = center + (0, 0, zoff), with |R - rz| < |zoff| < R + rz so that Z cuts
 * Gamma.  Omega_1 = Omega inside Z (classified as dpm_geom kind 3: axes = (R, rz,
 * zoff)), Omega_2 = Omega outside Z (kind 4, same axes).  Sub-domain l has its
 * own box, the cube origin_l + [lo_l, hi_l]^3 (global coordinates; the grid and
 * every per-node output are in the local frame x - origin_l), N_l interior nodes
 * per axis.
 * Grid-boundary split (gamma_l and zeta_l, Section 3): a grid-boundary node of
 * Omega_l (Definition 2.1 on Omega_l's own point sets) is a Gamma node when it is
 * a grid-boundary node of the sphere Omega on the same grid, a Z node when it is
 * one of the ball inside Z, both in the one-layer wedge where Z meets Gamma
 * (a node in neither, possible only for a node exactly on a sphere, goes to the
 * nearer surface).  A wedge node's density is the mean of its Gamma value and
 * its Z value, and each node of gamma_in gives one BEP row per surface it
 * belongs to (eq. reduced_DD2_BEP; rows: Omega_1's gamma_in nodes in ascending
 * order, a Gamma row before a Z row, then Omega_2's).
 * Unknowns: zonal harmonics Y_nu(theta) = sqrt((2 nu + 1)/(4 pi)) P_nu(cos theta),
 * nu < M, theta the polar angle about each sphere's centre from +z: three series
 * of MZ terms on Z (u, du/dnu, d2u/dnu2, nu = (x - c_Z)/|x - c_Z|, shared by both
 * sub-domains) then two of MG terms on Gamma (u, d2u/dn2; du/dn is the Neumann
 * data).  On Z the argument of P_nu is cos theta_Z mapped from the range that
 * the part of Z inside Omega spans ([-1, c*] for zoff > 0, [c*, 1] otherwise, c*
 * = (R^2 - zoff^2 - rz^2)/(2 zoff rz)) to [-1, 1]: the same polynomials of degree
 * < MZ in cos theta_Z, in a basis that stays well conditioned on the partial
 * sphere.  Columns: term-major, Z first.  The problem must be symmetric about
 * the z axis through both centres for the zonal basis to represent it.  The
 * least squares use the FP64 Gram of the column-equilibrated matrix.
 * MZ in [1, 64], MG in [1, 1024]; N_l <= 256; precision as for Case 1. */
typedef struct dpm_dd2 dpm_dd2;
typedef struct dpm_dd2_pks dpm_dd2_pks;

typedef struct {
    double center[3];
    double R, rz, zoff;
    int N1;
    double lo1, hi1, origin1[3];  /* Omega_1 (inside Z) */
    int N2;
    double lo2, hi2, origin2[3];  /* Omega_2 (outside Z) */
    int MZ, MG;
    int precision;
    int gamma_series;  /* unknown series on Gamma: 2 (0 = default) for the 3-term
                          extension u + d g_N + (d^2/2) d2u/dn2, 1 for the 2-term
                          extension u + d g_N (Section 4 uses it on the boundary
                          for Test (B); it stays well conditioned with MG beyond
                          what the 3-term one tolerates) */
} dpm_dd2_params;

typedef struct {
    int N[2];
    double h[2];
    int precision[2];
    int64_t n_mplus[2], n_gin[2], n_gamma[2];
    int64_t n_rows[2];            /* BEP rows of each sub-domain */
    int64_t n_wedge[2];           /* grid-boundary nodes on both surfaces */
    int ncol;
    double sigma;
} dpm_dd2_info;

/* Steps 1-2 for both sub-domains at shift sigma (synchronises). */
int dpm_dd2_build(dpm_ctx *ctx, const dpm_dd2_params *params, double sigma, dpm_dd2 **out,
                  cudaStream_t stream);
int dpm_dd2_get_info(const dpm_dd2 *dd, dpm_dd2_info *info);
/* The stacked BEP matrix: device double[(n_rows[0] + n_rows[1]) * ncol], column-major. */
int dpm_dd2_matrix(dpm_dd2 *dd, double *A, cudaStream_t stream);
/* Grid boundary of sub-domain l: ascending linear node indices (int32[n_gamma]),
 * surface flags (uint8: bit 0 Gamma, bit 1 Z) and the foot points on Gamma in
 * the local frame (double[n_gamma][3]).  Any pointer may be NULL.  Device. */
int dpm_dd2_gamma(dpm_dd2 *dd, int l, int32_t *gamma_idx, uint8_t *flags, double *foot_gamma,
                  cudaStream_t stream);
/*
 * (sigma - Lap) u = f on Omega_1 + Omega_2 with du/dn = g_N on Gamma: f1 / f2
 * device [N1^3] / [N2^3] (float, or double for DPM_PREC_FP64) used on M^+;
 * neumann1 / neumann2 device double[n_gamma[l]]: g_N at the Gamma foot points of
 * sub-domain l's grid-boundary nodes (read on its Gamma nodes), or NULL for zero;
 * u1 / u2 device outputs valid on N^+ of each sub-domain; coeffs device
 * double[ncol] or NULL.
 */
int dpm_dd2_solve(dpm_dd2 *dd, const void *f1, const void *f2, const double *neumann1,
                  const double *neumann2, void *u1, void *u2, double *coeffs, cudaStream_t stream);
int dpm_dd2_destroy(dpm_dd2 *dd);

/* PKS time stepping on the two sub-domains of Case 2 (as dpm_dd_pks_*, zero
 * Neumann data; rho0 / c0 in global coordinates; the gamma_ex nodes take the
 * data at their foot point on Gamma, or on Z for Z-only nodes; the clamp
 * u_gamma >= 0 acts on the effective densities; the second moment is taken in
 * global coordinates). */
int dpm_dd2_pks_create(dpm_ctx *ctx, const dpm_dd2_params *params, double chi, double dt_max,
                       int dt_mode, int rebuild, int clamp, const dpm_gaussian *rho0,
                       const dpm_gaussian *c0, dpm_dd2_pks **out, cudaStream_t stream);
int dpm_dd2_pks_step(dpm_dd2_pks *pks, int nsteps, dpm_pks_stats *stats, cudaStream_t stream);
/* Graph stepping of the Case 2 loop (Section 3, eq. reduced_DD2_BEP), as
 * dpm_dd_pks_set_graph. */
int dpm_dd2_pks_set_graph(dpm_dd2_pks *pks, int on, cudaStream_t stream);
int dpm_dd2_pks_get_state(dpm_dd2_pks *pks, int l, void *rho, void *c, cudaStream_t stream);
int dpm_dd2_pks_destroy(dpm_dd2_pks *pks);

/* ---- layered domain decomposition (Section 3's Case 1 with more interfaces) ----
 * L sub-domains (2 <= L <= 16): the ball |x - center| < radii[0] and the shells
 * radii[l-1] < |x - center| < radii[l], l = 1..L-1, radii[L-1] = R the outer
 * boundary Gamma; sub-domain l on its own N[l]^3 grid of [lo[l], hi[l]]^3.
 * Sphere m = 1..L-1 (|x - c| = radii[m-1]) is an interface: three real SH series
 * of degree K[m-1] -- u, du/dnu, d2u/dnu2 with nu = (x - c)/|x - c| -- shared by
 * the two sub-domains it separates; Gamma carries two of degree KG (u, d2u/dn2;
 * du/dn the Neumann data).  A shell's grid-boundary node belongs to the nearer of
 * its two spheres (the outer on a tie).  Columns: sphere by sphere, term-major;
 * rows: gamma_in of sub-domain 0, 1, ..., L-1 (each block involves only the
 * columns of its own spheres).  With L = 2 this is Case 1 (dpm_dd_*).
 * Sub-domains whose grids use the SIMT solver run their batched solves as one
 * grouped set of launches (DPM_DD_GROUP=0: one batch each); a tensor-core grid
 * (N = 128 or 256 with DPM_PREC_TC32) runs its own.  K, KG in [0, 16]. */
#define DPM_ML_MAX 16
typedef struct dpm_ml dpm_ml;
typedef struct dpm_ml_pks dpm_ml_pks;

typedef struct {
    double center[3];
    int L;
    double radii[DPM_ML_MAX];
    int N[DPM_ML_MAX];
    double lo[DPM_ML_MAX], hi[DPM_ML_MAX];
    int K[DPM_ML_MAX];  /* per interface: the first L - 1 entries */
    int KG;
    int precision;
} dpm_ml_params;

typedef struct {
    int L;
    int N[DPM_ML_MAX];
    double h[DPM_ML_MAX];
    int precision[DPM_ML_MAX];
    int64_t n_mplus[DPM_ML_MAX], n_gin[DPM_ML_MAX], n_gamma[DPM_ML_MAX];
    int ncol;
    double sigma;
} dpm_ml_info;

/* Steps 1-2 for all sub-domains at shift sigma (synchronises). */
int dpm_ml_build(dpm_ctx *ctx, const dpm_ml_params *params, double sigma, dpm_ml **out, cudaStream_t stream);
int dpm_ml_get_info(const dpm_ml *ml, dpm_ml_info *info);
/* The stacked BEP matrix: device double[(sum n_gin) * ncol], column-major. */
int dpm_ml_matrix(dpm_ml *ml, double *A, cudaStream_t stream);
/*
 * (sigma - Lap) u = f on the union of the sub-domains, du/dn = g_N on Gamma:
 * f[l] device [N[l]^3] (float, or double for DPM_PREC_FP64) used on M^+ of
 * sub-domain l; neumann device double[n_gamma[L-1]] (values at the outermost
 * sub-domain's grid-boundary nodes in ascending node order, read on its Gamma
 * nodes) or NULL; u[l] device outputs valid on N^+ of each sub-domain; coeffs
 * device double[ncol] or NULL.  f and u are host arrays of L device pointers.
 */
int dpm_ml_solve(dpm_ml *ml, const void *const *f, const double *neumann, void *const *u, double *coeffs,
                 cudaStream_t stream);
int dpm_ml_destroy(dpm_ml *ml);

/* PKS time stepping on the L sub-domains (as dpm_dd_pks_*: dt from the CFL bounds
 * of all grids in dt_mode 1, dt_max in dt_mode 0; the stacked BEP rebuilt when dt
 * decreases or always with rebuild = 1; statistics summed / extremised over all). */
int dpm_ml_pks_create(dpm_ctx *ctx, const dpm_ml_params *params, double chi, double dt_max, int dt_mode,
                      int rebuild, int clamp, const dpm_gaussian *rho0, const dpm_gaussian *c0, dpm_ml_pks **out,
                      cudaStream_t stream);
int dpm_ml_pks_step(dpm_ml_pks *pks, int nsteps, dpm_pks_stats *stats, cudaStream_t stream);
/* Graph stepping of the layered loop, as dpm_pks_set_graph (Steps 3-7 of the
 * main algorithm on every sub-domain, Section 3): dt from the CFL maxima of
 * all grids by a kernel, every sub-domain's batched solves prepared once (the
 * SIMT grids' right-hand sides as one group of launches), the whole step
 * captured in one CUDA graph and replayed per step.  Same kernels and
 * arithmetic as the default stepping; the stacked BEP is rebuilt as
 * dpm_pks_set_graph rebuilds it (with dt_mode 1 and rebuild = 0 only when dt
 * decreases, by a conditional graph node); with dt_mode 0 and no rebuild the
 * stacked BEP of sigma = 1/dt_max is built when graph stepping starts.  on = 0
 * returns to the default stepping (synchronises to read the time back). */
int dpm_ml_pks_set_graph(dpm_ml_pks *pks, int on, cudaStream_t stream);
int dpm_ml_pks_get_state(dpm_ml_pks *pks, int l, void *rho, void *c, cudaStream_t stream);
int dpm_ml_pks_destroy(dpm_ml_pks *pks);

#ifdef __cplusplus
}
#endif
#endif /* DPM_H_ */
