// FP64 least squares for the spectral coefficients of the BEP (eq. BEP_recast,
// Steps 2 and 5 of the main algorithm).
//
// Factor (once per BEP): Householder QR of A (m x n, column-major, m >> n),
// one reflector per column, H_j = I - tau_j v_j v_j^T, keeping R and a copy
// of A.  Solve (every step): the normal equations through the QR factor,
// R^T R C = A^T b (the "semi-normal equations"), followed by one step of
// iterative refinement on the residual r = b - A C.  Both steps are FP64
// GEMVs spread over all SMs plus n x n triangular solves in one CTA, so the
// per-step cost does not depend on forming Q.
#include <math.h>

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
__global__ void k_atb(int m, int n, const double *A0, const T *b, int ldb, double *y, int nr) {
    __shared__ double sh[32];
    int c = blockIdx.x, q = blockIdx.y;
    const double *a = A0 + (size_t)c * m;
    const T *bq = b + (size_t)q * ldb;
    double s = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) s += a[r] * (double)bq[r];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) y[(size_t)q * n + c] = s;
}

// res[q][r] = b[q][r] - sum_c A0[r][c] C[q][c]
template <class T>
__global__ void k_resid(int m, int n, const double *A0, const T *b, int ldb, const double *C,
                        double *res, int nr) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    int q = blockIdx.y;
    if (r >= m) return;
    const double *cq = C + (size_t)q * n;
    double s = (double)b[(size_t)q * ldb + r];
    for (int c = 0; c < n; ++c) s -= A0[(size_t)c * m + r] * cq[c];
    res[(size_t)q * m + r] = s;
}

// Solve R^T z = y then R x = z (R row-major upper triangular); C[q] (+)= x.
__global__ void k_trisolve(int n, const double *R, const double *y, double *C, int accumulate,
                           int *status) {
    extern __shared__ double z[];
    int q = blockIdx.x;
    const double *yq = y + (size_t)q * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] = yq[i];
    __syncthreads();
    // forward: R^T z = y  (column i of R^T is row i of R)
    for (int i = 0; i < n; ++i) {
        if (threadIdx.x == 0) {
            double d = R[(size_t)i * n + i];
            if (d == 0.0) { status[0] = 1; d = 1.0; }
            z[i] /= d;
        }
        __syncthreads();
        double zi = z[i];
        for (int k = i + 1 + threadIdx.x; k < n; k += blockDim.x) z[k] -= R[(size_t)i * n + k] * zi;
        __syncthreads();
    }
    // backward: R x = z
    for (int i = n - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            double d = R[(size_t)i * n + i];
            z[i] /= (d == 0.0 ? 1.0 : d);
        }
        __syncthreads();
        double zi = z[i];
        for (int k = threadIdx.x; k < i; k += blockDim.x) z[k] -= R[(size_t)k * n + i] * zi;
        __syncthreads();
    }
    double *cq = C + (size_t)q * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) cq[i] = accumulate ? cq[i] + z[i] : z[i];
}

}  // namespace

int lsq_factor(LsqFactor &f, const int *cond_flag, cudaStream_t s) {
    (void)cond_flag;
    const int m = f.m, n = f.n;
    if (m < n || n < 1) { set_error("least squares: need m >= n >= 1 (m=%d n=%d)", m, n); return DPM_EINVAL; }
    // layout of f.work: [A0 m*n][w n][rdiag n][R n*n][status (64 B)][y 4*n][res 4*m]
    size_t need = sizeof(double) * ((size_t)m * n + 2 * (size_t)n + (size_t)n * n) + 64 +
                  sizeof(double) * 4 * ((size_t)n + (size_t)m);
    DPM_RET(f.work.reserve(need));
    DPM_RET(f.tau.reserve(sizeof(double) * n));
    double *A0 = f.work.as<double>();
    double *w = A0 + (size_t)m * n;
    double *rdiag = w + n;
    double *R = rdiag + n;
    int *status = reinterpret_cast<int *>(R + (size_t)n * n);
    DPM_CUDA(cudaMemcpyAsync(A0, f.A.p, sizeof(double) * m * n, cudaMemcpyDeviceToDevice, s));
    DPM_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
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
    int h_status = 0;
    DPM_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    DPM_CUDA(cudaStreamSynchronize(s));
    if (h_status) { set_error("BEP matrix is rank deficient (a zero Householder column)"); return DPM_ENUMERIC; }
    return DPM_OK;
}

template <class T>
int lsq_apply(const LsqFactor &f, const T *b, int ldb, double *C, int nr, cudaStream_t s) {
    const int m = f.m, n = f.n;
    const double *A0 = f.work.as<double>();
    const double *R = A0 + (size_t)m * n + 2 * (size_t)n;
    int *status = reinterpret_cast<int *>(const_cast<double *>(R) + (size_t)n * n);
    if (nr < 1 || nr > 4) { set_error("least squares: 1..4 right-hand sides per call"); return DPM_EINVAL; }
    // scratch after the factor: y[nr][n], res[nr][m]
    size_t base = sizeof(double) * ((size_t)m * n + 2 * (size_t)n + (size_t)n * n) + 64;
    double *y = reinterpret_cast<double *>(static_cast<char *>(f.work.p) + base);
    double *res = y + (size_t)nr * n;
    size_t tri_smem = sizeof(double) * n;
    k_atb<T><<<dim3(n, nr), kT, 0, s>>>(m, n, A0, b, ldb, y, nr);
    DPM_LAUNCHED();
    k_trisolve<<<nr, 256, tri_smem, s>>>(n, R, y, C, 0, status);
    DPM_LAUNCHED();
    // one step of iterative refinement
    k_resid<T><<<dim3((m + 255) / 256, nr), 256, 0, s>>>(m, n, A0, b, ldb, C, res, nr);
    DPM_LAUNCHED();
    k_atb<double><<<dim3(n, nr), kT, 0, s>>>(m, n, A0, res, m, y, nr);
    DPM_LAUNCHED();
    k_trisolve<<<nr, 256, tri_smem, s>>>(n, R, y, C, 1, status);
    DPM_LAUNCHED();
    return DPM_OK;
}

template int lsq_apply<float>(const LsqFactor &, const float *, int, double *, int, cudaStream_t);
template int lsq_apply<double>(const LsqFactor &, const double *, int, double *, int, cudaStream_t);

}  // namespace dpm
