// bisect.cu -- eigenvalues of the final symmetric tridiagonal by Sturm-count
// bisection (the "compute its eigenvalues" step of Algorithm 4.3), plus the
// small copy kernels between dense, packed-band and tridiagonal storage.
//
// The Sturm count at x is the number of negative pivots of LDL^T(T - xI):
//   q_0 = d_0 - x,  q_i = (d_i - x) - e_{i-1}^2 / q_{i-1},
// with |q_i| < pivmin replaced by -pivmin, pivmin = DBL_MIN max(1, max e^2).
// Every FP64 operation is written with an explicit round-to-nearest
// intrinsic so no multiply-add is contracted: the result is the exact IEEE
// evaluation of the recurrence in the order written.
#include "common.cuh"

namespace sev {

// ------------------------------------------------------------ storage copies
template <typename T>
__global__ void band_from_dense_kernel(int n, const T *__restrict__ A, int lda, int b, T *__restrict__ AB, int ldab) {
    const long total = (long)ldab * n;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int d = (int)(idx % ldab);
        const int j = (int)(idx / ldab);
        T v = 0;
        if (d <= b && j + d < n) v = A[(size_t)(j + d) + (size_t)j * lda];
        AB[idx] = v;
    }
}

template <typename T>
int launch_band_from_dense(sev_ctx *h, int n, const T *A, int lda, int b, T *AB, int ldab) {
    if (n <= 0) return SEV_OK;
    const long total = (long)ldab * n;
    int grid = (int)((total + kThreads - 1) / kThreads);
    if (grid > h->sm_count * 16) grid = h->sm_count * 16;
    SEV_LAUNCH(h, K_BAND_FROM_DENSE, band_from_dense_kernel<T>, grid, kThreads, 0, n, A, lda, b, AB, ldab);
    return SEV_OK;
}

template <typename T>
__global__ void tridiag_extract_kernel(int n, const T *__restrict__ AB, int ldab, double *__restrict__ d,
                                       double *__restrict__ e) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        d[j] = (double)AB[(size_t)j * ldab];
        if (j + 1 < n) e[j] = (double)AB[1 + (size_t)j * ldab];
    }
}

template <typename T>
int launch_tridiag_extract(sev_ctx *h, int n, const T *AB, int ldab, double *d, double *e) {
    if (n <= 0) return SEV_OK;
    int grid = (n + kThreads - 1) / kThreads;
    if (grid > h->sm_count * 4) grid = h->sm_count * 4;
    SEV_LAUNCH(h, K_TRIDIAG_EXTRACT, tridiag_extract_kernel<T>, grid, kThreads, 0, n, AB, ldab, d, e);
    return SEV_OK;
}

template int launch_band_from_dense<float>(sev_ctx *, int, const float *, int, int, float *, int);
template int launch_band_from_dense<double>(sev_ctx *, int, const double *, int, int, double *, int);
template int launch_tridiag_extract<float>(sev_ctx *, int, const float *, int, double *, double *);
template int launch_tridiag_extract<double>(sev_ctx *, int, const double *, int, double *, double *);

// ----------------------------------------------------------------- bisection
// par[0] = gl, par[1] = gu (widened Gershgorin interval), par[2] = pivmin,
// par[3] = tnorm (max |end| of the unwidened interval).
__global__ void bisect_prep_kernel(int n, const double *__restrict__ d, const double *__restrict__ e,
                                   double *__restrict__ e2, double *__restrict__ par) {
    __shared__ double red[32];
    double lo = INFINITY, hi = -INFINITY, emax = 1.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double r = 0.0;
        if (i > 0) r = __dadd_rn(r, fabs(e[i - 1]));
        if (i + 1 < n) {
            r = __dadd_rn(r, fabs(e[i]));
            const double t = __dmul_rn(e[i], e[i]);
            e2[i] = t;
            emax = fmax(emax, t);
        }
        lo = fmin(lo, __dsub_rn(d[i], r));
        hi = fmax(hi, __dadd_rn(d[i], r));
    }
    lo = -block_max(-lo, red);
    hi = block_max(hi, red);
    emax = block_max(emax, red);
    if (threadIdx.x == 0) {
        const double pivmin = __dmul_rn(DBL_MIN, emax);
        const double tnorm = fmax(fabs(lo), fabs(hi));
        const double pad = __dadd_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, (double)n), DBL_EPSILON), tnorm),
                                     __dmul_rn(4.0, pivmin));
        par[0] = __dsub_rn(lo, pad);
        par[1] = __dadd_rn(hi, pad);
        par[2] = pivmin;
        par[3] = tnorm;
        if (n > 0) e2[n - 1] = 0.0;
    }
}

__device__ __forceinline__ int sturm_count(int n, const double *__restrict__ d, const double *__restrict__ e2,
                                           double x, double pivmin) {
    int c = 0;
    double q = __dsub_rn(__ldg(d), x);
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < 0.0;
    for (int i = 1; i < n; ++i) {
        q = __dsub_rn(__dsub_rn(__ldg(d + i), x), __ddiv_rn(__ldg(e2 + i - 1), q));
        if (fabs(q) < pivmin) q = -pivmin;
        c += q < 0.0;
    }
    return c;
}

// One thread per eigenvalue index k (the (k+1)-th smallest).
__global__ void bisect_kernel(int n, const double *__restrict__ d, const double *__restrict__ e2,
                              const double *__restrict__ par, double rtol, int maxit, double *__restrict__ eigs,
                              int *err) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (n == 1) {
        eigs[0] = d[0];
        return;
    }
    const double pivmin = par[2];
    const double atol = __dmul_rn(rtol, par[3]);
    double lo = par[0], hi = par[1];
    int it = 0;
    for (;;) {
        const double w = __dsub_rn(hi, lo);
        const double mag = fmax(fabs(lo), fabs(hi));
        double tol = __dmul_rn(rtol, mag);
        if (atol > tol) tol = atol;
        if (w <= tol) break;
        if (it >= maxit) {
            latch_error(err, SEV_ERR_NOCONV);
            break;
        }
        const double mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(n, d, e2, mid, pivmin) >= k + 1)
            hi = mid;
        else
            lo = mid;
        ++it;
    }
    eigs[k] = __dmul_rn(0.5, __dadd_rn(lo, hi));
}

size_t bisect_workspace(int n) {
    Carver c(nullptr);
    c.take<double>((size_t)n + 1);
    c.take<double>(4);
    return c.bytes();
}

int launch_bisect(sev_ctx *h, int n, const double *d, const double *e, double rtol, double *eigs, void *ws,
                  size_t ws_bytes) {
    if (n <= 0) return SEV_OK;
    if (ws_bytes < bisect_workspace(n)) return SEV_ERR_WORKSPACE;
    Carver c(ws);
    double *e2 = c.take<double>((size_t)n + 1);
    double *par = c.take<double>(4);
    SEV_LAUNCH(h, K_BISECT_PREP, bisect_prep_kernel, 1, 1024, 0, n, d, e, e2, par);
    // one thread per eigenvalue; small blocks spread the indices over all SMs
    int bs = 64;
    while (bs > 32 && (n + bs - 1) / bs < h->sm_count) bs >>= 1;
    SEV_LAUNCH(h, K_BISECT, bisect_kernel, (n + bs - 1) / bs, bs, 0, n, d, e2, par, rtol, 200, eigs, h->d_err);
    return SEV_OK;
}

}  // namespace sev

// ------------------------------------------------- allocation-free variant
// sev_tridiag_bisect_static: the same two kernels as sev_tridiag_bisect, but
// their scratch (the squared off-diagonal, the Gershgorin/pivmin parameters
// and an unused status slot) lives in this file-scope device array instead
// of handle workspace, so a call allocates nothing.  The array is
// (kStaticMaxN + 8) doubles (~512 KiB) on every device that loads the
// library, held until the process exits.
namespace sev {
constexpr int kStaticMaxN = 65536;
static __device__ __align__(256) double g_bisect_scratch[kStaticMaxN + 8];

struct StaticScratch {
    double *ptr = nullptr;
    int sm_count = 0;
};
static StaticScratch g_static_dev[128];
}  // namespace sev

extern "C" int sev_tridiag_bisect_static(int n, const double *d, const double *e, double rtol, double *eigs,
                                         void *stream) {
    using namespace sev;
    if (n < 0 || n > kStaticMaxN) return -1;
    if (n > 0 && !d) return -2;
    if (n > 1 && !e) return -3;
    if (!(rtol >= 1e-16) || !(rtol < 1.0)) return -4;
    if (n > 0 && !eigs) return -5;
    if (n == 0) return SEV_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return SEV_ERR_CUDA;
    StaticScratch &S = g_static_dev[dev];
    if (!S.ptr) {
        // once per device, with that device current: the array's device
        // address (the host-side name is only a stand-in for it)
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bisect_scratch) != cudaSuccess) return SEV_ERR_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SEV_ERR_CUDA;
        S.sm_count = sms;
        S.ptr = (double *)p;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double *e2 = S.ptr;                   // n + 1 doubles
    double *par = S.ptr + kStaticMaxN + 2;  // 4 doubles
    int *status = (int *)(S.ptr + kStaticMaxN + 6);
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return SEV_ERR_CUDA;
    bisect_prep_kernel<<<1, 1024, 0, st>>>(n, d, n > 1 ? e : d, e2, par);
    if (cudaGetLastError() != cudaSuccess) return SEV_ERR_CUDA;
    int bs = 64;
    while (bs > 32 && (n + bs - 1) / bs < S.sm_count) bs >>= 1;
    bisect_kernel<<<(n + bs - 1) / bs, bs, 0, st>>>(n, d, e2, par, rtol, 200, eigs, status);
    return cudaGetLastError() == cudaSuccess ? SEV_OK : SEV_ERR_CUDA;
}
