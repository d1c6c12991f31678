// common.cuh -- internal declarations shared by the sev library's translation
// units: the handle, kernel ids and timing, workspace carving, and the
// CTA-cooperative device helpers (reductions, Householder reflector, QR of a
// shared-memory block, small shared-memory GEMMs, packed-band access).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cfloat>
#include <cmath>
#include <vector>

#include "../../include/sev.h"

namespace sev {

// ----------------------------------------------------------------- kernel ids
enum KernelId {
    K_BISECT_PREP = 0,
    K_BISECT,
    K_BAND_FROM_DENSE,
    K_TRIDIAG_EXTRACT,
    K_BAND_CHASE,
    K_TSQR_LEAF,
    K_TSQR_TREE,
    K_TSQR_DOWN,
    K_TSQR_LEAF_Q,
    K_RECON_LU,
    K_RECON_U2,
    K_SYMM,
    K_VFORM_XT,
    K_VFORM_UTX,
    K_VFORM_REDUCE,
    K_VFORM_V,
    K_SYR2K,
    K_SPLIT_BF16,
    K_SYR2K_TC,
    K_SYMM_TC,
    K_MISC,
    K_COUNT
};
extern const char *const kKernelNames[K_COUNT];

// ---------------------------------------------------------------- the handle
struct TimedLaunch {
    int kid;
    cudaEvent_t e0, e1;
};

}  // namespace sev

struct sev_ctx {
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    cudaStream_t stream = nullptr;
    void *ws_own = nullptr;
    size_t ws_own_bytes = 0;
    void *ws_ext = nullptr;
    size_t ws_ext_bytes = 0;
    int *d_err = nullptr;       // device error word (first error latched)
    void *h_stage = nullptr;    // device staging buffer for the host entry point
    size_t h_stage_bytes = 0;
    unsigned long long timing = 0;  // bit k: time kernel id k
    int leaf_rows_override = 0;  // SEV_LEAF_ROWS: rows per tree-QR leaf (tests)
    std::vector<sev::TimedLaunch> pending;
    std::vector<cudaEvent_t> event_pool;
    double tot_ms[sev::K_COUNT] = {};
    long launches[sev::K_COUNT] = {};
};

namespace sev {

// -------------------------------------------------------------- host helpers
void timing_begin(sev_ctx *h, int kid);
void timing_end(sev_ctx *h, int kid);
int check_launch(sev_ctx *h);

#define SEV_LAUNCH(h, kid, kernel, grid, block, smem, ...)                  \
    do {                                                                    \
        ::sev::timing_begin((h), (kid));                                    \
        kernel<<<(grid), (block), (smem), (h)->stream>>>(__VA_ARGS__);      \
        ::sev::timing_end((h), (kid));                                      \
        int _rc = ::sev::check_launch(h);                                   \
        if (_rc) return _rc;                                                \
    } while (0)

#define SEV_CUDA(call)                                                      \
    do {                                                                    \
        if ((call) != cudaSuccess) return SEV_ERR_CUDA;                     \
    } while (0)

// Carve 256-byte aligned pieces out of a workspace buffer.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base((char *)b) {}
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = (T *)(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
    size_t bytes() const { return (off + 255) & ~(size_t)255; }
};

// Returns a device workspace of at least `bytes`, owned by the caller (set
// with sev_set_workspace) or by the handle (grown with cudaMalloc).
int get_workspace(sev_ctx *h, size_t bytes, void **out);

// Device error codes latched in *err (first one wins).
__device__ __forceinline__ void latch_error(int *err, int code) { atomicCAS(err, 0, code); }

constexpr int kThreads = 256;
constexpr long kSpinCap = 20000000;  // ~ a few seconds of polling with back-off

// ------------------------------------------------------ reductions (CTA-wide)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum over the CTA; every thread receives the total.  red: >= 32 doubles of
// shared scratch.  Contains two __syncthreads.
__device__ __forceinline__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = lane < nw ? red[lane] : 0.0;
    return warp_sum(r);
}
__device__ __forceinline__ double block_max(double v, double *red) {
    v = warp_max(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = lane < nw ? red[lane] : 0.0;
    return warp_max(r);
}

// ------------------------------------------------------------- Householder
// Reflector of the column segment x[0..m-1] (shared memory, stride 1), in
// the "always reflect" convention: beta = -sgn(alpha)||x|| (sgn(0) = +1),
// tau = (beta - alpha)/beta in [1, 2]; zero vector -> tau = beta = 0.  The
// norm, beta and tau are computed in FP64 whatever T is.  x[1..m-1] is
// scaled in place to v[1..m-1] (v[0] = 1 implicit); x[0] is NOT modified.
// Ends with a __syncthreads (scaled vector visible to the CTA).
template <typename T>
__device__ void cta_house(int m, T *x, double *red, double *tau_out, double *beta_out) {
    const double alpha = (double)x[0];
    double ssq = 0.0;
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) {
        double t = (double)x[i];
        ssq += t * t;
    }
    ssq = block_sum(ssq, red);
    double scale = 1.0;
    if (sizeof(T) == 8 && ((ssq != 0.0 && ssq < 1e-280) || !(ssq < 1e300) || fabs(alpha) > 1e150)) {
        // rare path: rescale by an exact power of two so squares neither
        // overflow nor underflow
        double amax = fabs(alpha);
        for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) amax = fmax(amax, fabs((double)x[i]));
        amax = block_max(amax, red);
        int e2;
        frexp(amax, &e2);
        scale = ldexp(1.0, -e2);
        ssq = 0.0;
        for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) {
            double t = (double)x[i] * scale;
            ssq += t * t;
        }
        ssq = block_sum(ssq, red);
    }
    double tau, beta;
    if (ssq == 0.0 && alpha == 0.0) {
        tau = 0.0;
        beta = 0.0;
    } else {
        const double as = alpha * scale;
        const double nrm = sqrt(as * as + ssq) / scale;
        beta = alpha < 0.0 ? nrm : -nrm;
        tau = (beta - alpha) / beta;
        const double inv = 1.0 / (alpha - beta);
        for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) x[i] = (T)((double)x[i] * inv);
    }
    *tau_out = tau;
    *beta_out = beta;
    __syncthreads();
}

// Householder QR of the m x nc block P (shared memory, column-major, ld):
// r = min(nc, m-1) reflectors.  On return R is in the upper trapezoid, the
// Householder vectors are stored below the diagonal (unit diagonal
// implicit) and tau[0..r-1] holds the scalars.  Returns r.
template <typename T>
__device__ int cta_qr(int m, int nc, T *P, int ld, T *tau, double *red) {
    const int r = nc < m - 1 ? nc : m - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < r; ++k) {
        double tk, bk;
        cta_house(m - k, &P[k + (size_t)k * ld], red, &tk, &bk);
        const T tkt = (T)tk;
        if (tk != 0.0) {
            for (int c = k + 1 + warp; c < nc; c += nw) {
                T *col = &P[(size_t)c * ld];
                const T *v = &P[(size_t)k * ld];
                T s = 0;
                for (int i = k + lane; i < m; i += 32) s += (i == k ? col[i] : v[i] * col[i]);
                s = warp_sum(s) * tkt;
                for (int i = k + lane; i < m; i += 32) col[i] -= (i == k ? s : s * v[i]);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            P[k + (size_t)k * ld] = (T)bk;
            tau[k] = tkt;
        }
        __syncthreads();
    }
    return r;
}

// Compact-WY factor T (r x r, upper, ldt) from the Householder vectors held
// below the diagonal of P (as left by cta_qr) and tau:
//   T[k,k] = tau_k,  T[0:k,k] = -tau_k T[0:k,0:k] (U[:,0:k]^T U[:,k]).
// G: r x r shared scratch (ldg) for U^T U.  Ends with a __syncthreads.
template <typename T>
__device__ void cta_form_t(int m, int r, const T *P, int ld, const T *tau, T *Tm, int ldt, T *G, int ldg) {
    // G[a,c] = sum_i U[i,a] U[i,c] for a < c  (U[i,c] = 0 for i < c, 1 at i = c)
    for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
        const int a = idx % r, c = idx / r;
        if (a >= c) continue;
        const T *ua = &P[(size_t)a * ld], *uc = &P[(size_t)c * ld];
        T s = ua[c];  // i = c: U[c,a] * 1
        for (int i = c + 1; i < m; ++i) s += ua[i] * uc[i];
        G[a + (size_t)c * ldg] = s;
    }
    for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
        const int a = idx % r, c = idx / r;
        Tm[a + (size_t)c * ldt] = (a == c) ? tau[c] : T(0);
    }
    __syncthreads();
    for (int k = 1; k < r; ++k) {
        for (int a = threadIdx.x; a < k; a += blockDim.x) {
            T s = 0;
            for (int q = a; q < k; ++q) s += Tm[a + (size_t)q * ldt] * G[q + (size_t)k * ldg];
            Tm[a + (size_t)k * ldt] = -tau[k] * s;
        }
        __syncthreads();
    }
}

// Explicit unit lower-trapezoidal U (m x r, ldu) from the vectors stored
// below the diagonal of P; columns r..rp-1 are zero-filled.
template <typename T>
__device__ void cta_extract_u(int m, int r, int rp, const T *P, int ld, T *U, int ldu) {
    for (int idx = threadIdx.x; idx < m * rp; idx += blockDim.x) {
        const int i = idx % m, c = idx / m;
        T v = 0;
        if (c < r) v = (i < c) ? T(0) : (i == c ? T(1) : P[i + (size_t)c * ld]);
        U[i + (size_t)c * ldu] = v;
    }
}

// C = alpha * op(A) op(B) + beta * C on shared-memory operands (column-major).
// op(A) is M x K, op(B) is K x N.  TA: A stored K x M; TB: B stored N x K.
template <typename T, bool TA, bool TB>
__device__ void cta_gemm(int M, int N, int K, T alpha, const T *A, int lda, const T *B, int ldb, T beta, T *C,
                         int ldc) {
    for (int idx = threadIdx.x; idx < M * N; idx += blockDim.x) {
        const int m = idx % M, n = idx / M;
        T acc = 0;
        for (int k = 0; k < K; ++k) {
            const T a = TA ? A[k + (size_t)m * lda] : A[m + (size_t)k * lda];
            const T b = TB ? B[n + (size_t)k * ldb] : B[k + (size_t)n * ldb];
            acc += a * b;
        }
        T *c = &C[m + (size_t)n * ldc];
        *c = (beta == T(0)) ? alpha * acc : alpha * acc + beta * *c;
    }
}

// ---------------------------------------------------- packed-band addressing
// AB[d + j*ldab] = A(j + d, j).  Loads bypass L1 (other CTAs write the band).
template <typename T>
__device__ __forceinline__ T ld_cg(const T *p) {
    return __ldcg(p);
}

// ------------------------------------------------------------- launchers
// bisect.cu
template <typename T>
int launch_band_from_dense(sev_ctx *h, int n, const T *A, int lda, int b, T *AB, int ldab);
template <typename T>
int launch_tridiag_extract(sev_ctx *h, int n, const T *AB, int ldab, double *d, double *e);
int launch_bisect(sev_ctx *h, int n, const double *d, const double *e, double rtol, double *eigs, void *ws,
                  size_t ws_bytes);
size_t bisect_workspace(int n);

// band.cu
template <typename T>
int launch_band_to_band(sev_ctx *h, int n, T *AB, int ldab, int b, int hh, void *ws, size_t ws_bytes);
size_t band_workspace(int n, int b, int hh);
template <typename T>
size_t band_smem_bytes(int b, int hh);

// panel.cu + update.cu
template <typename T>
int launch_full_to_band(sev_ctx *h, int n, T *A, int lda, int b, T *AB, int ldab, void *ws, size_t ws_bytes);
template <typename T>
size_t full_to_band_workspace(sev_ctx *h, int n, int b);

}  // namespace sev
