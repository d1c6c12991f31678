// api.cu -- the C ABI (include/sev.h): handle, workspace, argument checks,
// per-kernel timing, and the eigvalsh driver that chains the stages of
// Algorithm 4.3: full-to-band, band-to-band stages b0 -> ... -> 1 (the stage
// widths come from schedule() below), and bisection on the final
// tridiagonal.
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <new>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace sev {

const char *const kKernelNames[K_COUNT] = {
    "bisect_prep",  "bisect",       "band_from_dense", "tridiag_extract", "band_chase", "band_tri",
    "tsqr_leaf_qr", "tsqr_node_qr", "tsqr_node_apply", "tsqr_leaf_apply", "recon_lu",
    "recon_u2",     "symm",         "vform_xt",        "vform_utx",       "vform_reduce",
    "vform_v",      "syr2k",        "split_bf16",      "syr2k_tc",        "batch",
    "check_finite", "misc"};

static cudaEvent_t pool_get(sev_ctx *h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void timing_begin(sev_ctx *h, int kid) {
    if (!((h->timing >> kid) & 1ULL)) return;
    TimedLaunch t;
    t.kid = kid;
    t.e0 = pool_get(h);
    t.e1 = pool_get(h);
    cudaEventRecord(t.e0, h->stream);
    h->pending.push_back(t);
}

void timing_end(sev_ctx *h, int kid) {
    if (!((h->timing >> kid) & 1ULL) || h->pending.empty()) return;
    TimedLaunch &t = h->pending.back();
    if (t.kid == kid) cudaEventRecord(t.e1, h->stream);
}

int check_launch(sev_ctx *) {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SEV_OK : SEV_ERR_CUDA;
}

static void drain_timing(sev_ctx *h) {
    for (TimedLaunch &t : h->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.e0, t.e1) == cudaSuccess) {
            h->tot_ms[t.kid] += ms;
            h->launches[t.kid] += 1;
        }
        h->event_pool.push_back(t.e0);
        h->event_pool.push_back(t.e1);
    }
    h->pending.clear();
}

int get_workspace(sev_ctx *h, size_t bytes, void **out) {
    if (h->ws_ext) {
        if (h->ws_ext_bytes < bytes) return SEV_ERR_WORKSPACE;
        *out = h->ws_ext;
        return SEV_OK;
    }
    if (h->ws_own_bytes < bytes) {
        if (h->ws_own) {
            cudaStreamSynchronize(h->stream);
            cudaFree(h->ws_own);
            h->ws_own = nullptr;
            h->ws_own_bytes = 0;
        }
        if (cudaMalloc(&h->ws_own, bytes) != cudaSuccess) {
            cudaGetLastError();
            return SEV_ERR_WORKSPACE;
        }
        h->ws_own_bytes = bytes;
    }
    *out = h->ws_own;
    return SEV_OK;
}

static int default_b0(int n, int prec) {
    if (prec == SEV_FP64) return n >= 4096 ? 64 : 32;
    return n >= 1024 ? 64 : 32;  // 64 -> 16 -> 1 measured best at n = 16384 (1.18 s against 1.51 s for 128)
}

// b0 for a call with b0 = 0: the autotuned width of the order's bucket if
// sev_autotune chose one on this handle, else the default rule.
static int pick_b0(const sev_ctx *h, int n, int prec) {
    const TunedBands *t = tuned_for(h, n, prec);
    return (t && t->b0 > 0) ? t->b0 : default_b0(n, prec);
}

// Band schedule (Algorithm 4.3; the paper allows a reduction factor k > 2
// per stage).  Measured on GB300 at n = 16384 (FP32): the one-stage b -> 1
// kernel is fastest from b = 16 (192 ms, against 366 ms from 32), a
// 32 -> 16 stage costs 139 ms, 64 -> 16 238 ms and 128 -> 32 372 ms (128 ->
// 16 607 ms, 128 -> 64 312 ms).  So: a band of width <= 16 the b -> 1
// kernel supports goes straight to 1; a band of 128 or more first goes to
// 32; a wider band that 16 divides goes to 16; otherwise to the widest
// supported width that divides it, or is halved; an odd band finishes with
// b -> 1.  b0 = 128 gives 128 -> 32 -> 16 -> 1, b0 = 64 gives 64 -> 16 -> 1.
static int schedule(int b0, int elem, int *out) {
    int k = 0;
    out[k++] = b0;
    while (out[k - 1] > 1) {
        const int b = out[k - 1];
        int next = b % 2 != 0 ? 1 : b / 2;
        if (b <= 16 && band_tri_supported(b, elem)) {
            next = 1;
        } else if (b >= 128 && b % 32 == 0) {
            next = 32;
        } else if (b > 16 && b % 16 == 0) {
            next = 16;
        } else if (band_tri_supported(b, elem)) {
            next = 1;
        } else {
            for (int w = 16; w >= 2; w >>= 1)
                if (band_tri_supported(w, elem) && b % w == 0 && w < b) {
                    next = w;
                    break;
                }
        }
        out[k++] = next;
    }
    return k;
}

template <typename T>
static int band_stage(sev_ctx *h, int n, T *AB, int ldab, int b, int hh, void *ws, size_t ws_bytes) {
    if (hh == 1 && band_tri_supported(b, (int)sizeof(T))) return launch_band_tri<T>(h, n, AB, ldab, b, ws, ws_bytes);
    return launch_band_to_band<T>(h, n, AB, ldab, b, hh, ws, ws_bytes);
}

// The stage widths sev_eigvalsh runs from b0: the autotuned table of the
// order's bucket when it reaches 1 from b0, else schedule().
static int stages_for(const sev_ctx *h, int n, int b0, int prec, int *out) {
    if (const TunedBands *t = tuned_for(h, n, prec)) {
        const int k = tuned_schedule(*t, b0, out, 40);
        if (k > 0) return k;
    }
    return schedule(b0, prec == SEV_FP64 ? 8 : 4, out);
}

template <typename T>
static size_t eig_workspace(sev_ctx *h, int n, int b0) {
    int sched[40];
    const int ns = stages_for(h, n, b0, sizeof(T) == 8 ? SEV_FP64 : SEV_MIXED, sched);
    const int ldab = 2 * b0 > 2 ? 2 * b0 : 2;
    size_t stage = bisect_workspace(n);
    if (b0 < n - 1) {
        const size_t f = full_to_band_workspace<T>(h, n, b0);
        if (f > stage) stage = f;
    }
    for (int s = 0; s + 1 < ns; ++s) {
        const size_t w = band_workspace(n, sched[s], sched[s + 1]);
        if (w > stage) stage = w;
    }
    if (band_tri_workspace(n) > stage) stage = band_tri_workspace(n);
    Carver c(nullptr);
    c.take<T>((size_t)ldab * n);
    c.take<double>((size_t)n);
    c.take<double>((size_t)n);
    c.take<int>(1);
    c.take<char>(stage);
    return c.bytes();
}

template <typename T>
static int eigvalsh_t(sev_ctx *h, int n, T *A, int lda, int b0, double *eigs) {
    if (b0 > n - 1) b0 = n - 1 > 1 ? n - 1 : 1;
    int sched[40];
    const int ns = stages_for(h, n, b0, sizeof(T) == 8 ? SEV_FP64 : SEV_MIXED, sched);
    for (int s = 0; s + 1 < ns; ++s)
        if (!(sched[s + 1] == 1 && band_tri_supported(sched[s], (int)sizeof(T))) &&
            band_smem_bytes<T>(sched[s], sched[s + 1]) > h->smem_optin)
            return SEV_ERR_UNSUPPORTED;
    const int ldab = 2 * b0 > 2 ? 2 * b0 : 2;
    void *ws = nullptr;
    const size_t need = eig_workspace<T>(h, n, b0);
    int rc = get_workspace(h, need, &ws);
    if (rc) return rc;
    Carver c(ws);
    T *AB = c.take<T>((size_t)ldab * n);
    double *d = c.take<double>((size_t)n);
    double *e = c.take<double>((size_t)n);
    int *nonfinite = c.take<int>(1);
    const size_t stage_bytes = need - c.bytes();
    void *stage = c.take<char>(stage_bytes);
    // non-finite input: latch SEV_ERR_NONFINITE; the reductions still run
    // (bounded work, no data-dependent control flow) and the bisection,
    // whose step count depends on the data, is skipped (NaN eigenvalues)
    SEV_CUDA(cudaMemsetAsync(nonfinite, 0, sizeof(int), h->stream));
    rc = launch_check_finite<T>(h, n, A, lda, nonfinite);
    if (rc) return rc;
    if (b0 < n - 1) {
        rc = launch_full_to_band<T>(h, n, A, lda, b0, AB, ldab, stage, stage_bytes);
    } else {
        rc = launch_band_from_dense<T>(h, n, A, lda, b0, AB, ldab);
    }
    if (rc) return rc;
    for (int s = 0; s + 1 < ns; ++s) {
        rc = band_stage<T>(h, n, AB, ldab, sched[s], sched[s + 1], stage, stage_bytes);
        if (rc) return rc;
    }
    rc = launch_tridiag_extract<T>(h, n, AB, ldab, d, e);
    if (rc) return rc;
    const double rtol = sizeof(T) == 8 ? 1e-14 : 1e-9;
    return launch_bisect(h, n, d, e, rtol, eigs, stage, stage_bytes, nonfinite);
}

}  // namespace sev

// ------------------------------------------------------------ batched plan
// A plan fixes the matrices (device pointers, orders, leading dimensions)
// and the band width of one batch, uploads the per-matrix descriptors once
// and reserves every workspace, so that running it only launches kernels.
// Matrices whose whole path fits one CTA's shared memory go to the batched
// kernel (batched.cu), largest first; the others run the single-matrix path
// one after another on the handle's stream.
struct sev_batch_s {
    int device = 0;
    int prec = SEV_MIXED;
    int b = 0;             // band width of the batched kernel
    int small_count = 0;   // matrices in the batched kernel
    int nmax_small = 0;
    int grid = 0;          // persistent CTAs of the batched launch
    void *d_mats = nullptr;  // descriptors (largest first), then the queue counter
    int *d_queue = nullptr;
    struct Big {
        void *A;
        double *eigs;
        int n, lda;
    };
    std::vector<Big> big;
};

namespace sev {

static int g_batch_small_max = 1024;

static int batch_default_b(sev_ctx *h, int prec) {
    const int tuned = prec == SEV_FP64 ? h->batch_b_fp64 : h->batch_b_mixed;
    if (tuned > 0) return tuned;
    return prec == SEV_FP64 ? 8 : 16;
}

static bool batch_fits(sev_ctx *h, int prec, int b, int n) {
    if (n > g_batch_small_max) return false;
    const size_t s = prec == SEV_FP64 ? batch_smem_bytes<double>(b, n) : batch_smem_bytes<float>(b, n);
    return s > 0 && s <= h->smem_optin;
}

static double batch_rtol(int prec) { return prec == SEV_FP64 ? 1e-14 : 1e-9; }

}  // namespace sev

using namespace sev;

extern "C" {

int sev_create(sev_handle *handle, int device) {
    if (!handle) return -1;
    *handle = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return device < 0 ? -2 : SEV_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SEV_ERR_CUDA;
    sev_ctx *h = new (std::nothrow) sev_ctx();
    if (!h) return SEV_ERR_WORKSPACE;
    h->device = device;
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    h->smem_optin = (size_t)optin;
    if (cudaMalloc(&h->d_err, sizeof(DevStatus)) != cudaSuccess) {
        delete h;
        return SEV_ERR_CUDA;
    }
    const DevStatus st0{0, 0, kWaitCyclesDefault};
    if (cudaMemcpy(h->d_err, &st0, sizeof(st0), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(h->d_err);
        delete h;
        return SEV_ERR_CUDA;
    }
    if (const char *v = getenv("SEV_LEAF_ROWS")) h->leaf_rows_override = atoi(v);
    if (const char *v = getenv("SEV_CHASE_X3_MIN_B")) h->chase_x3_min_b = atoi(v);
    tune_cache_load(h);
    *handle = h;
    return SEV_OK;
}

int sev_destroy(sev_handle h) {
    if (!h) return -1;
    for (TimedLaunch &t : h->pending) {
        cudaEventDestroy(t.e0);
        cudaEventDestroy(t.e1);
    }
    for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
    if (h->ws_own) cudaFree(h->ws_own);
    if (h->h_stage) cudaFree(h->h_stage);
    if (h->d_err) cudaFree(h->d_err);
    delete h;
    return SEV_OK;
}

int sev_set_stream(sev_handle h, void *stream) {
    if (!h) return -1;
    h->stream = (cudaStream_t)stream;
    return SEV_OK;
}

int sev_workspace_query(sev_handle h, int n, int b0, int prec, size_t *bytes) {
    if (!h) return -1;
    if (n < 0) return -2;
    if (b0 < 0) return -3;
    if (prec != SEV_FP64 && prec != SEV_MIXED) return -4;
    if (!bytes) return -5;
    if (n == 0) {
        *bytes = 0;
        return SEV_OK;
    }
    if (b0 == 0) b0 = pick_b0(h, n, prec);
    if (b0 > n - 1) b0 = n - 1 > 1 ? n - 1 : 1;
    *bytes = prec == SEV_FP64 ? eig_workspace<double>(h, n, b0) : eig_workspace<float>(h, n, b0);
    return SEV_OK;
}

int sev_set_workspace(sev_handle h, void *ws, size_t bytes) {
    if (!h) return -1;
    if (ws && ((uintptr_t)ws & 255)) return -2;
    h->ws_ext = bytes ? ws : nullptr;
    h->ws_ext_bytes = ws ? bytes : 0;
    return SEV_OK;
}

int sev_eigvalsh(sev_handle h, int n, void *A, int lda, int b0, int prec, double *eigs) {
    if (!h) return -1;
    if (n < 0) return -2;
    if (n > 0 && !A) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (b0 < 0) return -5;
    if (prec != SEV_FP64 && prec != SEV_MIXED) return -6;
    if (n > 0 && !eigs) return -7;
    if (n == 0) return SEV_OK;
    if (cudaSetDevice(h->device) != cudaSuccess) return SEV_ERR_CUDA;
    if (b0 == 0) b0 = pick_b0(h, n, prec);
    if (n == 1) {
        // a 1 x 1 matrix: its entry is the eigenvalue
        const int rc = prec == SEV_FP64 ? launch_check_finite<double>(h, 1, (const double *)A, lda, nullptr)
                                        : launch_check_finite<float>(h, 1, (const float *)A, lda, nullptr);
        if (rc) return rc;
        if (prec == SEV_FP64) {
            SEV_CUDA(cudaMemcpyAsync(eigs, A, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
            return SEV_OK;
        }
        return launch_tridiag_extract<float>(h, 1, (const float *)A, 1, eigs, eigs);
    }
    return prec == SEV_FP64 ? eigvalsh_t<double>(h, n, (double *)A, lda, b0, eigs)
                            : eigvalsh_t<float>(h, n, (float *)A, lda, b0, eigs);
}

int sev_eigvalsh_host(sev_handle h, int n, const void *A_host, int lda, int b0, int prec, double *eigs_host) {
    if (!h) return -1;
    if (n < 0) return -2;
    if (n > 0 && !A_host) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (b0 < 0) return -5;
    if (prec != SEV_FP64 && prec != SEV_MIXED) return -6;
    if (n > 0 && !eigs_host) return -7;
    if (n == 0) return SEV_OK;
    if (cudaSetDevice(h->device) != cudaSuccess) return SEV_ERR_CUDA;
    const size_t es = prec == SEV_FP64 ? sizeof(double) : sizeof(float);
    const size_t abytes = ((es * (size_t)n * n + 255) & ~(size_t)255);
    const size_t need = abytes + sizeof(double) * (size_t)n;
    if (h->h_stage_bytes < need) {
        if (h->h_stage) {
            cudaStreamSynchronize(h->stream);
            cudaFree(h->h_stage);
            h->h_stage = nullptr;
            h->h_stage_bytes = 0;
        }
        if (cudaMalloc(&h->h_stage, need) != cudaSuccess) {
            cudaGetLastError();
            return SEV_ERR_WORKSPACE;
        }
        h->h_stage_bytes = need;
    }
    void *dA = h->h_stage;
    double *dE = (double *)((char *)h->h_stage + abytes);
    SEV_CUDA(cudaMemcpy2DAsync(dA, es * n, A_host, es * lda, es * n, n, cudaMemcpyHostToDevice, h->stream));
    int rc = sev_eigvalsh(h, n, dA, n, b0, prec, dE);
    if (rc) return rc;
    SEV_CUDA(cudaMemcpyAsync(eigs_host, dE, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    return sev_get_error(h);
}

int sev_full_to_band(sev_handle h, int n, void *A, int lda, int b, int prec, void *AB, int ldab) {
    if (!h) return -1;
    if (n < 0) return -2;
    if (n > 0 && !A) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (b < 1) return -5;
    if (prec != SEV_FP64 && prec != SEV_MIXED) return -6;
    if (n > 0 && !AB) return -7;
    if (ldab < b + 1) return -8;
    if (n == 0) return SEV_OK;
    if (cudaSetDevice(h->device) != cudaSuccess) return SEV_ERR_CUDA;
    if (b >= n - 1) {
        return prec == SEV_FP64 ? launch_band_from_dense<double>(h, n, (double *)A, lda, b, (double *)AB, ldab)
                                : launch_band_from_dense<float>(h, n, (float *)A, lda, b, (float *)AB, ldab);
    }
    const size_t need = prec == SEV_FP64 ? full_to_band_workspace<double>(h, n, b) : full_to_band_workspace<float>(h, n, b);
    void *ws = nullptr;
    int rc = get_workspace(h, need, &ws);
    if (rc) return rc;
    rc = prec == SEV_FP64 ? launch_check_finite<double>(h, n, (const double *)A, lda, nullptr)
                          : launch_check_finite<float>(h, n, (const float *)A, lda, nullptr);
    if (rc) return rc;
    return prec == SEV_FP64 ? launch_full_to_band<double>(h, n, (double *)A, lda, b, (double *)AB, ldab, ws, need)
                            : launch_full_to_band<float>(h, n, (float *)A, lda, b, (float *)AB, ldab, ws, need);
}

int sev_band_to_band(sev_handle h, int n, void *AB, int ldab, int b, int hh, int prec) {
    if (!h) return -1;
    if (n < 0) return -2;
    if (n > 0 && !AB) return -3;
    if (ldab < 2 * b) return -4;
    if (b < 2) return -5;
    if (hh < 1 || hh >= b || b % hh != 0) return -6;
    if (prec != SEV_FP64 && prec != SEV_MIXED) return -7;
    if (n == 0) return SEV_OK;
    if (cudaSetDevice(h->device) != cudaSuccess) return SEV_ERR_CUDA;
    const bool tri = hh == 1 && band_tri_supported(b, prec == SEV_FP64 ? 8 : 4);
    if (!tri && (prec == SEV_FP64 ? band_smem_bytes<double>(b, hh) : band_smem_bytes<float>(b, hh)) > h->smem_optin)
        return SEV_ERR_UNSUPPORTED;
    const size_t need = tri ? band_tri_workspace(n) : band_workspace(n, b, hh);
    void *ws = nullptr;
    int rc = get_workspace(h, need, &ws);
    if (rc) return rc;
    return prec == SEV_FP64 ? band_stage<double>(h, n, (double *)AB, ldab, b, hh, ws, need)
                            : band_stage<float>(h, n, (float *)AB, ldab, b, hh, ws, need);
}

int sev_tridiag_bisect(sev_handle h, int n, const double *d, const double *e, double rtol, double *eigs) {
    if (!h) return -1;
    if (n < 0) return -2;
    if (n > 0 && !d) return -3;
    if (n > 1 && !e) return -4;
    if (!(rtol > 0.0) || !(rtol < 1.0)) return -5;
    if (n > 0 && !eigs) return -6;
    if (n == 0) return SEV_OK;
    if (cudaSetDevice(h->device) != cudaSuccess) return SEV_ERR_CUDA;
    const size_t need = bisect_workspace(n);
    void *ws = nullptr;
    int rc = get_workspace(h, need, &ws);
    if (rc) return rc;
    return launch_bisect(h, n, d, n > 1 ? e : d, rtol, eigs, ws, need);
}

int sev_band_tridiag_extract(sev_handle h, int n, const void *AB, int ldab, int prec, double *d, double *e) {
    if (!h) return -1;
    if (n < 0) return -2;
    if (n > 0 && !AB) return -3;
    if (ldab < 2) return -4;
    if (prec != SEV_FP64 && prec != SEV_MIXED) return -5;
    if (n > 0 && !d) return -6;
    if (n > 1 && !e) return -7;
    if (n == 0) return SEV_OK;
    if (cudaSetDevice(h->device) != cudaSuccess) return SEV_ERR_CUDA;
    return prec == SEV_FP64 ? launch_tridiag_extract<double>(h, n, (const double *)AB, ldab, d, e ? e : d)
                            : launch_tridiag_extract<float>(h, n, (const float *)AB, ldab, d, e ? e : d);
}

int sev_batch_plan_create(sev_handle h, int count, const int *n, const int *lda, void *const *A, double *const *eigs,
                          int b, int prec, sev_batch_plan *plan) {
    if (!plan) return -9;
    *plan = nullptr;
    if (!h) return -1;
    if (count < 0) return -2;
    if (count > 0 && (!n || !lda || !A || !eigs)) return -3;
    if (b < 0) return -7;
    if (prec != SEV_FP64 && prec != SEV_MIXED) return -8;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 0) return -3;
        if (n[i] > 0 && (!A[i] || !eigs[i] || lda[i] < n[i])) return -3;
    }
    if (cudaSetDevice(h->device) != cudaSuccess) return SEV_ERR_CUDA;
    if (b == 0) b = batch_default_b(h, prec);
    if (!batch_supported(b, prec == SEV_FP64 ? 8 : 4)) return SEV_ERR_UNSUPPORTED;
    sev_batch_s *P = new (std::nothrow) sev_batch_s();
    if (!P) return SEV_ERR_WORKSPACE;
    P->device = h->device;
    P->prec = prec;
    P->b = b;
    std::vector<int> order;
    for (int i = 0; i < count; ++i) {
        if (n[i] <= 0) continue;
        if (batch_fits(h, prec, b, n[i]))
            order.push_back(i);
        else
            P->big.push_back({A[i], eigs[i], n[i], lda[i]});
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return n[x] > n[y]; });
    P->small_count = (int)order.size();
    P->nmax_small = order.empty() ? 0 : n[order[0]];
    if (!order.empty()) {
        const size_t mb = batch_mat_bytes();
        const size_t bytes = ((mb * order.size() + 255) & ~(size_t)255) + 256;
        std::vector<unsigned char> host(bytes, 0);
        for (size_t k = 0; k < order.size(); ++k) {
            const int i = order[k];
            batch_pack_mat(host.data() + k * mb, A[i], eigs[i], n[i], lda[i]);
        }
        if (cudaMalloc(&P->d_mats, bytes) != cudaSuccess) {
            delete P;
            return SEV_ERR_WORKSPACE;
        }
        if (cudaMemcpy(P->d_mats, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(P->d_mats);
            delete P;
            return SEV_ERR_CUDA;
        }
        P->d_queue = (int *)((char *)P->d_mats + bytes - 256);
        const int rc = prec == SEV_FP64 ? prepare_batch_small<double>(h, P->small_count, b, P->nmax_small, &P->grid)
                                        : prepare_batch_small<float>(h, P->small_count, b, P->nmax_small, &P->grid);
        if (rc) {
            cudaFree(P->d_mats);
            delete P;
            return rc;
        }
    }
    // reserve the single-matrix workspace now, so that running the plan allocates nothing
    size_t need = 0;
    for (const auto &g : P->big) {
        const int b0 = pick_b0(h, g.n, prec);
        const size_t w = prec == SEV_FP64 ? eig_workspace<double>(h, g.n, b0 > g.n - 1 ? g.n - 1 : b0)
                                          : eig_workspace<float>(h, g.n, b0 > g.n - 1 ? g.n - 1 : b0);
        if (w > need) need = w;
    }
    if (need) {
        void *ws = nullptr;
        const int rc = get_workspace(h, need, &ws);
        if (rc) {
            if (P->d_mats) cudaFree(P->d_mats);
            delete P;
            return rc;
        }
    }
    *plan = P;
    return SEV_OK;
}

int sev_batch_run(sev_handle h, sev_batch_plan P) {
    if (!h) return -1;
    if (!P) return -2;
    if (P->device != h->device) return -2;
    if (cudaSetDevice(h->device) != cudaSuccess) return SEV_ERR_CUDA;
    int rc = SEV_OK;
    if (P->small_count > 0) {
        rc = P->prec == SEV_FP64
                 ? launch_batch_small<double>(h, P->small_count, P->d_mats, P->d_queue, P->b, P->nmax_small,
                                              batch_rtol(P->prec), P->grid)
                 : launch_batch_small<float>(h, P->small_count, P->d_mats, P->d_queue, P->b, P->nmax_small,
                                             batch_rtol(P->prec), P->grid);
        if (rc) return rc;
    }
    for (const auto &g : P->big) {
        rc = sev_eigvalsh(h, g.n, g.A, g.lda, 0, P->prec, g.eigs);
        if (rc) return rc;
    }
    return SEV_OK;
}

int sev_batch_plan_destroy(sev_batch_plan P) {
    if (!P) return -1;
    if (P->d_mats) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(P->device);
        cudaFree(P->d_mats);
        cudaSetDevice(cur);
    }
    delete P;
    return SEV_OK;
}

int sev_batch_plan_info(sev_batch_plan P, int *b, int *small_count, int *large_count) {
    if (!P) return -1;
    if (b) *b = P->b;
    if (small_count) *small_count = P->small_count;
    if (large_count) *large_count = (int)P->big.size();
    return SEV_OK;
}

int sev_eigvalsh_batched(sev_handle h, int count, const int *n, const int *lda, void *const *A, int b, int prec,
                         double *const *eigs) {
    sev_batch_plan P = nullptr;
    int rc = sev_batch_plan_create(h, count, n, lda, A, eigs, b, prec, &P);
    if (rc) return rc;
    rc = sev_batch_run(h, P);
    // the descriptors must outlive the launch
    if (cudaStreamSynchronize(h->stream) != cudaSuccess && rc == SEV_OK) rc = SEV_ERR_CUDA;
    sev_batch_plan_destroy(P);
    return rc;
}

int sev_batch_autotune(sev_handle h, int count, const int *n, int prec, int *b_best) {
    if (!h) return -1;
    if (count < 0) return -2;
    if (count > 0 && !n) return -3;
    if (prec != SEV_FP64 && prec != SEV_MIXED) return -4;
    if (!b_best) return -5;
    if (cudaSetDevice(h->device) != cudaSuccess) return SEV_ERR_CUDA;
    const int elem = prec == SEV_FP64 ? 8 : 4;
    const int cands[] = {4, 8, 16, 32};
    // a strided sample (at most 4096) of the sizes that fit the batched kernel at the narrowest band
    std::vector<int> sizes;
    for (int i = 0; i < count; ++i)
        if (n[i] > 0 && batch_fits(h, prec, 8, n[i])) sizes.push_back(n[i]);
    std::sort(sizes.begin(), sizes.end());
    std::vector<int> sample;
    const size_t want = sizes.size() < 4096 ? sizes.size() : 4096;
    for (size_t k = 0; k < want; ++k) sample.push_back(sizes[k * sizes.size() / want]);
    *b_best = 0;
    if (sample.empty()) return SEV_OK;
    size_t total = 0;
    std::vector<size_t> off;
    for (int m : sample) {
        off.push_back(total);
        total += (((size_t)elem * m * m + 255) & ~(size_t)255) + (((size_t)8 * m + 255) & ~(size_t)255);
    }
    void *buf = nullptr;
    if (cudaMalloc(&buf, total) != cudaSuccess) return SEV_ERR_WORKSPACE;
    std::vector<void *> As(sample.size());
    std::vector<double *> Es(sample.size());
    for (size_t k = 0; k < sample.size(); ++k) {
        As[k] = (char *)buf + off[k];
        Es[k] = (double *)((char *)As[k] + (((size_t)elem * sample[k] * sample[k] + 255) & ~(size_t)255));
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 0.f;
    int rc = SEV_OK;
    for (int b : cands) {
        if (!batch_supported(b, elem)) continue;
        bool ok = true;
        for (int m : sample) ok = ok && batch_fits(h, prec, b, m);
        if (!ok) continue;
        sev_batch_plan P = nullptr;
        rc = sev_batch_plan_create(h, (int)sample.size(), sample.data(), sample.data(), As.data(), Es.data(), b, prec,
                                   &P);
        if (rc) break;
        float ms = 0.f;
        for (int rep = 0; rep < 2 && rc == SEV_OK; ++rep) {  // warm-up, then timed
            rc = prec == SEV_FP64 ? launch_batch_fill<double>(h, P->small_count, P->d_mats, 0x5EEDull)
                                  : launch_batch_fill<float>(h, P->small_count, P->d_mats, 0x5EEDull);
            if (rc) break;
            cudaEventRecord(e0, h->stream);
            rc = sev_batch_run(h, P);
            cudaEventRecord(e1, h->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = SEV_ERR_CUDA;
            cudaEventElapsedTime(&ms, e0, e1);
        }
        sev_batch_plan_destroy(P);
        if (rc) break;
        if (*b_best == 0 || ms < best_ms) {
            best_ms = ms;
            *b_best = b;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc) return rc;
    if (prec == SEV_FP64)
        h->batch_b_fp64 = *b_best;
    else
        h->batch_b_mixed = *b_best;
    return SEV_OK;
}

int sev_band_schedule(int n, int b0, int prec, int *bands, int max_bands) {
    if (n < 0) return -1;
    if (b0 < 0) return -2;
    if (prec != SEV_FP64 && prec != SEV_MIXED) return -3;
    if (!bands) return -4;
    if (n <= 1) return 0;
    if (b0 == 0) b0 = default_b0(n, prec);
    if (b0 > n - 1) b0 = n - 1 > 1 ? n - 1 : 1;
    int sched[40];
    const int ns = schedule(b0, prec == SEV_FP64 ? 8 : 4, sched);
    if (ns > max_bands) return -5;
    for (int k = 0; k < ns; ++k) bands[k] = sched[k];
    return ns;
}

int sev_eigvalsh_bands(sev_handle h, int n, int b0, int prec, int *bands, int max_bands) {
    if (!h) return -1;
    if (n < 0) return -2;
    if (b0 < 0) return -3;
    if (prec != SEV_FP64 && prec != SEV_MIXED) return -4;
    if (!bands) return -5;
    if (n <= 1) return 0;
    if (b0 == 0) b0 = pick_b0(h, n, prec);
    if (b0 > n - 1) b0 = n - 1 > 1 ? n - 1 : 1;
    int sched[40];
    const int ns = stages_for(h, n, b0, prec, sched);
    if (ns > max_bands) return -6;
    for (int k = 0; k < ns; ++k) bands[k] = sched[k];
    return ns;
}

int sev_get_error(sev_handle h) {
    if (!h) return -1;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SEV_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SEV_ERR_CUDA;
    if (v) cudaMemset(h->d_err, 0, sizeof(int));
    return v;
}

int sev_set_wait_limit(sev_handle h, long long cycles) {
    if (!h) return -1;
    if (cycles < 0) return -2;
    if (cudaSetDevice(h->device) != cudaSuccess) return SEV_ERR_CUDA;
    const long long v = cycles == 0 ? kWaitCyclesDefault : cycles;
    // ordered after the work already enqueued on the handle's stream
    SEV_CUDA(cudaStreamSynchronize(h->stream));
    SEV_CUDA(cudaMemcpy((char *)h->d_err + offsetof(DevStatus, wait_cycles), &v, sizeof(v), cudaMemcpyHostToDevice));
    return SEV_OK;
}

const char *sev_status_string(int code) {
    if (code < 0) return "invalid argument";
    switch (code) {
        case SEV_OK: return "ok";
        case SEV_ERR_NONFINITE: return "input holds NaN or Inf";
        case SEV_ERR_NOCONV: return "bisection did not converge within its iteration cap";
        case SEV_ERR_TIMEOUT: return "a device-side wait hit its iteration cap";
        case SEV_ERR_CUDA: return "CUDA runtime error";
        case SEV_ERR_WORKSPACE: return "workspace too small or allocation failed";
        case SEV_ERR_UNSUPPORTED: return "unsupported parameter combination";
        case SEV_ERR_INTERNAL: return "internal index check failed";
        default: return "unknown status";
    }
}

int sev_set_kernel_timing(sev_handle h, unsigned long long mask) {
    if (!h) return -1;
    h->timing = mask;
    return SEV_OK;
}

int sev_kernel_count(void) { return K_COUNT; }

const char *sev_kernel_name(int k) { return (k >= 0 && k < K_COUNT) ? kKernelNames[k] : ""; }

int sev_kernel_time(sev_handle h, int k, double *total_ms, long *launches, int reset) {
    if (!h) return -1;
    if (k < 0 || k >= K_COUNT) return -2;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SEV_ERR_CUDA;
    drain_timing(h);
    if (total_ms) *total_ms = h->tot_ms[k];
    if (launches) *launches = h->launches[k];
    if (reset) {
        h->tot_ms[k] = 0.0;
        h->launches[k] = 0;
    }
    return SEV_OK;
}

}  // extern "C"
