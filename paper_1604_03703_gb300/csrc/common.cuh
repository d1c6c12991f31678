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
    K_BAND_TRI,
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
    K_BATCH,
    K_CHECK_FINITE,
    K_MISC,
    K_COUNT
};
extern const char *const kKernelNames[K_COUNT];

// ---------------------------------------------------------------- the handle
struct TimedLaunch {
    int kid;
    cudaEvent_t e0, e1;
};

// Autotuned band schedule for one bucket of orders and precision: next[k]
// is the width after 2^k (0: none), b0 the chosen first width (0: none).
constexpr int kTuneWidths = 8;  // widths 1, 2, 4, ..., 128
struct TunedBands {
    int bucket = 0, prec = 0, b0 = 0;
    int next[kTuneWidths] = {};
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
    int *d_err = nullptr;       // device status block (DevStatus): error word, wait limit
    void *h_stage = nullptr;    // device staging buffer for the host entry point
    size_t h_stage_bytes = 0;
    unsigned long long timing = 0;  // bit k: time kernel id k
    int leaf_rows_override = 0;  // SEV_LEAF_ROWS: rows per tree-QR leaf (tests)
    int chase_x3_min_b = 64;     // SEV_CHASE_X3_MIN_B: narrowest band chased by three-CTA clusters
    int batch_b_fp64 = 0;        // band width chosen by sev_batch_autotune (0: default)
    int batch_b_mixed = 0;
    std::vector<sev::TunedBands> tuned;  // sev_autotune results
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
// The handle's device status block: the latched error word (first error
// wins), then the time limit of every device-side wait in SM clock cycles
// (default ~2 s at 2 GHz; sev_set_wait_limit changes it per handle).  Kernels
// receive a pointer to it as `int *err`.
struct DevStatus {
    int err;
    int pad;
    long long wait_cycles;
};
constexpr long long kWaitCyclesDefault = 4000000000LL;
__device__ __forceinline__ long long wait_cap(const int *err) {
    return reinterpret_cast<const DevStatus *>(err)->wait_cycles;
}
__device__ __forceinline__ bool wait_expired(long long t0, const int *err) { return clock64() - t0 > wait_cap(err); }

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
// On this part every FP64 instruction has ~64 cycles of latency and an IEEE
// FP64 division or square root ~650, so the reflector scalars below avoid
// both while staying FP64-accurate:
//  * the sum of squares of FP32 data is accumulated as an unevaluated pair
//    of floats with error-free transformations (x^2 split exactly by an FMA,
//    Knuth's TwoSum for the additions), reduced across the warp in that
//    form and finished in FP64 -- the relative error is ~2^-44, far below
//    what the FP64 scalars need;
//  * 1/||x|| and 1/(alpha - beta) come from an FP32 hardware seed refined by
//    two Newton steps in FP64 (y <- y + y(1 - s y^2)/2 and
//    r <- r + r(1 - d r)): 22 correct bits become full double precision.
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {  // TwoSum of the leading parts, then renormalise
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    const float lo = e + a.lo + b.lo;
    const float hi = s + lo;
    return {hi, lo - (hi - s)};
}
__device__ __forceinline__ void f2_add_sq(F2 &a, float x) {
    const float p = x * x;
    const float pe = fmaf(x, x, -p);  // x^2 = p + pe exactly
    a = f2_add(a, F2{p, pe});
}
template <int WIDTH = 32>
__device__ __forceinline__ F2 warp_sum_f2(F2 v) {
#pragma unroll
    for (int o = WIDTH / 2; o > 0; o >>= 1) {
        F2 w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = f2_add(v, w);
    }
    return v;
}

// 2^k for |k| < 1000, by building the exponent field.
__device__ __forceinline__ double pow2i(int k) { return __hiloint2double((1023 + k) << 20, 0); }

// Householder scalars in FP64 from alpha = x_0 and ssq = sum_{i>0} x_i^2:
// beta = -sgn(alpha) sqrt(alpha^2 + ssq) (sgn(0) = +1), tau = (beta - alpha)/beta,
// inv = 1/(alpha - beta); a zero vector gives tau = beta = inv = 0.
__device__ __forceinline__ void house_scalars(double alpha, double ssq, double *tau, double *beta, double *inv) {
    const double s = fma(alpha, alpha, ssq);
    if (!(s > 0.0)) {
        *tau = *beta = *inv = 0.0;
        return;
    }
    // seed for s^(-1/2): s = m 2^(2k), m in [2^-2, 2^2)
    const int e = ((__double2hiint(s) >> 20) & 0x7ff) - 1023;
    const int k = e >> 1;
    const double m = s * pow2i(-2 * k);
    double y = (double)rsqrtf((float)m) * pow2i(-k);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double t = s * y;
        const double eps = fma(-t, y, 1.0);  // 1 - s y^2
        y = fma(0.5 * y, eps, y);
    }
    double nrm = s * y;
    nrm = fma(0.5 * y, fma(-nrm, nrm, s), nrm);  // one correction of the square root itself
    const double aa = fabs(alpha);
    *beta = alpha < 0.0 ? nrm : -nrm;
    const double d = aa + nrm;  // |alpha - beta|
    *tau = d * y;               // (nrm + |alpha|) / nrm
    // 1/d: seed from FP32 on the scaled value, two Newton steps
    const int ed = ((__double2hiint(d) >> 20) & 0x7ff) - 1023;
    const double dm = d * pow2i(-ed);
    double r = (double)(1.0f / (float)dm) * pow2i(-ed);
#pragma unroll
    for (int it = 0; it < 2; ++it) r = fma(r, fma(-d, r, 1.0), r);
    *inv = alpha < 0.0 ? -r : r;  // alpha - beta = sgn(alpha) d
}

// The same scalars for FP32 data, evaluated in pair-float arithmetic (an
// unevaluated sum of two floats, ~48 significant bits) and rounded to FP32:
// on GB300 every FP64 warp instruction holds a sub-partition's FP64 pipe for
// ~64 cycles, so the FP64 chain above costs ~1700 cycles per reflector and
// this one ~240 -- and the reflector's scalars sit on the critical path of
// every QR step and bulge chase.  s = alpha^2 + ssq is formed error-free
// (TwoProd, TwoSum); sqrt(s) is the FP32 rsqrt estimate times s, corrected
// once with the exact residual s - q^2 (an FMA); tau = d / nrm and
// 1/d (d = |alpha| + nrm) each take one correction step with their exact
// residuals.  On 2^20 random inputs over 12 decades the FP32 results equal
// the FP64 evaluation rounded to FP32 (a GPU test keeps checking this).
__device__ __forceinline__ F2 two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
// The same from s = alpha^2 + ssq given directly (pair-float).
__device__ __forceinline__ void house_scalars_f2s(float alpha, F2 s, float *tau, float *beta, float *inv) {
    if (!(s.hi > 0.f)) {
        *tau = *beta = *inv = 0.f;
        return;
    }
    const float y = rsqrtf(s.hi);
    const float q = s.hi * y;
    const float r = fmaf(-q, q, s.hi) + s.lo;  // s - q^2, q^2 split exactly by the FMA
    const float ql = r * (0.5f * y);
    F2 nrm;
    nrm.hi = q + ql;
    nrm.lo = ql - (nrm.hi - q);
    const float aa = fabsf(alpha);
    *beta = alpha < 0.f ? nrm.hi : -nrm.hi;
    const F2 d = f2_add(nrm, F2{aa, 0.f});
    const float rn = 1.0f / nrm.hi;
    const float t0 = d.hi * rn;
    const float rt = fmaf(-t0, nrm.hi, d.hi) + (d.lo - t0 * nrm.lo);  // d - t0 nrm
    *tau = fmaf(rt, rn, t0);
    const float r0 = 1.0f / d.hi;
    const float e = fmaf(-d.hi, r0, 1.0f) - d.lo * r0;  // 1 - d r0
    const float iv = fmaf(r0, e, r0);
    *inv = alpha < 0.f ? -iv : iv;  // alpha - beta = sgn(alpha) d
}
__device__ __forceinline__ void house_scalars_f2(float alpha, F2 ssq, float *tau, float *beta, float *inv) {
    house_scalars_f2s(alpha, f2_add(ssq, two_prod(alpha, alpha)), tau, beta, inv);
}

// Reflector of the column segment x[0..m-1] (shared memory, stride 1),
// computed by ONE warp, in the "always reflect" convention:
// beta = -sgn(alpha)||x|| (sgn(0) = +1), tau = (beta - alpha)/beta in [1, 2];
// a zero vector gives tau = beta = 0.  Norm, beta and tau are FP64-accurate
// (see above); the scalars are formed in lane 0 and broadcast.  On return
// x[1..m-1] holds v[1..m-1] (v[0] = 1 implicit), x[0] = beta and
// *tau_out = tau.
template <typename T>
__device__ double warp_house(int m, T *x, T *tau_out) {
    const int lane = threadIdx.x & 31;
    const double alpha = (double)x[0];
    double ssq;
    if (sizeof(T) == 4) {
        F2 acc{0.f, 0.f};
        for (int i = 1 + lane; i < m; i += 32) f2_add_sq(acc, (float)x[i]);
        acc = warp_sum_f2(acc);
        float tau = 0.f, beta = 0.f, inv = 0.f;
        house_scalars_f2((float)x[0], acc, &tau, &beta, &inv);
        if (tau != 0.f)
            for (int i = 1 + lane; i < m; i += 32) x[i] = (T)((float)x[i] * inv);
        __syncwarp();
        if (lane == 0) {
            x[0] = (T)beta;
            *tau_out = (T)tau;
        }
        __syncwarp();
        return (double)tau;
    } else {
        double a = 0.0;
        for (int i = 1 + lane; i < m; i += 32) {
            const double t = (double)x[i];
            a = fma(t, t, a);
        }
        ssq = warp_sum(a);
        if ((ssq != 0.0 && ssq < 1e-280) || !(ssq < 1e300) || fabs(alpha) > 1e150 ||
            (alpha != 0.0 && fabs(alpha) < 1e-140)) {
            // rare path for FP64 data: rescale by an exact power of two
            double amax = fabs(alpha);
            for (int i = 1 + lane; i < m; i += 32) amax = fmax(amax, fabs((double)x[i]));
            amax = warp_max(amax);
            int e2;
            frexp(amax, &e2);
            const double sc = ldexp(1.0, -e2);
            double a2 = 0.0;
            for (int i = 1 + lane; i < m; i += 32) {
                const double t = (double)x[i] * sc;
                a2 = fma(t, t, a2);
            }
            a2 = warp_sum(a2);
            double tau = 0.0, beta = 0.0, inv = 0.0;
            if (lane == 0) house_scalars(alpha * sc, a2, &tau, &beta, &inv);
            tau = __shfl_sync(0xffffffffu, tau, 0);
            beta = __shfl_sync(0xffffffffu, beta, 0) / sc;
            inv = __shfl_sync(0xffffffffu, inv, 0) * sc;
            if (tau != 0.0)
                for (int i = 1 + lane; i < m; i += 32) x[i] = (T)((double)x[i] * inv);
            __syncwarp();
            if (lane == 0) {
                x[0] = (T)beta;
                *tau_out = (T)tau;
            }
            __syncwarp();
            return tau;
        }
    }
    double tau = 0.0, beta = 0.0, inv = 0.0;
    if (lane == 0) house_scalars(alpha, ssq, &tau, &beta, &inv);
    tau = __shfl_sync(0xffffffffu, tau, 0);
    if (tau != 0.0) {
        const T invt = (T)__shfl_sync(0xffffffffu, inv, 0);
        for (int i = 1 + lane; i < m; i += 32) x[i] = x[i] * invt;
    }
    __syncwarp();
    if (lane == 0) {
        x[0] = (T)beta;
        *tau_out = (T)tau;
    }
    __syncwarp();
    return tau;
}

// H = I - tau v v^T applied by one warp to up to four column segments
// col[k..m-1] (v[k] = 1 implicit, v[k+1..] stored); the four dot products
// are reduced together so their shuffle chains overlap.
template <typename T>
__device__ __forceinline__ void warp_apply4(int m, int k, const T *v, T tk, T *c0, T *c1, T *c2, T *c3) {
    const int lane = threadIdx.x & 31;
    T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int i = k + lane; i < m; i += 32) {
        const T vi = (i == k) ? T(1) : v[i];
        s0 += vi * c0[i];
        if (c1) s1 += vi * c1[i];
        if (c2) s2 += vi * c2[i];
        if (c3) s3 += vi * c3[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    }
    s0 *= tk;
    s1 *= tk;
    s2 *= tk;
    s3 *= tk;
    for (int i = k + lane; i < m; i += 32) {
        const T vi = (i == k) ? T(1) : v[i];
        c0[i] -= s0 * vi;
        if (c1) c1[i] -= s1 * vi;
        if (c2) c2[i] -= s2 * vi;
        if (c3) c3[i] -= s3 * vi;
    }
    __syncwarp();
}
template <typename T>
__device__ __forceinline__ void warp_apply2(int m, int k, const T *v, T tk, T *c0, T *c1) {
    warp_apply4(m, k, v, tk, c0, c1, (T *)nullptr, (T *)nullptr);
}

// The owner warp's step of cta_qr for FP32 data with the column segment in
// registers (rows k + lane + 32t, up to 256 rows): apply H_k to it
// (do_apply), then form reflector k+1 from its rows k+1.. (do_house) --
// pair-float sum of squares in two independent accumulators, pair-float
// scalars -- and store the segment once.  Same results as warp_apply2 +
// warp_house up to the order of the FP32 dot product's terms.
__device__ __forceinline__ void warp_apply_house_f32(int m, int k, const float *v, float tk, float *col,
                                                     float *tau_next, bool do_apply, bool do_house) {
    const int lane = threadIdx.x & 31;
    float x[8], vv[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int row = k + lane + 32 * t;
        const bool in = row < m;
        x[t] = in ? col[row] : 0.f;
        vv[t] = in ? (row == k ? 1.f : v[row]) : 0.f;
    }
    if (do_apply) {
        float d0 = 0.f, d1 = 0.f;
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            d0 = fmaf(x[t], vv[t], d0);
            d1 = fmaf(x[t + 1], vv[t + 1], d1);
        }
        const float sc = tk * warp_sum(d0 + d1);
#pragma unroll
        for (int t = 0; t < 8; ++t) x[t] = fmaf(-sc, vv[t], x[t]);
    }
    if (do_house) {
        F2 a0{0.f, 0.f}, a1{0.f, 0.f};
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int row = k + lane + 32 * t;
            if (row >= k + 2 && row < m) {
                if (t & 1)
                    f2_add_sq(a1, x[t]);
                else
                    f2_add_sq(a0, x[t]);
            }
        }
        const F2 acc = warp_sum_f2(f2_add(a0, a1));
        const float alpha = __shfl_sync(0xffffffffu, x[0], 1);  // row k + 1
        float tau = 0.f, beta = 0.f, inv = 0.f;
        house_scalars_f2(alpha, acc, &tau, &beta, &inv);
        if (tau != 0.f) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int row = k + lane + 32 * t;
                if (row >= k + 2) x[t] *= inv;
            }
        }
        if (lane == 1) x[0] = beta;
        if (lane == 0) *tau_next = tau;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int row = k + lane + 32 * t;
        if (row < m) col[row] = x[t];
    }
    __syncwarp();
}

// Householder QR of the m x nc block P (shared memory, column-major, ld):
// r = min(nc, m-1) reflectors.  At step k the warp `own` = (k+1) mod nw
// applies H_k to column k+1 and forms reflector k+1 (lookahead) and nothing
// else, keeping the serial per-column chain short (FP32 with m-k <= 256: the
// fused register-resident warp_apply_house_f32 with pair-float scalars;
// otherwise warp_apply2 then warp_house), while the other warps apply H_k
// to columns k+2.. , four at a time.  One
// __syncthreads per step.  On return R is in the upper trapezoid, the
// Householder vectors below the diagonal (unit diagonal implicit) and
// tau[0..r-1] holds the scalars.  Returns r.
template <typename T>
__device__ int cta_qr(int m, int nc, T *P, int ld, T *tau, double * /*unused*/) {
    const int r = nc < m - 1 ? nc : m - 1;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (r <= 0) {
        __syncthreads();
        return r < 0 ? 0 : r;
    }
    if (warp == 0) warp_house(m, P, &tau[0]);
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        const T tk = tau[k];
        const T *v = P + (size_t)k * ld;
        const int own = (k + 1) % nw;
        if (warp == own) {
            if constexpr (sizeof(T) == 4) {
                if (m - k <= 256 && k + 1 < nc) {
                    warp_apply_house_f32(m, k, (const float *)v, (float)tk, (float *)(P + (size_t)(k + 1) * ld),
                                         (float *)&tau[k + 1], tk != T(0), k + 1 < r);
                } else {
                    if (tk != T(0) && k + 1 < nc) warp_apply2(m, k, v, tk, P + (size_t)(k + 1) * ld, (T *)nullptr);
                    if (k + 1 < r) warp_house(m - k - 1, P + (k + 1) + (size_t)(k + 1) * ld, &tau[k + 1]);
                }
            } else {
                if (tk != T(0) && k + 1 < nc) warp_apply2(m, k, v, tk, P + (size_t)(k + 1) * ld, (T *)nullptr);
                if (k + 1 < r) warp_house(m - k - 1, P + (k + 1) + (size_t)(k + 1) * ld, &tau[k + 1]);
            }
        } else if (tk != T(0)) {
            // the other nw - 1 warps share columns k+2 .. nc-1
            const int q = nw - 1;
            const int widx = (warp - own - 1 + nw) % nw;
            for (int c = k + 2 + widx; c < nc; c += 4 * q) {
                T *c1 = (c + q < nc) ? P + (size_t)(c + q) * ld : (T *)nullptr;
                T *c2 = (c + 2 * q < nc) ? P + (size_t)(c + 2 * q) * ld : (T *)nullptr;
                T *c3 = (c + 3 * q < nc) ? P + (size_t)(c + 3 * q) * ld : (T *)nullptr;
                warp_apply4(m, k, v, tk, P + (size_t)c * ld, c1, c2, c3);
            }
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
// Each thread computes a 4 x 4 block of C: rows mb + Mb*i (interleaved, so
// a warp's A loads hit consecutive addresses) and columns 4*nb + j (a
// warp's B loads are broadcasts).
template <typename T, bool TA, bool TB>
__device__ void cta_gemm(int M, int N, int K, T alpha, const T *A, int lda, const T *B, int ldb, T beta, T *C,
                         int ldc) {
    const int Mb = (M + 3) >> 2, Nb = (N + 3) >> 2;
    for (int blk = threadIdx.x; blk < Mb * Nb; blk += blockDim.x) {
        const int mb = blk % Mb, nb = blk / Mb;
        int mi[4];
        bool mv[4], nv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            mi[i] = mb + Mb * i;
            mv[i] = mi[i] < M;
            if (!mv[i]) mi[i] = M - 1;
            nv[i] = 4 * nb + i < N;
        }
        T acc[4][4] = {};
        // unrolled so later k's loads issue ahead of the FMAs (each output's
        // sum keeps its k order: the results do not change)
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
            T a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = TA ? A[k + (size_t)mi[i] * lda] : A[mi[i] + (size_t)k * lda];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = nv[j] ? 4 * nb + j : N - 1;
                bb[j] = TB ? B[n + (size_t)k * ldb] : B[k + (size_t)n * ldb];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!mv[i] || !nv[j]) continue;
                T *c = &C[mi[i] + (size_t)(4 * nb + j) * ldc];
                *c = (beta == T(0)) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *c;
            }
    }
}

// C = alpha * (A1 B1 + A2 B2) + beta * C on shared-memory operands with
// register tiles: every thread computes TM x TN outputs, rows m0 .. m0+TM-1
// (consecutive: threads with consecutive blocks read consecutive addresses)
// and columns n0 .. n0+TN-1 (threads of a warp mostly share them: broadcast
// reads).  A_p(m, k) = A_p[m + k lda] (m contiguous); B_p(k, n) =
// B_p[n + k ldb] when BT (n contiguous) else B_p[k + n ldb].  The second
// pair is skipped when K2 = 0.  VEC (T = float only): lda, ldb, ldc are
// multiples of 4 and the bases 16-byte aligned, so full tiles use float4
// loads; ragged tiles fall back to clamped scalar reads (never outside the
// M x K / K x N operands).  Each output sums its k terms in order (A1 B1
// first); no barrier inside.  LOWER (M = N, TM = TN): only the tiles on or
// below the diagonal are computed, numbered consecutively so that the busy
// threads fill whole warps (the diagonal tiles are computed in full).
template <typename T, int TM, int TN, bool BT, bool VEC, bool LOWER = false>
__device__ void cta_mm(int M, int N, int K1, T alpha, const T *A1, int lda1, const T *B1, int ldb1, int K2,
                       const T *A2, int lda2, const T *B2, int ldb2, T beta, T *C, int ldc) {
    static_assert(!VEC || (sizeof(T) == 4 && TM % 4 == 0 && (!BT || TN % 4 == 0)), "vector loads need float tiles");
    static_assert(!LOWER || TM == TN, "lower-triangle tiles need square tiles");
    const int Mb = (M + TM - 1) / TM, Nb = (N + TN - 1) / TN;
    const int ntiles = LOWER ? Mb * (Mb + 1) / 2 : Mb * Nb;
    for (int blk = threadIdx.x; blk < ntiles; blk += blockDim.x) {
        int m0, n0;
        if constexpr (LOWER) {
            // tile t of the lower triangle, row by row: I (I + 1) / 2 <= t
            int I = (int)((sqrtf(8.f * (float)blk + 1.f) - 1.f) * 0.5f);
            while ((I + 1) * (I + 2) / 2 <= blk) ++I;
            while (I * (I + 1) / 2 > blk) --I;
            m0 = I * TM;
            n0 = (blk - I * (I + 1) / 2) * TN;
        } else {
            m0 = (blk % Mb) * TM;
            n0 = (blk / Mb) * TN;
        }
        const bool full = m0 + TM <= M && n0 + TN <= N;
        T acc[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
        for (int p = 0; p < 2; ++p) {
            const int K = p == 0 ? K1 : K2;
            const T *A = p == 0 ? A1 : A2;
            const T *B = p == 0 ? B1 : B2;
            const int lda = p == 0 ? lda1 : lda2, ldb = p == 0 ? ldb1 : ldb2;
            if (K <= 0) continue;
            if (VEC && full) {
#pragma unroll 2
                for (int k = 0; k < K; ++k) {
                    T a[TM], bb[TN];
#pragma unroll
                    for (int i = 0; i < TM; i += 4) {
                        const float4 v = *reinterpret_cast<const float4 *>(A + m0 + i + (size_t)k * lda);
                        a[i] = v.x;
                        a[i + 1] = v.y;
                        a[i + 2] = v.z;
                        a[i + 3] = v.w;
                    }
                    if constexpr (BT) {
#pragma unroll
                        for (int j = 0; j < TN; j += 4) {
                            const float4 v = *reinterpret_cast<const float4 *>(B + n0 + j + (size_t)k * ldb);
                            bb[j] = v.x;
                            bb[j + 1] = v.y;
                            bb[j + 2] = v.z;
                            bb[j + 3] = v.w;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < TN; ++j) bb[j] = B[k + (size_t)(n0 + j) * ldb];
                    }
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * bb[j];
                }
            } else {
                int mi[TM], nj[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) mi[i] = m0 + i < M ? m0 + i : M - 1;
#pragma unroll
                for (int j = 0; j < TN; ++j) nj[j] = n0 + j < N ? n0 + j : N - 1;
#pragma unroll 2
                for (int k = 0; k < K; ++k) {
                    T a[TM], bb[TN];
#pragma unroll
                    for (int i = 0; i < TM; ++i) a[i] = A[mi[i] + (size_t)k * lda];
#pragma unroll
                    for (int j = 0; j < TN; ++j) bb[j] = BT ? B[nj[j] + (size_t)k * ldb] : B[k + (size_t)nj[j] * ldb];
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * bb[j];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                if (m0 + i >= M || n0 + j >= N) continue;
                T *c = &C[(m0 + i) + (size_t)(n0 + j) * ldc];
                *c = (beta == T(0)) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *c;
            }
    }
}

// --------------------------------------------------- blocked (level-3) QR
// Householder QR of the m x nc block P in panels of kQrNB columns: each
// panel is factorised column by column (cta_qr, reflectors applied inside
// the panel only), its compact-WY factor T_j formed (cta_form_t), and the
// trailing columns updated at once, C <- (I - V T_j^T V^T) C = C - V (T_j^T
// (V^T C)), as two shared-memory GEMMs -- each trailing element is read and
// written twice per panel instead of twice per reflector.  The reflectors
// and the result are those of cta_qr up to rounding.  T_j (upper, jb x jb)
// is left in Tblk at columns [j0, j0 + jb) (an kQrNB x nc array, ld kQrNB).
// Scratch: Wk (kQrNB x nc), Gb and Rs (kQrNB x kQrNB).  Returns r = min(nc, m-1).
constexpr int kQrNB = 32;

// Compact-WY factor T (r x r, r <= 32, upper, ldt) from G = V^T V (ldg) and
// tau by the forward recurrence T[0:k, k] = -tau_k T[0:k, 0:k] G[0:k, k],
// T[k, k] = tau_k, run by warp 0 (lane a owns row a).  Ends with a
// __syncthreads.
template <typename T>
__device__ void form_t_from_g(int r, const T *G, int ldg, const T *tau, T *Tm, int ldt) {
    if ((threadIdx.x >> 5) == 0) {
        const int a = threadIdx.x & 31;
        for (int k = 0; k < r; ++k) {
            T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
            int q = 0;
            for (; q + 4 <= k; q += 4) {  // T[a, q] = 0 for q < a (written at step q); rows a >= r unused
                s0 += Tm[a + (size_t)q * ldt] * G[q + (size_t)k * ldg];
                s1 += Tm[a + (size_t)(q + 1) * ldt] * G[q + 1 + (size_t)k * ldg];
                s2 += Tm[a + (size_t)(q + 2) * ldt] * G[q + 2 + (size_t)k * ldg];
                s3 += Tm[a + (size_t)(q + 3) * ldt] * G[q + 3 + (size_t)k * ldg];
            }
            for (; q < k; ++q) s0 += Tm[a + (size_t)q * ldt] * G[q + (size_t)k * ldg];
            const T s = (s0 + s1) + (s2 + s3);
            if (a < r) Tm[a + (size_t)k * ldt] = a < k ? -tau[k] * s : (a == k ? tau[k] : T(0));
            __syncwarp();
        }
    }
    __syncthreads();
}

template <typename T>
__device__ int cta_qr_blocked(int m, int nc, T *P, int ld, T *tau, T *Tblk, T *Wk, T *Gb, T *Rs) {
    const int r = nc < m - 1 ? nc : m - 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (r <= 0) {
        __syncthreads();
        return r < 0 ? 0 : r;
    }
    for (int j0 = 0; j0 < r; j0 += kQrNB) {
        const int jb = r - j0 < kQrNB ? r - j0 : kQrNB;
        T *Pj = P + j0 + (size_t)j0 * ld;
        const int mj = m - j0;
        const int rj = cta_qr(mj, jb, Pj, ld, tau + j0, nullptr);  // = jb: j0 + jb <= r <= m - 1
        // V explicit in place (unit diagonal, zeros above); R's triangle saved in Rs
        for (int idx = tid; idx < jb * jb; idx += nt) {
            const int i = idx % jb, c = idx / jb;
            if (i <= c) {
                Rs[i + (size_t)c * kQrNB] = Pj[i + (size_t)c * ld];
                Pj[i + (size_t)c * ld] = i == c ? T(1) : T(0);
            }
        }
        __syncthreads();
        T *Tj = Tblk + (size_t)j0 * kQrNB;
        cta_gemm<T, true, false>(rj, rj, mj, T(1), Pj, ld, Pj, ld, T(0), Gb, kQrNB);  // G = V^T V
        __syncthreads();
        form_t_from_g(rj, Gb, kQrNB, tau + j0, Tj, kQrNB);
        const int nct = nc - j0 - jb;
        if (nct > 0) {
            T *C = Pj + (size_t)jb * ld;
            cta_gemm<T, true, false>(jb, nct, mj, T(1), Pj, ld, C, ld, T(0), Wk, kQrNB);  // W = V^T C
            __syncthreads();
            for (int c = tid; c < nct; c += nt) {  // W <- T^T W, bottom row first (in place)
                T *w = Wk + (size_t)c * kQrNB;
                for (int i = jb - 1; i >= 0; --i) {
                    T acc = 0;
                    for (int q = 0; q <= i; ++q) acc += Tj[q + (size_t)i * kQrNB] * w[q];
                    w[i] = acc;
                }
            }
            __syncthreads();
            cta_gemm<T, false, false>(mj, nct, jb, T(-1), Pj, ld, Wk, kQrNB, T(1), C, ld);  // C -= V W
            __syncthreads();
        }
        for (int idx = tid; idx < jb * jb; idx += nt) {
            const int i = idx % jb, c = idx / jb;
            if (i <= c) Pj[i + (size_t)c * ld] = Rs[i + (size_t)c * kQrNB];
        }
        __syncthreads();
    }
    return r;
}

// M (rows x w, ld) <- H_0 H_1 ... H_{nr-1} M with the reflectors held
// explicitly (unit lower trapezoidal) in Y (rows x nr, ld) and the blocked
// compact-WY factors of cta_qr_blocked in Tblk: block by block from the
// last, M <- M - V (T_j (V^T M)).  Scratch Wk (kQrNB x w).
template <typename T>
__device__ void cta_apply_blocked(int rows, int w, int nr, const T *Y, int ld, const T *Tblk, T *M, T *Wk) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nblk = (nr + kQrNB - 1) / kQrNB;
    for (int jbk = nblk - 1; jbk >= 0; --jbk) {
        const int j0 = jbk * kQrNB;
        const int jb = nr - j0 < kQrNB ? nr - j0 : kQrNB;
        const T *V = Y + j0 + (size_t)j0 * ld;
        const T *Tj = Tblk + (size_t)j0 * kQrNB;
        T *Mj = M + j0;
        const int mj = rows - j0;
        cta_gemm<T, true, false>(jb, w, mj, T(1), V, ld, Mj, ld, T(0), Wk, kQrNB);  // W = V^T M
        __syncthreads();
        for (int c = tid; c < w; c += nt) {  // W <- T W, top row first (in place)
            T *wc = Wk + (size_t)c * kQrNB;
            for (int i = 0; i < jb; ++i) {
                T acc = 0;
                for (int q = i; q < jb; ++q) acc += Tj[i + (size_t)q * kQrNB] * wc[q];
                wc[i] = acc;
            }
        }
        __syncthreads();
        cta_gemm<T, false, false>(mj, w, jb, T(-1), V, ld, Wk, kQrNB, T(1), Mj, ld);  // M -= V W
        __syncthreads();
    }
}

// --------------------------------------------------- batched global copies
// Copy `count` elements, element k read by src(k) (a global load) and written
// by dst(k, v), with U independent loads in flight per thread before any of
// them is stored: a plain load-then-store loop would wait one full memory
// latency per element.  Threads [t0, t0 + nt) of the block take part.
template <typename T, int U = 8, typename Src, typename Dst>
__device__ __forceinline__ void batched_copy(int count, int t, int nt, Src src, Dst dst) {
    for (int base = t; base < count; base += U * nt) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = base + u * nt;
            v[u] = k < count ? src(k) : T{};
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = base + u * nt;
            if (k < count) dst(k, v[u]);
        }
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
// skip (device, may be null): when *skip != 0 at run time the bisection does
// no work and writes NaN eigenvalues (set by launch_check_finite).
int launch_bisect(sev_ctx *h, int n, const double *d, const double *e, double rtol, double *eigs, void *ws,
                  size_t ws_bytes, const int *skip = nullptr);
// Scans the lower triangle of A (n x n, lda); if it holds a NaN or an Inf,
// latches SEV_ERR_NONFINITE and sets *flag (device, may be null; the caller
// zeroes it first).
template <typename T>
int launch_check_finite(sev_ctx *h, int n, const T *A, int lda, int *flag);
size_t bisect_workspace(int n);

// band.cu
template <typename T>
int launch_band_to_band(sev_ctx *h, int n, T *AB, int ldab, int b, int hh, void *ws, size_t ws_bytes);
size_t band_workspace(int n, int b, int hh);
template <typename T>
size_t band_smem_bytes(int b, int hh);

// band_tri.cu: b -> 1 in one stage for b in {2, 4, 8, 16, 32}
int band_tri_supported(int b, int elem);
size_t band_tri_workspace(int n);
template <typename T>
int launch_band_tri(sev_ctx *h, int n, T *AB, int ldab, int b, void *ws, size_t ws_bytes);

// batched.cu: one CTA per matrix, whole path, persistent over a queue
int batch_supported(int b, int elem);
template <typename T>
size_t batch_smem_bytes(int b, int nmax);
template <typename T>
int prepare_batch_small(sev_ctx *h, int count, int b, int nmax, int *grid);
template <typename T>
int launch_batch_small(sev_ctx *h, int count, const void *mats, int *queue, int b, int nmax, double rtol, int grid);
size_t batch_mat_bytes();
void batch_pack_mat(void *dst, void *A, double *eigs, int n, int lda);
template <typename T>
int launch_batch_fill(sev_ctx *h, int count, const void *mats, unsigned long long seed);

// autotune.cu
int tune_bucket(int n);
const TunedBands *tuned_for(const sev_ctx *h, int n, int prec);
int tuned_schedule(const TunedBands &t, int b0, int *out, int max_out);
void tune_cache_load(sev_ctx *h);

// update.cu: Y = sum of the K-split partial products (N x b each, split order)
int launch_symm_reduce(sev_ctx *h, int N, int b, int splits, const float *part, float *Y);

// panel.cu + panel_reg.cu + update.cu
// Buffers of the register-resident panel factorisation (panel_reg.cu).
template <typename T>
struct RegPanelBufs {
    T *Yleaf, *Ynode, *tau, *Rbuf, *Zbuf, *Q, *Winv;
    int *nref;
};
template <typename T>
int reg_panel_supported(int b);
template <typename T>
int reg_panel_factor(sev_ctx *h, int N, int b, T *P, int lda, T *U, T *Tm, const RegPanelBufs<T> &B);
// T and the band block of a one-leaf panel (U explicit, tau, R from the leaf QR).
template <typename T>
int panel_finish_single_leaf(sev_ctx *h, int N, int b, const T *U, const T *tau, const int *nref, const T *R, T *Tm,
                             T *P, int lda);
// U[b:N] = Q[b:N] W1^{-1}; zeroes the panel below its top b rows.
template <typename T>
int panel_form_u2(sev_ctx *h, int N, int b, const T *Q, const T *Winv, T *U, T *P, int lda);
template <typename T>
int launch_full_to_band(sev_ctx *h, int n, T *A, int lda, int b, T *AB, int ldab, void *ws, size_t ws_bytes);
template <typename T>
size_t full_to_band_workspace(sev_ctx *h, int n, int b);

}  // namespace sev
