// bisect.cu -- eigenvalues of the final symmetric tridiagonal by Sturm-count
// bisection (the last step of Algorithm 4.3, which returns the tridiagonal's
// eigenvalues as the result), plus the
// small copy kernels between dense, packed-band and tridiagonal storage.
//
// The bisection runs on T scaled by an exact power of two 2^-s that brings
// its Gershgorin bound into [0.5, 1).  The Sturm count at x is the number of
// sign changes of the leading principal minors of T - xI (Sturm's theorem),
//   p_1 = d_0 - x,  p_{i+1} = (d_i - x) p_i - e_{i-1}^2 p_{i-1},
// the division-free form of the LDL^T pivot count: per step one FMA on the
// dependence chain (instead of a ~1000-cycle FP64 division), the pair
// (p_{i-1}, p_i) rescaled by a power of two when |p_i| leaves
// [2^-256, 2^256], a zero minor counted as a sign change.  Every FP64
// operation is written with an explicit round-to-nearest intrinsic so no
// multiply-add is contracted: the result is the exact IEEE evaluation of the
// recurrence in the order written.
#include <atomic>

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

// Non-finite scan of the lower triangle (diagonal included): CTA c takes
// columns c, c + grid, ...; its threads read down a column (coalesced).
template <typename T>
__global__ void check_finite_kernel(int n, const T *__restrict__ A, int lda, int *__restrict__ flag, int *err) {
    bool bad = false;
    for (int j = blockIdx.x; j < n; j += gridDim.x)
        for (int i = j + threadIdx.x; i < n; i += blockDim.x) bad |= !isfinite(A[(size_t)i + (size_t)j * lda]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) {
        latch_error(err, SEV_ERR_NONFINITE);
        if (flag) atomicExch(flag, 1);
    }
}

template <typename T>
int launch_check_finite(sev_ctx *h, int n, const T *A, int lda, int *flag) {
    if (n <= 0) return SEV_OK;
    int grid = n < h->sm_count * 8 ? n : h->sm_count * 8;
    SEV_LAUNCH(h, K_CHECK_FINITE, check_finite_kernel<T>, grid, kThreads, 0, n, A, lda, flag, h->d_err);
    return SEV_OK;
}

template int launch_check_finite<float>(sev_ctx *, int, const float *, int, int *);
template int launch_check_finite<double>(sev_ctx *, int, const double *, int, int *);
template int launch_band_from_dense<float>(sev_ctx *, int, const float *, int, int, float *, int);
template int launch_band_from_dense<double>(sev_ctx *, int, const double *, int, int, double *, int);
template int launch_tridiag_extract<float>(sev_ctx *, int, const float *, int, double *, double *);
template int launch_tridiag_extract<double>(sev_ctx *, int, const double *, int, double *, double *);

// ----------------------------------------------------------------- bisection
// par[0] = gl, par[1] = gu (scaled, widened Gershgorin interval), par[2] = sc
// = 2^-s, par[3] = tnorm (scaled max |end| of the unwidened interval),
// par[4] = 2^s, par[5] = 1 if T = 0 (a zero Gershgorin bound), par[6] = 1 if
// the caller's skip flag was set (non-finite input: no bisection, NaN
// eigenvalues).  e2s[i] = (e_i 2^-s)^2.
__device__ __forceinline__ double pow2_exact(int k) {  // 2^k, -1022 <= k <= 1023
    return __longlong_as_double((long long)(1023 + k) << 52);
}

__global__ void bisect_prep_kernel(int n, const double *__restrict__ d, const double *__restrict__ e,
                                   double *__restrict__ e2s, double *__restrict__ par, const int *skip) {
    __shared__ double red[32];
    __shared__ double s_sc;
    double lo = INFINITY, hi = -INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double r = 0.0;
        if (i > 0) r = __dadd_rn(r, fabs(e[i - 1]));
        if (i + 1 < n) r = __dadd_rn(r, fabs(e[i]));
        lo = fmin(lo, __dsub_rn(d[i], r));
        hi = fmax(hi, __dadd_rn(d[i], r));
    }
    lo = -block_max(-lo, red);
    hi = block_max(hi, red);
    if (threadIdx.x == 0) {
        double tnorm = fmax(fabs(lo), fabs(hi));
        int s = 0;
        if (tnorm > 0.0) (void)frexp(tnorm, &s);  // tnorm = m 2^s, m in [0.5, 1)
        const double sc = pow2_exact(-s);
        lo = __dmul_rn(lo, sc);
        hi = __dmul_rn(hi, sc);
        tnorm = __dmul_rn(tnorm, sc);
        const double pad = __dadd_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, (double)n), DBL_EPSILON), tnorm), 0x1p-1000);
        par[0] = __dsub_rn(lo, pad);
        par[1] = __dadd_rn(hi, pad);
        par[2] = sc;
        par[3] = tnorm;
        par[4] = pow2_exact(s);
        par[5] = tnorm == 0.0 ? 1.0 : 0.0;
        par[6] = (skip && *skip) ? 1.0 : 0.0;
        s_sc = sc;
    }
    __syncthreads();
    const double sc = s_sc;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (i + 1 < n) {
            const double es = __dmul_rn(e[i], sc);
            e2s[i] = __dmul_rn(es, es);
        } else {
            e2s[i] = 0.0;
        }
    }
}

// One step of the minors recurrence with t = d_i sc - x: u = e_{i-1}^2 a,
// p = t b - u; sign, zero test and exponent from the bits (integer work, so
// the FP64 pipe sees only the three operations), rescaling by a power of two
// when |p| leaves [2^-256, 2^256].
__device__ __forceinline__ void sturm_step(double di, double e2i, double x, double sc, double &a, double &b,
                                           bool &neg, int &c) {
    const double t = __fma_rn(di, sc, -x);
    const double u = __dmul_rn(e2i, a);
    const double p = __fma_rn(t, b, -u);
    const long long pb = __double_as_longlong(p);
    const bool zero = (pb << 1) == 0;
    const bool pn = zero ? !neg : pb < 0;
    c += pn != neg;
    neg = pn;
    a = b;
    b = p;
    const int ex = (int)((pb >> 52) & 0x7FF);
    if (__builtin_expect(ex > 1023 + 256 || (ex < 1023 - 256 && !zero), 0)) {
        int k = 1023 - ex;
        k = k > 512 ? 512 : (k < -512 ? -512 : k);
        const double f = pow2_exact(k);
        a = __dmul_rn(a, f);
        b = __dmul_rn(b, f);
    }
}

// The loads of d and e^2 do not depend on the recurrence, so blocks of kSturmU
// steps are loaded one block ahead (the chain waits on the FP64 pipe, not on
// a memory latency per step); the operations and their order are those of
// the plain loop.
constexpr int kSturmU = 4;
__device__ __forceinline__ int sturm_count(int n, const double *__restrict__ d, const double *__restrict__ e2s,
                                           double x, double sc) {
    double a = 1.0, b = __fma_rn(__ldg(d), sc, -x);
    bool neg = b <= 0.0;  // p_0 = 1 > 0: a zero p_1 counts as negative
    int c = neg;
    double dn[kSturmU], en[kSturmU];
#pragma unroll
    for (int u = 0; u < kSturmU; ++u) {
        const int i = 1 + u;
        dn[u] = i < n ? __ldg(d + i) : 0.0;
        en[u] = i < n ? __ldg(e2s + i - 1) : 0.0;
    }
    for (int i0 = 1; i0 < n; i0 += kSturmU) {
        double dc[kSturmU], ec[kSturmU];
#pragma unroll
        for (int u = 0; u < kSturmU; ++u) {
            dc[u] = dn[u];
            ec[u] = en[u];
            const int i = i0 + kSturmU + u;
            dn[u] = i < n ? __ldg(d + i) : 0.0;
            en[u] = i < n ? __ldg(e2s + i - 1) : 0.0;
        }
        if (i0 + kSturmU <= n) {
#pragma unroll
            for (int u = 0; u < kSturmU; ++u) sturm_step(dc[u], ec[u], x, sc, a, b, neg, c);
        } else {
#pragma unroll
            for (int u = 0; u < kSturmU; ++u)
                if (i0 + u < n) sturm_step(dc[u], ec[u], x, sc, a, b, neg, c);
        }
    }
    return c;
}

// One thread per eigenvalue index k (the (k+1)-th smallest).
__global__ void bisect_kernel(int n, const double *__restrict__ d, const double *__restrict__ e2s,
                              const double *__restrict__ par, double rtol, int maxit, double *__restrict__ eigs,
                              int *err) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (n == 1) {
        eigs[0] = d[0];
        return;
    }
    if (par[5] != 0.0) {
        eigs[k] = 0.0;
        return;
    }
    const double sc = par[2];
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
        if (sturm_count(n, d, e2s, mid, sc) >= k + 1)
            hi = mid;
        else
            lo = mid;
        ++it;
    }
    eigs[k] = __dmul_rn(__dmul_rn(0.5, __dadd_rn(lo, hi)), par[4]);
}

// ------------------------------------------------- shared-interval rounds
// The per-eigenvalue bisection above visits, for index k, the path of
// intervals that the counts at its midpoints dictate.  Indices whose
// intervals coincide take identical steps (same midpoint, same count, same
// stopping test), and by monotonicity of the count they form contiguous
// runs of k.  bisect_rounds_kernel exploits both facts without changing a
// single rounding: every round (1) lists the distinct active intervals
// (leaders), (2) evaluates, for each leader, the counts at all midpoints of
// its subtree of depth d -- the midpoints its next d bisection steps can
// reach, computed by the same IEEE operations -- with d as deep as the
// thread budget allows, and (3) lets every index walk d steps down its
// leader's subtree using those counts.  The result is bitwise the one of
// bisect_kernel; the chain of dependent Sturm counts per index shrinks from
// one per level to one per round (the early levels, where few intervals are
// distinct, are resolved many at a time).
//
// The kernel is persistent and cooperative (all CTAs resident); the three
// phases of a round are separated by a grid barrier with a capped wait.
struct BisCtl {
    int bar;    // monotone arrival counter of the grid barrier
    int D;      // leaders this round
    int depth;  // subtree depth this round
    int done;   // no active index left
    int abort;  // a wait hit its cap
    int rounds;       // rounds run (diagnostics)
    long long items;  // subtree midpoints evaluated (diagnostics)
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier number `seq` (1, 2, ...): returns false if the wait hit its cap
// or another CTA gave up.
__device__ bool bis_barrier(BisCtl *ctl, int seq, int *err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&ctl->bar, 1);
        const int target = seq * (int)gridDim.x;
        const long long t0 = clock64();
        int ok = 1;
        while (ld_acquire_gpu(&ctl->bar) < target) {
            if (*(volatile int *)&ctl->abort) {
                ok = 0;
                break;
            }
            if (wait_expired(t0, err)) {
                latch_error(err, SEV_ERR_TIMEOUT);
                *(volatile int *)&ctl->abort = 1;
                ok = 0;
                break;
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The stopping test of one bisection step on [lo, hi] (same operations and
// order as bisect_kernel).  Returns 0 to continue with mid, 1 when converged
// or mid no longer splits, 2 when the step cap is reached.
__device__ __forceinline__ int bis_step_test(double lo, double hi, int it, double rtol, double atol, int maxit,
                                             double &mid) {
    const double w = __dsub_rn(hi, lo);
    const double mag = fmax(fabs(lo), fabs(hi));
    double tol = __dmul_rn(rtol, mag);
    if (atol > tol) tol = atol;
    if (w <= tol) return 1;
    if (it >= maxit) return 2;
    mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
    if (mid <= lo || mid >= hi) return 1;
    return 0;
}

__device__ __forceinline__ int sturm_chain(int n, const double *__restrict__ d, const double *__restrict__ e2s, double x,
                                        double sc) {
    return sturm_count(n, d, e2s, x, sc);
}

struct BisWs {
    double *lo, *hi;
    int *it, *st;        // steps taken; state: 0 active, 1 finished
    int *lead, *leadof;  // leader list; leader slot of each index
    int *cnt;            // counts of the round's subtree midpoints
    BisCtl *ctl;
};

#ifndef SEV_BIS_CHAINS_PER_SM
#define SEV_BIS_CHAINS_PER_SM 128
#endif
constexpr int kBisThreads = 1024;
constexpr int kBisMaxItems = 131072;

__global__ void __launch_bounds__(kBisThreads) bisect_rounds_kernel(int n, const double *__restrict__ d,
                                                                    const double *__restrict__ e2,
                                                                    const double *__restrict__ par, double rtol,
                                                                    int maxit, int budget, double *__restrict__ eigs,
                                                                    BisWs W, int *err) {
    __shared__ int s_scan[kBisThreads];
    const double sc = par[2];
    const double atol = __dmul_rn(rtol, par[3]);
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gthreads = gridDim.x * blockDim.x;
    if (par[6] != 0.0) {  // non-finite input (every CTA reads the same flag: no barrier is entered)
        for (int k = gtid; k < n; k += gthreads) eigs[k] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    const int zero = par[5] != 0.0;  // T = 0: every eigenvalue is exactly 0 (lo = hi = 0, finished)
    for (int k = gtid; k < n; k += gthreads) {
        W.lo[k] = zero ? 0.0 : par[0];
        W.hi[k] = zero ? 0.0 : par[1];
        W.it[k] = 0;
        W.st[k] = zero;
    }
    int seq = 0;
    if (!bis_barrier(W.ctl, ++seq, err)) return;
    for (;;) {
        // ---- (1) leaders: CTA 0 compacts the distinct active intervals
        if (blockIdx.x == 0) {
            const int chunk = (n + kBisThreads - 1) / kBisThreads;
            const int k0 = threadIdx.x * chunk, k1 = min(n, k0 + chunk);
            int mine = 0;
            for (int k = k0; k < k1; ++k)
                if (W.st[k] == 0 && (k == 0 || W.st[k - 1] != 0 || W.lo[k] != W.lo[k - 1] || W.hi[k] != W.hi[k - 1]))
                    ++mine;
            s_scan[threadIdx.x] = mine;
            __syncthreads();
            for (int off = 1; off < kBisThreads; off <<= 1) {  // inclusive scan
                const int v = threadIdx.x >= off ? s_scan[threadIdx.x - off] : 0;
                __syncthreads();
                s_scan[threadIdx.x] += v;
                __syncthreads();
            }
            int pos = s_scan[threadIdx.x] - mine;  // leaders before this chunk
            for (int k = k0; k < k1; ++k) {
                if (W.st[k] != 0) continue;
                if (k == 0 || W.st[k - 1] != 0 || W.lo[k] != W.lo[k - 1] || W.hi[k] != W.hi[k - 1]) W.lead[pos++] = k;
                W.leadof[k] = pos - 1;
            }
            if (threadIdx.x == kBisThreads - 1) {
                // depth: fewest rounds per level, counting a round as one
                // chain latency while its items fit the budget of chains the
                // GPU keeps in flight, and proportionally longer beyond it
                const int D = s_scan[kBisThreads - 1];
                const long cap = n > kBisMaxItems ? n : kBisMaxItems;
                int dep = 1;
                double best = 2.0;
                for (int t = 1; t <= 24; ++t) {
                    const long items = (long)D * ((1L << t) - 1);
                    if (items > cap) break;
                    const double cost = fmax(1.0, (double)items / (double)budget) / t;
                    if (cost < best) {
                        best = cost;
                        dep = t;
                    }
                }
                W.ctl->D = D;
                W.ctl->depth = dep;
                W.ctl->done = D == 0;
                if (D > 0) {
                    W.ctl->rounds += 1;
                    W.ctl->items += (long long)D * ((1L << dep) - 1);
                }
            }
        }
        if (!bis_barrier(W.ctl, ++seq, err)) return;
        if (*(volatile int *)&W.ctl->done) break;
        const int D = *(volatile int *)&W.ctl->D;
        const int dep = *(volatile int *)&W.ctl->depth;
        const int M = (1 << dep) - 1;
        // ---- (2) counts at every midpoint of every leader's subtree
        const long items = (long)D * M;
        // items are dealt round-robin over the CTAs so every SM gets its share
        for (long w = blockIdx.x + (long)threadIdx.x * gridDim.x; w < items; w += gthreads) {
            const int j = (int)(w / M), m = (int)(w % M);
            const int k = W.lead[j];
            double lo = W.lo[k], hi = W.hi[k], mid = 0.0;
            int it = W.it[k];
            // node m in heap order: its depth is floor(log2(m + 1)); the bits of
            // m + 1 below the leading one, top first, are the turns (1 = right)
            const int path = m + 1;
            const int lev = 31 - __clz(path);
            bool live = true;
            for (int l = lev - 1; l >= 0 && live; --l) {
                if (bis_step_test(lo, hi, it, rtol, atol, maxit, mid) != 0) {
                    live = false;
                    break;
                }
                if ((path >> l) & 1)
                    lo = mid;
                else
                    hi = mid;
                ++it;
            }
            int c = -1;
            if (live && bis_step_test(lo, hi, it, rtol, atol, maxit, mid) == 0) c = sturm_chain(n, d, e2, mid, sc);
            W.cnt[w] = c;
        }
        if (!bis_barrier(W.ctl, ++seq, err)) return;
        // ---- (3) every active index walks dep steps down its leader's subtree
        for (int k = gtid; k < n; k += gthreads) {
            if (W.st[k] != 0) continue;
            const int j = W.leadof[k];
            double lo = W.lo[k], hi = W.hi[k], mid = 0.0;
            int it = W.it[k], node = 0, state = 0;
            for (int l = 0; l < dep; ++l) {
                const int r = bis_step_test(lo, hi, it, rtol, atol, maxit, mid);
                if (r != 0) {
                    state = r;
                    break;
                }
                if (W.cnt[(long)j * M + node] >= k + 1) {
                    hi = mid;
                    node = 2 * node + 1;
                } else {
                    lo = mid;
                    node = 2 * node + 2;
                }
                ++it;
            }
            if (state == 0) state = bis_step_test(lo, hi, it, rtol, atol, maxit, mid);
            if (state == 2) latch_error(err, SEV_ERR_NOCONV);
            W.lo[k] = lo;
            W.hi[k] = hi;
            W.it[k] = it;
            W.st[k] = state != 0;
        }
        if (!bis_barrier(W.ctl, ++seq, err)) return;
    }
    const double up = par[4];
    for (int k = gtid; k < n; k += gthreads) eigs[k] = __dmul_rn(__dmul_rn(0.5, __dadd_rn(W.lo[k], W.hi[k])), up);
}

size_t bisect_workspace(int n) {
    Carver c(nullptr);
    c.take<double>((size_t)n + 1);
    c.take<double>(8);
    c.take<double>((size_t)n);
    c.take<double>((size_t)n);
    for (int a = 0; a < 4; ++a) c.take<int>((size_t)n);
    c.take<int>((size_t)(n > kBisMaxItems ? n : kBisMaxItems));
    c.take<BisCtl>(1);
    return c.bytes();
}

int launch_bisect(sev_ctx *h, int n, const double *d, const double *e, double rtol, double *eigs, void *ws,
                  size_t ws_bytes, const int *skip) {
    if (n <= 0) return SEV_OK;
    if (ws_bytes < bisect_workspace(n)) return SEV_ERR_WORKSPACE;
    Carver c(ws);
    double *e2 = c.take<double>((size_t)n + 1);
    double *par = c.take<double>(8);
    BisWs W;
    W.lo = c.take<double>((size_t)n);
    W.hi = c.take<double>((size_t)n);
    W.it = c.take<int>((size_t)n);
    W.st = c.take<int>((size_t)n);
    W.lead = c.take<int>((size_t)n);
    W.leadof = c.take<int>((size_t)n);
    W.cnt = c.take<int>((size_t)(n > kBisMaxItems ? n : kBisMaxItems));
    W.ctl = c.take<BisCtl>(1);
    SEV_LAUNCH(h, K_BISECT_PREP, bisect_prep_kernel, 1, 1024, 0, n, d, e, e2, par, skip);
    if (n == 1) {
        SEV_CUDA(cudaMemcpyAsync(eigs, d, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        return SEV_OK;
    }
    SEV_CUDA(cudaMemsetAsync(W.ctl, 0, sizeof(BisCtl), h->stream));
    // one CTA per SM: enough Sturm chains in flight to cover the FP64 divide
    // latency, and every CTA resident for the grid barrier
    int per_sm = 0;
    SEV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bisect_rounds_kernel, kBisThreads, 0));
    if (per_sm < 1) return SEV_ERR_UNSUPPORTED;
    // A Sturm step is three FP64 instructions on its dependence chain.  The
    // budget of chains per round (128 per SM) is the measured best at
    // n = 16384 since the Sturm loop loads ahead (64: 63.0 ms, 128: 58.5,
    // 256: 58.3 on a random tridiagonal); 1024 threads per CTA run a round
    // of up to 150K chains in a single pass.
    const int grid = h->sm_count;
    int budget = grid * SEV_BIS_CHAINS_PER_SM;
    int maxit = 200;
    void *args[] = {(void *)&n, (void *)&d, (void *)&e2, (void *)&par, (void *)&rtol, (void *)&maxit,
                    (void *)&budget, (void *)&eigs, (void *)&W, (void *)&h->d_err};
    timing_begin(h, K_BISECT);
    SEV_CUDA(cudaLaunchCooperativeKernel((const void *)bisect_rounds_kernel, grid, kBisThreads, args, 0, h->stream));
    timing_end(h, K_BISECT);
    return SEV_OK;
}

}  // namespace sev

// ------------------------------------------------- allocation-free variant
// sev_tridiag_bisect_static runs bisect_prep_kernel (the kernel
// sev_tridiag_bisect also starts with) and then bisect_kernel, one thread per
// eigenvalue index.  The handle path runs the cooperative bisect_rounds_kernel
// instead; for every index that kernel takes the same IEEE operations in the
// same order as bisect_kernel (the shared-interval rounds only change which
// thread evaluates a count, never its value), so both give the same bits.
// The scratch -- the squared scaled off-diagonal, the scaling and Gershgorin
// parameters and the status word -- lives in this file-scope device array
// instead of handle workspace, so a call allocates nothing.  The array is
// (kStaticMaxN + 16) doubles (~512 KiB) on every device that loads the
// library, held until the process exits.
namespace sev {
constexpr int kStaticMaxN = 65536;
constexpr int kStaticPar = kStaticMaxN + 1;     // 8 doubles of bisection parameters
constexpr int kStaticStatus = kStaticMaxN + 9;  // status word (a DevStatus-sized slot)
static __device__ __align__(256) double g_bisect_scratch[kStaticMaxN + 16];

// The array's device address and the SM count, per device ordinal.  They are
// looked up again by every call made outside stream capture (so a
// cudaDeviceReset, which reloads the module at a new address, is picked up)
// and published atomically (concurrent first calls from several host
// threads store the same values).
struct StaticScratch {
    std::atomic<double *> ptr{nullptr};
    std::atomic<int> sm_count{0};
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
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SEV_ERR_CUDA;
    StaticScratch &S = g_static_dev[dev];
    double *ptr = S.ptr.load(std::memory_order_acquire);
    if (cap == cudaStreamCaptureStatusNone || !ptr) {
        // with the device current: the array's device address (in host code
        // the array's name is only a stand-in for it)
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bisect_scratch) != cudaSuccess) return SEV_ERR_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SEV_ERR_CUDA;
        S.sm_count.store(sms, std::memory_order_relaxed);
        ptr = (double *)p;
        S.ptr.store(ptr, std::memory_order_release);
    }
    const int sm_count = S.sm_count.load(std::memory_order_relaxed);
    double *e2 = ptr;                  // n + 1 doubles
    double *par = ptr + kStaticPar;    // 8 doubles
    int *status = (int *)(ptr + kStaticStatus);
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return SEV_ERR_CUDA;
    bisect_prep_kernel<<<1, 1024, 0, st>>>(n, d, n > 1 ? e : d, e2, par, nullptr);
    if (cudaGetLastError() != cudaSuccess) return SEV_ERR_CUDA;
    int bs = 64;
    while (bs > 32 && (n + bs - 1) / bs < sm_count) bs >>= 1;
    bisect_kernel<<<(n + bs - 1) / bs, bs, 0, st>>>(n, d, e2, par, rtol, 200, eigs, status);
    return cudaGetLastError() == cudaSuccess ? SEV_OK : SEV_ERR_CUDA;
}
