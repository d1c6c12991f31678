// batched.cu -- eigenvalues of many independent small symmetric matrices in
// one persistent launch.  The paper treats one matrix; batching is this
// library's addition for workloads of many small uneven matrices (a
// sequence of SCF-style eigenproblems).  Each matrix runs the paper's path
// unchanged, inside one CTA:
//
//   full-to-band (Algorithm 4.1) -- per panel the Householder QR of the
//     N x b panel (the tree of Algorithm 3.2 with a single leaf: the panel
//     fits in shared memory), the compact-WY factor T (Cor. 3.7's form
//     Q = I - U T U^T) and the two-sided update A22 += U V^T + V U^T with
//     V = U (T^T U^T A22 U T) / 2 - A22 U T (Eq. 4.1);
//   b -> 1 band reduction (Algorithm 4.2 with h = 1) on the whole band held
//     in shared memory: every warp owns one sweep at a time, and chase
//     (i, j) starts once sweep i - 1 has finished chase j + 2 (the legal
//     dependency of the wavefront, Sec. 4.2);
//   Sturm bisection of the tridiagonal (the final step of Algorithm 4.3).
//
// CTAs take matrices from a global queue (the host orders it largest
// first), so the launch load-balances uneven sizes by itself.  The matrix
// is overwritten (both triangles: the kernel first mirrors the lower
// triangle).  Nothing is allocated and nothing waits on the host, so the
// launch can be captured in a CUDA graph.
#include "tri_chase.cuh"

namespace sev {

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kDone = 2047;  // chase counter value of a finished sweep

struct BatchMat {
    void *A;
    double *eigs;
    int n;
    int lda;
};

template <typename T, int B>
struct BatchLayout {
    // full-to-band: U, Y (ldp x B each), Tm, G, Z (B x B), tau (B), red
    static __host__ __device__ size_t f_bytes(int ldp) {
        return sizeof(T) * (2 * (size_t)ldp * B + 3 * (size_t)B * B + B) + 64;
    }
    // band: nmax columns x 2B diagonals, per-warp vector buffers, counters
    static __host__ __device__ size_t b_bytes(int nmax) {
        return sizeof(T) * ((size_t)nmax * 2 * B + 2 * kBatchWarps * 32) + kBatchWarps * sizeof(int);
    }
    static __host__ __device__ size_t e_off(int nmax) {
        const size_t f = f_bytes(nmax), b = b_bytes(nmax);
        return ((f > b ? f : b) + 15) & ~(size_t)15;
    }
    // bisection: d, e, e^2 (n doubles each), parameters, reduction scratch
    static __host__ __device__ size_t bytes(int nmax) { return e_off(nmax) + sizeof(double) * (3 * (size_t)nmax + 48); }
};

// ------------------------------------------------------------ full to band
template <typename T, int B>
__device__ void batch_full_to_band(T *A, int n, int lda, unsigned char *smem, int ldp) {
    const int tid = threadIdx.x, nt = blockDim.x;
    T *U = (T *)smem;
    T *Y = U + (size_t)ldp * B;
    T *Tm = Y + (size_t)ldp * B;
    T *G = Tm + B * B;
    T *Z = G + B * B;
    T *tau = Z + B * B;
    for (int c0 = 0; c0 + B < n; c0 += B) {
        const int r0 = c0 + B, N = n - r0;
        if (N < 2) break;
        T *A22 = A + r0 + (size_t)r0 * lda;
        batched_copy<T>(
            N * B, tid, nt, [&](int k) { return A[(r0 + k % N) + (size_t)(c0 + k / N) * lda]; },
            [&](int k, T v) { U[k % N + (size_t)(k / N) * ldp] = v; });
        __syncthreads();
        const int r = cta_qr(N, B, U, ldp, tau, nullptr);
        // the band block: R's upper triangle (rows r0.., columns c0..)
        for (int idx = tid; idx < B * B; idx += nt) {
            const int i = idx % B, j = idx / B;
            if (i <= j && i < N) A[(r0 + i) + (size_t)(c0 + j) * lda] = U[i + (size_t)j * ldp];
        }
        cta_form_t(N, r, U, ldp, tau, Tm, B, G, B);
        // explicit U (unit lower trapezoidal, zero columns r..B-1), T padded with zeros
        for (int idx = tid; idx < N * B; idx += nt) {
            const int i = idx % N, c = idx / N;
            const T v = U[i + (size_t)c * ldp];
            U[i + (size_t)c * ldp] = (c < r) ? (i < c ? T(0) : (i == c ? T(1) : v)) : T(0);
        }
        for (int idx = tid; idx < B * B; idx += nt) {
            const int a = idx % B, c = idx / B;
            if (a >= r || c >= r) Tm[idx] = T(0);
        }
        __syncthreads();
        // Y = A22 U;  G = U^T Y;  Z = G T;  G = T^T Z  (= T^T U^T A22 U T)
        cta_gemm<T, false, false>(N, B, N, T(1), A22, lda, U, ldp, T(0), Y, ldp);
        __syncthreads();
        cta_gemm<T, true, false>(B, B, N, T(1), U, ldp, Y, ldp, T(0), G, B);
        __syncthreads();
        cta_gemm<T, false, false>(B, B, B, T(1), G, B, Tm, B, T(0), Z, B);
        __syncthreads();
        cta_gemm<T, true, false>(B, B, B, T(1), Tm, B, Z, B, T(0), G, B);
        __syncthreads();
        // V = U G / 2 - Y T, row by row in place of Y
        for (int i = tid; i < N; i += nt) {
            T y[B], u[B];
#pragma unroll
            for (int q = 0; q < B; ++q) {
                y[q] = Y[i + (size_t)q * ldp];
                u[q] = U[i + (size_t)q * ldp];
            }
#pragma unroll 4
            for (int c = 0; c < B; ++c) {
                T acc = 0;
#pragma unroll
                for (int k = 0; k < B; ++k) acc = fma(T(0.5) * u[k], G[k + c * B], fma(-y[k], Tm[k + c * B], acc));
                Y[i + (size_t)c * ldp] = acc;
            }
        }
        __syncthreads();
        // A22 += U V^T + V U^T (both triangles: the next panel's product reads all of A22)
        cta_gemm<T, false, true>(N, N, B, T(1), U, ldp, Y, ldp, T(1), A22, lda);
        cta_gemm<T, false, true>(N, N, B, T(1), Y, ldp, U, ldp, T(1), A22, lda);
        __syncthreads();
    }
}

// ------------------------------------------------------------- band to 1
// Returns false if a wait hit its cap.
template <typename T, int B>
__device__ bool batch_band_to_tri(const T *A, int n, int lda, unsigned char *smem, int *err) {
    constexpr int LDW = 2 * B;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    T *band = (T *)smem;
    T *vb = band + (size_t)n * LDW;
    T *wb = vb + kBatchWarps * 32;
    volatile int *sval = (volatile int *)(wb + kBatchWarps * 32);
    __shared__ int s_fail;
    for (int idx = tid; idx < n * LDW; idx += nt) {
        const int c = idx / LDW, d = idx % LDW;
        band[idx] = (d <= B && c + d < n) ? A[(c + d) + (size_t)c * lda] : T(0);
    }
    if (tid < kBatchWarps) sval[tid] = 0;
    if (tid == 0) s_fail = 0;
    __syncthreads();
    TriWin<T, B> W;
    W.w = band;
    W.wcap = n;  // the whole band: slots never wrap
    const int nsweeps = n >= 3 ? n - 2 : 0;
    for (int i = 1 + warp; i <= nsweeps; i += kBatchWarps) {
        const int Ji = tri_chases(n, B, i);
        const int Jp = i > 1 ? tri_chases(n, B, i - 1) : 0;
        T rv = T(0), rtau = T(0), rbeta = T(0);
        for (int j = 1; j <= Ji; ++j) {
            if (i > 1) {
                const int need = (i - 1) * 2048 + (j + 2 <= Jp ? j + 2 : kDone);
                int ok = 1;
                if (lane == 0) {
                    const long long t0 = clock64();
                    while (sval[(i - 2) % kBatchWarps] < need) {
                        if (*(volatile int *)&s_fail || wait_expired(t0, err)) {
                            ok = 0;
                            break;
                        }
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) {
                        latch_error(err, SEV_ERR_TIMEOUT);
                        s_fail = 1;
                    }
                    i = nsweeps + 1;  // leave both loops
                    break;
                }
                __threadfence_block();
            }
            const int o = i + (j - 1) * B;
            if (j == 1) {
                // the sweep's first reflector: column i - 1, rows [i, i + n_r)
                const int nr1 = min(n - o, B);
                T *xcol = band + (size_t)(o - 1) * LDW + 1;
                const T x = lane < nr1 ? xcol[lane] : T(0);
                tri_reflector<T, B>(x, nr1, rv, rtau, rbeta);
                if (lane < nr1) xcol[lane] = lane == 0 ? rbeta : T(0);
                __syncwarp();
            }
            if (j > 1 && j < Ji && o + 3 * B <= n)
                tri_chase_body<T, B, true>(n, o, j, true, W, vb + warp * 32, wb + warp * 32, rv, rtau, rbeta);
            else
                tri_chase_body<T, B>(n, o, j, j < Ji, W, vb + warp * 32, wb + warp * 32, rv, rtau, rbeta);
            __threadfence_block();
            __syncwarp();
            if (lane == 0) sval[(i - 1) % kBatchWarps] = i * 2048 + (j == Ji ? kDone : j);
        }
    }
    __syncthreads();
    return s_fail == 0;
}

// -------------------------------------------------------------- bisection
// The same scaling, minors count, stopping rule and IEEE operations as
// bisect.cu, on shared-memory d and (e 2^-s)^2.
__device__ __forceinline__ double batch_pow2(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

__device__ __forceinline__ int batch_sturm(int n, const double *d, const double *e2s, double x, double sc) {
    double a = 1.0, b = __fma_rn(d[0], sc, -x);
    bool neg = b <= 0.0;
    int c = neg;
    for (int i = 1; i < n; ++i) {
        const double t = __fma_rn(d[i], sc, -x);
        const double u = __dmul_rn(e2s[i - 1], a);
        const double p = __fma_rn(t, b, -u);
        // sign, zero test and exponent from the bits: integer work, so the
        // FP64 pipe sees only the three operations above
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
            const double f = batch_pow2(k);
            a = __dmul_rn(a, f);
            b = __dmul_rn(b, f);
        }
    }
    return c;
}

template <typename T, int B>
__device__ void batch_bisect(int n, int nmax, unsigned char *smem, double rtol, double *eigs, int *err) {
    constexpr int LDW = 2 * B;
    const int tid = threadIdx.x, nt = blockDim.x;
    const T *band = (const T *)smem;
    double *d = (double *)(smem + BatchLayout<T, B>::e_off(nmax));
    double *e = d + nmax;
    double *e2s = e + nmax;
    double *par = e2s + nmax;  // gl, gu, sc, tnorm, 2^s, zero
    double *red = par + 8;     // 32
    for (int i = tid; i < n; i += nt) {
        d[i] = (double)band[(size_t)i * LDW];
        e[i] = i + 1 < n ? (double)band[(size_t)i * LDW + 1] : 0.0;
    }
    __syncthreads();
    double lo = INFINITY, hi = -INFINITY;
    for (int i = tid; i < n; i += nt) {
        double r = 0.0;
        if (i > 0) r = __dadd_rn(r, fabs(e[i - 1]));
        if (i + 1 < n) r = __dadd_rn(r, fabs(e[i]));
        lo = fmin(lo, __dsub_rn(d[i], r));
        hi = fmax(hi, __dadd_rn(d[i], r));
    }
    lo = -block_max(-lo, red);
    hi = block_max(hi, red);
    if (tid == 0) {
        double tnorm = fmax(fabs(lo), fabs(hi));
        if (!isfinite(tnorm)) latch_error(err, SEV_ERR_NONFINITE);
        int s = 0;
        if (tnorm > 0.0 && isfinite(tnorm)) (void)frexp(tnorm, &s);
        const double sc = batch_pow2(-s);
        lo = __dmul_rn(lo, sc);
        hi = __dmul_rn(hi, sc);
        tnorm = __dmul_rn(tnorm, sc);
        const double pad = __dadd_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, (double)n), DBL_EPSILON), tnorm), 0x1p-1000);
        par[0] = __dsub_rn(lo, pad);
        par[1] = __dadd_rn(hi, pad);
        par[2] = sc;
        par[3] = tnorm;
        par[4] = batch_pow2(s);
        par[5] = tnorm == 0.0 ? 1.0 : 0.0;
    }
    __syncthreads();
    const double sc = par[2];
    for (int i = tid; i < n; i += nt) {
        if (i + 1 < n) {
            const double es = __dmul_rn(e[i], sc);
            e2s[i] = __dmul_rn(es, es);
        } else {
            e2s[i] = 0.0;
        }
    }
    __syncthreads();
    const double atol = __dmul_rn(rtol, par[3]);
    const bool zero = par[5] != 0.0;
    for (int k = tid; k < n; k += nt) {
        double a = par[0], b = par[1];
        int it = 0;
        for (; !zero;) {
            const double w = __dsub_rn(b, a);
            const double mag = fmax(fabs(a), fabs(b));
            double tol = __dmul_rn(rtol, mag);
            if (atol > tol) tol = atol;
            if (w <= tol) break;
            if (it >= 200) {
                latch_error(err, SEV_ERR_NOCONV);
                break;
            }
            const double mid = __dmul_rn(0.5, __dadd_rn(a, b));
            if (mid <= a || mid >= b) break;
            if (batch_sturm(n, d, e2s, mid, sc) >= k + 1)
                b = mid;
            else
                a = mid;
            ++it;
        }
        eigs[k] = zero ? 0.0 : __dmul_rn(__dmul_rn(0.5, __dadd_rn(a, b)), par[4]);
    }
    __syncthreads();
}

// ----------------------------------------------------------------- kernel
template <typename T, int B>
__global__ void __launch_bounds__(kBatchThreads) batch_eig_kernel(int count, const BatchMat *__restrict__ mats,
                                                                   int *queue, int nmax, double rtol, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_idx;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_idx = atomicAdd(queue, 1);
        __syncthreads();
        const int q = s_idx;
        if (q >= count) return;
        const BatchMat m = mats[q];
        T *A = (T *)m.A;
        const int n = m.n, lda = m.lda;
        if (n <= 0) continue;
        if (n == 1) {
            if (threadIdx.x == 0) m.eigs[0] = (double)A[0];
            continue;
        }
        // mirror the lower triangle: the panel products read all of A22
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
            const int i = idx % n, j = idx / n;
            if (i < j) A[i + (size_t)j * lda] = A[j + (size_t)i * lda];
        }
        __syncthreads();
        batch_full_to_band<T, B>(A, n, lda, smem, nmax);
        if (!batch_band_to_tri<T, B>(A, n, lda, smem, err)) return;
        batch_bisect<T, B>(n, nmax, smem, rtol, m.eigs, err);
    }
}

int batch_supported(int b, int elem) { return b == 4 || b == 8 || b == 16 || (b == 32 && elem == 4); }

template <typename T>
size_t batch_smem_bytes(int b, int nmax) {
    switch (b) {
        case 4: return BatchLayout<T, 4>::bytes(nmax);
        case 8: return BatchLayout<T, 8>::bytes(nmax);
        case 16: return BatchLayout<T, 16>::bytes(nmax);
        case 32: return BatchLayout<T, 32>::bytes(nmax);
        default: return 0;
    }
}

// Host preparation (outside any stream capture): opt in to the kernel's
// dynamic shared memory and size the persistent grid.
template <typename T, int B>
static int prepare_batch_b(sev_ctx *h, int count, int nmax, int *grid) {
    const size_t smem = BatchLayout<T, B>::bytes(nmax);
    if (smem > h->smem_optin) return SEV_ERR_UNSUPPORTED;
    auto kern = batch_eig_kernel<T, B>;
    SEV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SEV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, smem));
    if (per_sm < 1) return SEV_ERR_UNSUPPORTED;
    int g = h->sm_count * per_sm;
    if (g > count) g = count;
    *grid = g;
    return SEV_OK;
}

template <typename T, int B>
static int launch_batch_b(sev_ctx *h, int count, const BatchMat *mats, int *queue, int nmax, double rtol, int grid) {
    const size_t smem = BatchLayout<T, B>::bytes(nmax);
    SEV_CUDA(cudaMemsetAsync(queue, 0, sizeof(int), h->stream));
    auto kern = batch_eig_kernel<T, B>;
    SEV_LAUNCH(h, K_BATCH, kern, grid, kBatchThreads, smem, count, mats, queue, nmax, rtol, h->d_err);
    return SEV_OK;
}

template <typename T>
int prepare_batch_small(sev_ctx *h, int count, int b, int nmax, int *grid) {
    switch (b) {
        case 4: return prepare_batch_b<T, 4>(h, count, nmax, grid);
        case 8: return prepare_batch_b<T, 8>(h, count, nmax, grid);
        case 16: return prepare_batch_b<T, 16>(h, count, nmax, grid);
        case 32:
            if constexpr (sizeof(T) == 4) return prepare_batch_b<T, 32>(h, count, nmax, grid);
            return SEV_ERR_UNSUPPORTED;
        default: return SEV_ERR_UNSUPPORTED;
    }
}

template <typename T>
int launch_batch_small(sev_ctx *h, int count, const void *mats, int *queue, int b, int nmax, double rtol, int grid) {
    if (count <= 0) return SEV_OK;
    const BatchMat *m = (const BatchMat *)mats;
    switch (b) {
        case 4: return launch_batch_b<T, 4>(h, count, m, queue, nmax, rtol, grid);
        case 8: return launch_batch_b<T, 8>(h, count, m, queue, nmax, rtol, grid);
        case 16: return launch_batch_b<T, 16>(h, count, m, queue, nmax, rtol, grid);
        case 32:
            if constexpr (sizeof(T) == 4) return launch_batch_b<T, 32>(h, count, m, queue, nmax, rtol, grid);
            return SEV_ERR_UNSUPPORTED;
        default: return SEV_ERR_UNSUPPORTED;
    }
}

size_t batch_mat_bytes() { return sizeof(BatchMat); }

void batch_pack_mat(void *dst, void *A, double *eigs, int n, int lda) {
    BatchMat m;
    m.A = A;
    m.eigs = eigs;
    m.n = n;
    m.lda = lda;
    *(BatchMat *)dst = m;
}


// ---------------------------------------------------------------- autotune
// Synthetic symmetric matrices for timing candidate band widths: the lower
// triangle gets uniform(-1, 1) entries from a counter-based hash (splitmix64
// of the matrix index and the entry index).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

template <typename T>
__global__ void batch_fill_kernel(int count, const BatchMat *__restrict__ mats, unsigned long long seed) {
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        const BatchMat m = mats[q];
        T *A = (T *)m.A;
        for (int idx = threadIdx.x; idx < m.n * m.n; idx += blockDim.x) {
            const int i = idx % m.n, j = idx / m.n;
            if (i < j) continue;
            const unsigned long long r = splitmix64(seed ^ ((unsigned long long)q << 32) ^ (unsigned long long)idx);
            A[i + (size_t)j * m.lda] = (T)((double)(r >> 11) * 0x1.0p-52 - 1.0);
        }
    }
}

template <typename T>
int launch_batch_fill(sev_ctx *h, int count, const void *mats, unsigned long long seed) {
    if (count <= 0) return SEV_OK;
    SEV_LAUNCH(h, K_MISC, batch_fill_kernel<T>, count < 4096 ? count : 4096, 256, 0, count, (const BatchMat *)mats,
               seed);
    return SEV_OK;
}
template int launch_batch_fill<float>(sev_ctx *, int, const void *, unsigned long long);
template int launch_batch_fill<double>(sev_ctx *, int, const void *, unsigned long long);

template int launch_batch_small<float>(sev_ctx *, int, const void *, int *, int, int, double, int);
template int launch_batch_small<double>(sev_ctx *, int, const void *, int *, int, int, double, int);
template int prepare_batch_small<float>(sev_ctx *, int, int, int, int *);
template int prepare_batch_small<double>(sev_ctx *, int, int, int, int *);
template size_t batch_smem_bytes<float>(int, int);
template size_t batch_smem_bytes<double>(int, int);

}  // namespace sev
