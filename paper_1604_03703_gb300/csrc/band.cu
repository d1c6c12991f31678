// band.cu -- band-to-band reduction b -> h (Algorithm 4.2) on packed lower
// band storage, as one persistent kernel per stage.
//
// Chase (i, j) (1-based, as in the algorithm): with h the target width,
//   o_qr.r = (i-1)h + (j-1)b + h
//   j = 1: o_qr.c = o_qr.r - h, o_v = 0,     o_up.c = o_qr.r,      n_c = min(n - o_up.c, 2b)
//   j > 1: o_qr.c = o_qr.r - b, o_v = b - h, o_up.c = o_qr.c + h,  n_c = min(n - o_up.c, 3b - h)
//   n_r = min(n - o_qr.r, b); the chase exists while n - o_qr.r >= 2
// and performs: QR of B[qr rows, qr cols] (n_r x h); write [R; 0];
// W = B[up cols, qr rows] U T; V = -W; V[v rows] += 1/2 U (T^T (U^T W[v rows]));
// B[qr rows, up cols] += U V^T and the mirrored B[up cols, qr rows] += V U^T.
// With lower storage the mirrored pair is one entry: rows of W outside the
// qr rows get X <- X - (X U T) U^T (one-sided), the qr-row block gets the
// symmetric rank-2 update U V^T + V U^T.
//
// Schedule.  A CTA takes sweeps i in increasing order (global counter) and
// runs its chases j = 1, 2, ... (the grid is capped to the ~J/3 sweeps that
// can progress together); chase (i, j) waits until sweep i-1 has
// completed chase j+2 (or all of its chases).  Chase (i, j) overlaps chase
// (i-1, j+2) -- its bulge rows [o+2b-h, o+2b) are the rows that (i-1, j+2)
// factorises -- so the pipeline t = 2i + j that the Fig. 2 caption pictures
// is not legal; this rule gives t = 3i + j and reproduces the sequential
// order bit for bit.  Sweeps are handed out in order and each CTA finishes
// its sweep before taking another, so every awaited sweep is held by a
// running CTA: the waits cannot deadlock.  Every wait is capped; on expiry
// the kernel latches SEV_ERR_TIMEOUT and returns.
//
// Bands of width 64 or more run each sweep on a cluster of three CTAs
// (band_chase_x3_kernel, below): the QR and the diagonal block on one CTA,
// the rows above and below on the other two, with the same arithmetic per
// entry as the one-CTA chase.
#include "regtile.cuh"

#ifdef SEV_TRACE
static __device__ long long *sev_btrace = nullptr;
extern "C" int sev_trace_set_band(void *p) {
    return cudaMemcpyToSymbol(sev_btrace, &p, sizeof(p)) == cudaSuccess ? 0 : 1;
}
// the register QR's step clocks of CTA 0 (this file's copy of the trace pointer)
extern "C" int sev_trace_set_reg_band(void *p) {
    return cudaMemcpyToSymbol(sev_rtrace, &p, sizeof(p)) == cudaSuccess ? 0 : 1;
}
#define BTRACE(k)                                                              \
    do {                                                                       \
        if (threadIdx.x == 0 && sev_btrace && i == 40 && j == 20) sev_btrace[k] = clock64(); \
    } while (0)
// cluster chase: slot k of rank r at 16 + 16 r (each rank's own SM clock)
#define BTRACE3(k)                                                                            \
    do {                                                                                      \
        if (threadIdx.x == 0 && sev_btrace && i == 40 && j == 20) sev_btrace[16 + 16 * rank + (k)] = clock64(); \
    } while (0)
#else
#define BTRACE(k) \
    do {          \
    } while (0)
#define BTRACE3(k) \
    do {           \
    } while (0)
#endif

namespace sev {

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__host__ __device__ __forceinline__ int band_num_chases(int n, int b, int h, int i) {
    const int r = n - i * h;
    return r < 2 ? 0 : (n - 2 - i * h) / b + 1;
}
__host__ __device__ __forceinline__ int band_num_sweeps(int n, int h) { return n >= 2 ? (n - 2) / h : 0; }

// Band element (r, c) with r >= c; out-of-range indices are a bug: they are
// not dereferenced, the thread's flag `bad` is set and 0 is returned.  The
// flag is a register (OR-ed over the CTA at the end of the kernel): a flag
// in memory would be a store between consecutive loads and keep them from
// being in flight together.
template <typename T>
__device__ __forceinline__ T bld(const T *AB, int ldab, int n, int r, int c, int &bad) {
    const int d = r - c;
    if (d < 0 || d >= ldab || r >= n || c < 0) {
        bad = 1;
        return T(0);
    }
    return __ldcg(AB + d + (size_t)c * ldab);
}
template <typename T>
__device__ __forceinline__ void bst(T *AB, int ldab, int n, int r, int c, T v, int &bad) {
    const int d = r - c;
    if (d < 0 || d >= ldab || r >= n || c < 0) {
        bad = 1;
        return;
    }
    AB[d + (size_t)c * ldab] = v;
}
// Shared memory of one chase: U, U T, the block X being updated, W, T, a
// small product Z, tau, the three reflector buffers of the register QR, a
// reduction scratch and (one-CTA register path) a second block buffer Xb for
// the rows above the qr rows, loaded while the QR runs.
template <typename T>
struct ChaseSmem {
    T *Us, *UTs, *Xs, *Ws, *Ts, *Zs, *Z2s, *tau, *vs, *Xb;
    double *red;
    int ldb1, ldh1;
    __device__ ChaseSmem(unsigned char *base, int b, int h) {
        ldb1 = b + 4;  // a multiple of 4: 16-byte aligned columns for vector loads
        ldh1 = h + 1;
        Us = (T *)base;
        UTs = Us + (size_t)ldb1 * h;
        Xs = UTs + (size_t)ldb1 * h;
        Ws = Xs + (size_t)ldb1 * b;
        Ts = Ws + (size_t)ldb1 * h;
        Zs = Ts + (size_t)ldh1 * h;
        Z2s = Zs + (size_t)ldh1 * h;
        tau = Z2s + (size_t)ldh1 * h;
        vs = tau + h;
        size_t off = (size_t)((unsigned char *)(vs + 3 * 128) - base);
        off = (off + 15) & ~(size_t)15;
        red = (double *)(base + off);
        Xb = (T *)(base + off + 32 * sizeof(double));
    }
};

// Register tile of the chase QR, run by warps 0-3: rows up to 32 R (R = 0:
// the shared-memory cta_qr by the whole CTA), columns up to 4 Q.
__host__ __device__ constexpr int chase_tile_r(int b) { return b <= 32 ? 1 : (b <= 64 ? 2 : (b <= 128 ? 4 : 0)); }
__host__ __device__ constexpr int chase_tile_q(int h) {
    return h <= 4 ? 1 : (h <= 8 ? 2 : (h <= 16 ? 4 : (h <= 32 ? 8 : (h <= 64 ? 16 : 0))));
}

template <typename T>
static size_t band_smem_base(int b, int h) {
    const size_t ldb1 = b + 4, ldh1 = h + 1;
    size_t e = 3 * ldb1 * h + ldb1 * b + 3 * ldh1 * h + h + 3 * 128;
    size_t bytes = e * sizeof(T);
    bytes = (bytes + 15) & ~(size_t)15;
    return bytes + 32 * sizeof(double);
}
// The register path needs the Xb buffer as well.
template <typename T>
static size_t band_smem_reg(int b, int h) {
    return band_smem_base<T>(b, h) + sizeof(T) * (size_t)(b + 4) * b;
}

template <typename T>
size_t band_smem_bytes(int b, int h) {
    return band_smem_base<T>(b, h);
}

// The qr-row diagonal block X_d (n_r x n_r, mirrored in S.Xs) after U, T
// and U T are formed: W_d = X_d (U T); S = U^T W_d; Z = T^T S; V_d = -W_d +
// U Z / 2; X_d += U V_d^T + V_d U^T; the lower triangle written back.
#ifndef SEV_CHASE_PART_INLINE
#define SEV_CHASE_PART_INLINE
#endif
template <typename T>
__device__ SEV_CHASE_PART_INLINE void chase_diag_update(T *AB, int ldab, int n, int n_r, int nr, int o_qr_r,
                                                        ChaseSmem<T> &S, int &bad) {
    const int ldb1 = S.ldb1, ldh1 = S.ldh1;
    const int tid = threadIdx.x, nt = blockDim.x;
    constexpr bool kVec = sizeof(T) == 4;
    cta_mm<T, 4, 4, false, kVec>(n_r, nr, n_r, T(1), S.Xs, ldb1, S.UTs, ldb1, 0, nullptr, 0, nullptr, 0, T(0), S.Ws,
                                 ldb1);
    __syncthreads();
    cta_gemm<T, true, false>(nr, nr, n_r, T(1), S.Us, ldb1, S.Ws, ldb1, T(0), S.Zs, ldh1);
    __syncthreads();
    // Z = T^T S, every entry at once (T upper triangular): Z(a, c) = sum_{q <= a} T(q, a) S(q, c)
    for (int idx = tid; idx < nr * nr; idx += nt) {
        const int a = idx % nr, c = idx / nr;
        T z = 0;
        for (int q = 0; q <= a; ++q) z += S.Ts[q + (size_t)a * ldh1] * S.Zs[q + (size_t)c * ldh1];
        S.Z2s[a + (size_t)c * ldh1] = z;
    }
    __syncthreads();
    cta_mm<T, 4, 4, false, kVec>(n_r, nr, nr, T(0.5), S.Us, ldb1, S.Z2s, ldh1, 0, nullptr, 0, nullptr, 0, T(-1),
                                 S.Ws, ldb1);
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    if (n_r >= 64) {
        // X_d += [U V_d] [V_d U]^T on the tiles on or below the diagonal
        cta_mm<T, 8, 8, true, kVec, true>(n_r, n_r, nr, T(1), S.Us, ldb1, S.Ws, ldb1, nr, S.Ws, ldb1, S.Us, ldb1, T(1),
                                          S.Xs, ldb1);
        __syncthreads();
        // lower triangle, down the columns (band storage: rows of a column contiguous)
        for (int c = warp; c < n_r; c += nw)
            for (int r = c + lane; r < n_r; r += 32)
                bst(AB, ldab, n, o_qr_r + r, o_qr_r + c, S.Xs[r + (size_t)c * ldb1], bad);
    } else {
        for (int c = warp; c < n_r; c += nw)
            for (int r = c + lane; r < n_r; r += 32) {
                T s = 0;
                for (int m = 0; m < nr; ++m)
                    s += S.Us[r + (size_t)m * ldb1] * S.Ws[c + (size_t)m * ldb1] +
                         S.Ws[r + (size_t)m * ldb1] * S.Us[c + (size_t)m * ldb1];
                bst(AB, ldab, n, o_qr_r + r, o_qr_r + c, S.Xs[r + (size_t)c * ldb1] + s, bad);
            }
    }
}

// One chase (i, j) performed by the whole CTA.  RQ, QQ > 0: the n_r x h QR
// runs on a register tile of 32 RQ x 8 QQ (reg_qr); 0: on shared memory.
template <typename T, int RQ, int QQ>
__device__ void band_chase(T *AB, int ldab, int n, int b, int h, int i, int j, ChaseSmem<T> &S, int &bad) {
    const int o_qr_r = (i - 1) * h + (j - 1) * b + h;
    int o_qr_c, o_v, o_up_c, lim;
    if (j == 1) {
        o_qr_c = o_qr_r - h;
        o_v = 0;
        o_up_c = o_qr_r;
        lim = 2 * b;
    } else {
        o_qr_c = o_qr_r - b;
        o_v = b - h;
        o_up_c = o_qr_c + h;
        lim = 3 * b - h;
    }
    const int n_r = min(n - o_qr_r, b);
    const int n_c = min(n - o_up_c, lim);
    const int ldb1 = S.ldb1, ldh1 = S.ldh1;
    const int tid = threadIdx.x, nt = blockDim.x;

    BTRACE(0);
    int nr;
    if constexpr (RQ > 0) {
        const int warp = tid >> 5, lane = tid & 31;
        nr = n_r - 1 < h ? n_r - 1 : h;
        if (nr < 0) nr = 0;
        // warps 4-7 meanwhile: the diagonal block (stored lower triangle,
        // read down its columns, then mirrored) and the rows above the qr
        // rows (element (row, col) stored as (col, row): read along col)
        auto load_diag_and_above = [&]() {
            const int t4 = tid - 128;
            batched_copy<T>(
                n_r * n_r, t4, 128,
                [&](int k) {
                    const int r = k % n_r, c = k / n_r;
                    return r >= c ? bld(AB, ldab, n, o_qr_r + r, o_qr_r + c, bad) : T(0);
                },
                [&](int k, T v) {
                    const int r = k % n_r, c = k / n_r;
                    if (r >= c) S.Xs[r + (size_t)c * ldb1] = v;
                });
            batched_copy<T>(
                o_v * n_r, t4, 128, [&](int k) { return bld(AB, ldab, n, o_qr_r + k % n_r, o_up_c + k / n_r, bad); },
                [&](int k, T v) { S.Xb[k / n_r + (size_t)(k % n_r) * ldb1] = v; });
            asm volatile("bar.sync 2, 128;" ::: "memory");
            for (int idx = t4; idx < n_r * n_r; idx += 128) {
                const int r = idx % n_r, c = idx / n_r;
                if (r < c) S.Xs[r + (size_t)c * ldb1] = S.Xs[c + (size_t)r * ldb1];
            }
        };
        if constexpr (RQ == 1 && QQ <= 2) {
            if (warp == 0) {
                // 1. (n_r <= 32, h <= 8) warp 0 alone: QR of the n_r x h block,
                //    lane rows, all h columns in its registers, T formed on the
                //    way (for h = 16 the 4-warp QR below is faster)
                constexpr int QW = 4 * QQ;
                T a[QW];
#pragma unroll
                for (int c = 0; c < QW; ++c)
                    a[c] = (lane < n_r && c < h) ? bld(AB, ldab, n, o_qr_r + lane, o_qr_c + c, bad) : T(0);
                BTRACE(1);
                warp_qr<T, QW>(a, n_r, h, S.vs, S.tau, S.Ts, ldh1);
                BTRACE(2);
#pragma unroll
                for (int c = 0; c < QW; ++c)
                    if (lane < n_r && c < h) {
                        bst(AB, ldab, n, o_qr_r + lane, o_qr_c + c, lane <= c ? a[c] : T(0), bad);
                        if (c < nr) S.Us[lane + (size_t)c * ldb1] = lane < c ? T(0) : (lane == c ? T(1) : a[c]);
                    }
            } else if (warp >= 4 && nr > 0) {
                load_diag_and_above();
            }
        } else {
            if (warp < 4) {
                // 1. warps 0-3: QR of the n_r x h block in registers (lane rows,
                //    warp-cyclic columns), one warp per scheduler
                T a[QQ][RQ];
#pragma unroll
                for (int q = 0; q < QQ; ++q)
#pragma unroll
                    for (int t = 0; t < RQ; ++t) {
                        const int r = lane + 32 * t, c = warp + 4 * q;
                        a[q][t] = (r < n_r && c < h) ? bld(AB, ldab, n, o_qr_r + r, o_qr_c + c, bad) : T(0);
                    }
                BTRACE(1);
                reg_qr<T, RQ, QQ, 4, 1>(a, n_r, h, 0, S.vs, S.tau, S.Zs, S.Ts, ldh1);
                BTRACE(2);
                // 2. B[qr rows, qr cols] = [R; 0]; U explicit into shared memory
#pragma unroll
                for (int q = 0; q < QQ; ++q)
#pragma unroll
                    for (int t = 0; t < RQ; ++t) {
                        const int r = lane + 32 * t, c = warp + 4 * q;
                        if (r < n_r && c < h) {
                            bst(AB, ldab, n, o_qr_r + r, o_qr_c + c, r <= c ? a[q][t] : T(0), bad);
                            if (c < nr) S.Us[r + (size_t)c * ldb1] = r < c ? T(0) : (r == c ? T(1) : a[q][t]);
                        }
                    }
            } else if (nr > 0) {
                load_diag_and_above();
            }
        }
        __syncthreads();
        if (nr == 0) return;
    } else {
        // 1. QR of the n_r x h block
        batched_copy<T>(
            n_r * h, tid, nt, [&](int k) { return bld(AB, ldab, n, o_qr_r + k % n_r, o_qr_c + k / n_r, bad); },
            [&](int k, T v) { S.Xs[k % n_r + (size_t)(k / n_r) * ldb1] = v; });
        __syncthreads();
        BTRACE(1);
        nr = cta_qr(n_r, h, S.Xs, ldb1, S.tau, S.red);
        BTRACE(2);
        // 2. B[qr rows, qr cols] = [R; 0]
        for (int idx = tid; idx < n_r * h; idx += nt) {
            const int r = idx % n_r, c = idx / n_r;
            const T v = (r <= c) ? S.Xs[r + (size_t)c * ldb1] : T(0);
            bst(AB, ldab, n, o_qr_r + r, o_qr_c + c, v, bad);
        }
        if (nr == 0) {
            __syncthreads();
            return;
        }
        cta_extract_u(n_r, nr, nr, S.Xs, ldb1, S.Us, ldb1);
    }
    // 3. T (the register QR formed it; else from G = U^T U by one warp's
    //    recurrence when h <= 32) and U T
    if constexpr (RQ == 0) {
        if (nr <= 32) {
            __syncthreads();
            cta_gemm<T, true, false>(nr, nr, n_r, T(1), S.Us, ldb1, S.Us, ldb1, T(0), S.Zs, ldh1);
            __syncthreads();
            form_t_from_g(nr, S.Zs, ldh1, S.tau, S.Ts, ldh1);
        } else {
            __syncthreads();
            cta_form_t(n_r, nr, S.Us, ldb1, S.tau, S.Ts, ldh1, S.Zs, ldh1);
        }
    }
    constexpr bool kVec = sizeof(T) == 4;
    cta_mm<T, 4, 4, false, kVec>(n_r, nr, nr, T(1), S.Us, ldb1, S.Ts, ldh1, 0, nullptr, 0, nullptr, 0, T(0), S.UTs,
                                 ldb1);
    __syncthreads();
    BTRACE(3);
    // 4. the qr-row diagonal block X_d (n_r x n_r): two-sided update
    // (the stored lower triangle, read down its columns, then mirrored in
    // shared memory; on the register path it is already there)
    if constexpr (RQ == 0) {
        batched_copy<T>(
            n_r * n_r, tid, nt,
            [&](int k) {
                const int r = k % n_r, c = k / n_r;
                return r >= c ? bld(AB, ldab, n, o_qr_r + r, o_qr_r + c, bad) : T(0);
            },
            [&](int k, T v) {
                const int r = k % n_r, c = k / n_r;
                if (r >= c) S.Xs[r + (size_t)c * ldb1] = v;
            });
        __syncthreads();
        for (int idx = tid; idx < n_r * n_r; idx += nt) {
            const int r = idx % n_r, c = idx / n_r;
            if (r < c) S.Xs[r + (size_t)c * ldb1] = S.Xs[c + (size_t)r * ldb1];
        }
        __syncthreads();
    }
    BTRACE(6);
    chase_diag_update<T>(AB, ldab, n, n_r, nr, o_qr_r, S, bad);
    __syncthreads();
    BTRACE(4);
    // 5. the other rows of W (above: [0, o_v), below: [o_v + n_r, n_c)):
    //    X <- X - (X U T) U^T, in chunks of at most b rows
    for (int part = 0; part < 2; ++part) {
        const int a_begin = part == 0 ? 0 : o_v + n_r;
        const int a_end = part == 0 ? o_v : n_c;
        for (int a0 = a_begin; a0 < a_end; a0 += b) {
            const int rows = min(b, a_end - a0);
            // the block of this chunk: Xb for the rows above on the register
            // path (loaded during the QR; there is one chunk of o_v < b rows)
            T *X = (RQ > 0 && part == 0) ? S.Xb : S.Xs;
            if (part == 0 && RQ > 0) {
            } else if (part == 0) {
                // rows above the qr rows: element (row, col) is stored as (col, row), contiguous
                // along col -- consecutive threads take consecutive columns
                batched_copy<T>(
                    rows * n_r, tid, nt,
                    [&](int k) { return bld(AB, ldab, n, o_qr_r + k % n_r, o_up_c + a0 + k / n_r, bad); },
                    [&](int k, T v) { S.Xs[k / n_r + (size_t)(k % n_r) * ldb1] = v; });
            } else {
                batched_copy<T>(
                    rows * n_r, tid, nt,
                    [&](int k) { return bld(AB, ldab, n, o_up_c + a0 + k % rows, o_qr_r + k / rows, bad); },
                    [&](int k, T v) { S.Xs[k % rows + (size_t)(k / rows) * ldb1] = v; });
            }
            __syncthreads();
            if (part == 1 && a0 == a_begin) BTRACE(11);
            cta_mm<T, 4, 4, false, kVec>(rows, nr, n_r, T(1), X, ldb1, S.UTs, ldb1, 0, nullptr, 0, nullptr, 0, T(0),
                                         S.Ws, ldb1);
            __syncthreads();
            if (part == 1 && a0 == a_begin) BTRACE(12);
            // X <- X - W U^T: register-tiled for wide blocks, else folded into the stores
            const bool tiled = n_r >= 64;
            if (tiled) {
                cta_mm<T, 8, 8, true, kVec>(rows, n_r, nr, T(-1), S.Ws, ldb1, S.Us, ldb1, 0, nullptr, 0, nullptr, 0,
                                            T(1), X, ldb1);
                __syncthreads();
            }
            if (part == 1 && a0 == a_begin) BTRACE(13);
            auto updated = [&](int r, int c) {
                T v = X[r + (size_t)c * ldb1];
                if (!tiled)
                    for (int m = 0; m < nr; ++m) v -= S.Ws[r + (size_t)m * ldb1] * S.Us[c + (size_t)m * ldb1];
                return v;
            };
            if (part == 0) {
                for (int idx = tid; idx < rows * n_r; idx += nt) {
                    const int c = idx % n_r, r = idx / n_r;
                    bst(AB, ldab, n, o_qr_r + c, o_up_c + a0 + r, updated(r, c), bad);
                }
            } else {
                for (int idx = tid; idx < rows * n_r; idx += nt) {
                    const int r = idx % rows, c = idx / rows;
                    bst(AB, ldab, n, o_up_c + a0 + r, o_qr_r + c, updated(r, c), bad);
                }
            }
            __syncthreads();
        }
    }
    BTRACE(5);
}

// ------------------------------------------------ three-CTA cluster chase
// The same chase split over a cluster of three CTAs, for wide bands where
// one chase is long and only ~J/3 sweeps can progress at once (most SMs
// would idle): rank 0 factorises the qr block and updates the diagonal
// block X_d; rank 1 updates the rows above the qr rows and rank 2 the rows
// below (the one-sided X <- X - (X U T) U^T of each), each from its own
// copy of U and U T, read from rank 0's shared memory once rank 0 has
// formed them.  Ranks 1 and 2 load their blocks while rank 0 runs the QR.
// Two cluster barriers per chase: A (U, U T and nr ready on rank 0) and B
// (every write of the chase done; the next chase may start).
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_sync() {
    cluster_arrive();
    cluster_wait();
}
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Generic address of the same shared variable in CTA `rank` of the cluster.
template <typename P>
__device__ __forceinline__ P *cluster_map(P *p, unsigned rank) {
    unsigned long long out;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"((unsigned long long)p), "r"(rank));
    return (P *)out;
}

// One-sided update of one row block (rows x n_r, X[a + c ldb1], row a of
// the block <-> band position (row0 + a) for rank 2 or column (col0 + a) for
// rank 1): W = X (U T); X <- X - W U^T; written back.
template <typename T>
__device__ SEV_CHASE_PART_INLINE void chase_rows_update(T *AB, int ldab, int n, int rows, int n_r, int nr, int o_qr_r,
                                                        int base, bool above, ChaseSmem<T> &S, int &bad) {
    const int ldb1 = S.ldb1, tid = threadIdx.x, nt = blockDim.x;
    constexpr bool kVec = sizeof(T) == 4;
    T *X = S.Xs;
    cta_mm<T, 4, 4, false, kVec>(rows, nr, n_r, T(1), X, ldb1, S.UTs, ldb1, 0, nullptr, 0, nullptr, 0, T(0), S.Ws,
                                 ldb1);
    __syncthreads();
    const bool tiled = n_r >= 64;
    if (tiled) {
        cta_mm<T, 8, 8, true, kVec>(rows, n_r, nr, T(-1), S.Ws, ldb1, S.Us, ldb1, 0, nullptr, 0, nullptr, 0, T(1), X,
                                    ldb1);
        __syncthreads();
    }
    auto updated = [&](int r, int c) {
        T v = X[r + (size_t)c * ldb1];
        if (!tiled)
            for (int m = 0; m < nr; ++m) v -= S.Ws[r + (size_t)m * ldb1] * S.Us[c + (size_t)m * ldb1];
        return v;
    };
    if (above) {
        for (int idx = tid; idx < rows * n_r; idx += nt) {
            const int c = idx % n_r, r = idx / n_r;
            bst(AB, ldab, n, o_qr_r + c, base + r, updated(r, c), bad);
        }
    } else {
        for (int idx = tid; idx < rows * n_r; idx += nt) {
            const int r = idx % rows, c = idx / rows;
            bst(AB, ldab, n, base + r, o_qr_r + c, updated(r, c), bad);
        }
    }
}

// Rank `rank`'s share of chase (i, j).  *nr_r0 is rank 0's count of
// reflectors (shared-memory variable of rank 0, mapped).  Every rank passes
// cluster barrier A exactly once.
template <typename T, int RQ, int QQ>
__device__ void band_chase_x3(T *AB, int ldab, int n, int b, int h, int i, int j, ChaseSmem<T> &S, unsigned rank,
                              int *s_nr, int &bad) {
    const int o_qr_r = (i - 1) * h + (j - 1) * b + h;
    int o_qr_c, o_v, o_up_c, lim;
    if (j == 1) {
        o_qr_c = o_qr_r - h;
        o_v = 0;
        o_up_c = o_qr_r;
        lim = 2 * b;
    } else {
        o_qr_c = o_qr_r - b;
        o_v = b - h;
        o_up_c = o_qr_c + h;
        lim = 3 * b - h;
    }
    const int n_r = min(n - o_qr_r, b);
    const int n_c = min(n - o_up_c, lim);
    const int ldb1 = S.ldb1, ldh1 = S.ldh1;
    const int tid = threadIdx.x, nt = blockDim.x;
    constexpr bool kVec = sizeof(T) == 4;

    BTRACE3(0);
    if (rank != 0) {
        // the row block of this rank, loaded while rank 0 factorises
        const bool above = rank == 1;
        const int a0 = above ? 0 : o_v + n_r, rows = above ? o_v : n_c - (o_v + n_r);
        if (rows > 0) {
            if (above) {
                // element (qr row c, column o_up_c + a) is stored as (row, col) = (o_qr_r + c, o_up_c + a)
                batched_copy<T>(
                    rows * n_r, tid, nt, [&](int k) { return bld(AB, ldab, n, o_qr_r + k % n_r, o_up_c + k / n_r, bad); },
                    [&](int k, T v) { S.Xs[k / n_r + (size_t)(k % n_r) * ldb1] = v; });
            } else {
                batched_copy<T>(
                    rows * n_r, tid, nt,
                    [&](int k) { return bld(AB, ldab, n, o_up_c + a0 + k % rows, o_qr_r + k / rows, bad); },
                    [&](int k, T v) { S.Xs[k % rows + (size_t)(k / rows) * ldb1] = v; });
            }
        }
        BTRACE3(1);
        cluster_sync();  // A
        BTRACE3(2);
        int *nr0 = cluster_map(s_nr, 0);
        const int nr = *(volatile int *)nr0;
        if (rows <= 0 || nr <= 0) return;
        // U and U T from rank 0 (whole padded columns, 16-byte pieces)
        const float4 *src = (const float4 *)cluster_map(S.Us, 0);
        float4 *dst = (float4 *)S.Us;
        const int q_u = (int)(((size_t)ldb1 * nr * sizeof(T)) / 16);  // Us and UTs: columns of ldb1
        const int q_off = (int)(((size_t)ldb1 * h * sizeof(T)) / 16);  // UTs = Us + ldb1 h
        for (int q = tid; q < 2 * q_u; q += nt) {
            const int at = q < q_u ? q : q_off + (q - q_u);
            dst[at] = src[at];
        }
        __syncthreads();
        BTRACE3(3);
        chase_rows_update<T>(AB, ldab, n, rows, n_r, nr, o_qr_r, o_up_c + a0, above, S, bad);
        BTRACE3(4);
        return;
    }

    // ---- rank 0: QR of the n_r x h block, U, T, U T; then X_d
    const int warp = tid >> 5, lane = tid & 31;
    int nr = n_r - 1 < h ? n_r - 1 : h;
    if (nr < 0) nr = 0;
    if (warp < 4) {
        T a[QQ][RQ];
#pragma unroll
        for (int q = 0; q < QQ; ++q)
#pragma unroll
            for (int t = 0; t < RQ; ++t) {
                const int r = lane + 32 * t, c = warp + 4 * q;
                a[q][t] = (r < n_r && c < h) ? bld(AB, ldab, n, o_qr_r + r, o_qr_c + c, bad) : T(0);
            }
        BTRACE3(1);
        reg_qr<T, RQ, QQ, 4, 1>(a, n_r, h, 0, S.vs, S.tau, S.Zs, S.Ts, ldh1);
        BTRACE3(2);
#pragma unroll
        for (int q = 0; q < QQ; ++q)
#pragma unroll
            for (int t = 0; t < RQ; ++t) {
                const int r = lane + 32 * t, c = warp + 4 * q;
                if (r < n_r && c < h) {
                    bst(AB, ldab, n, o_qr_r + r, o_qr_c + c, r <= c ? a[q][t] : T(0), bad);
                    if (c < nr) S.Us[r + (size_t)c * ldb1] = r < c ? T(0) : (r == c ? T(1) : a[q][t]);
                }
            }
    } else if (nr > 0) {
        // warps 4-7 meanwhile: the diagonal block (lower triangle, mirrored)
        const int t4 = tid - 128;
        batched_copy<T>(
            n_r * n_r, t4, 128,
            [&](int k) {
                const int r = k % n_r, c = k / n_r;
                return r >= c ? bld(AB, ldab, n, o_qr_r + r, o_qr_r + c, bad) : T(0);
            },
            [&](int k, T v) {
                const int r = k % n_r, c = k / n_r;
                if (r >= c) S.Xs[r + (size_t)c * ldb1] = v;
            });
        asm volatile("bar.sync 2, 128;" ::: "memory");
        for (int idx = t4; idx < n_r * n_r; idx += 128) {
            const int r = idx % n_r, c = idx / n_r;
            if (r < c) S.Xs[r + (size_t)c * ldb1] = S.Xs[c + (size_t)r * ldb1];
        }
    }
    if (tid == 0) *s_nr = nr;
    __syncthreads();
    BTRACE3(3);
    if (nr > 0)  // T came out of the register QR
        cta_mm<T, 4, 4, false, kVec>(n_r, nr, nr, T(1), S.Us, ldb1, S.Ts, ldh1, 0, nullptr, 0, nullptr, 0, T(0),
                                     S.UTs, ldb1);
    BTRACE3(4);
    cluster_sync();  // A: U, U T and nr are ready for ranks 1 and 2
    BTRACE3(5);
    if (nr == 0) return;
    chase_diag_update<T>(AB, ldab, n, n_r, nr, o_qr_r, S, bad);
    BTRACE3(9);
}

// Capped wait of one thread until sweep s - 1 has completed `need` chases;
// false on expiry or a latched error (then the error word is set).
__device__ __forceinline__ bool wait_progress(const int *progress, int s, int need, int *err) {
    const long long t0 = clock64();
    while (ld_acquire(&progress[s - 1]) < need) {
        if (*(volatile int *)err != 0) return false;
        if (wait_expired(t0, err)) {
            latch_error(err, SEV_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// Cluster of three CTAs per sweep.  Rank 0 takes sweeps from the counter
// and hands the index to ranks 1 and 2 through its shared memory.  Every
// rank's thread 0 waits for the previous sweep itself (before barrier B of
// the preceding chase); a rank whose wait fails raises rank 0's abort flag,
// which every rank reads after the same barrier, so all three leave
// together, after one more barrier (no CTA exits while a peer may still
// read its shared memory).
template <typename T, int RQ, int QQ>
__global__ void __cluster_dims__(3, 1, 1) __launch_bounds__(kThreads)
    band_chase_x3_kernel(int n, T *AB, int ldab, int b, int h, int nsweeps, int *progress, int *sweep_ctr, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    ChaseSmem<T> S(smem, b, h);
    __shared__ int s_sweep, s_abort, s_nr;
    const unsigned rank = cluster_rank();
    int bad = 0;
    if (threadIdx.x == 0) {
        s_abort = 0;
        s_nr = 0;
    }
    int *abort0 = cluster_map(&s_abort, 0);
    int *sweep0 = cluster_map(&s_sweep, 0);
    cluster_sync();  // rank 0's flags are initialised before any rank may raise them
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) s_sweep = atomicAdd(sweep_ctr, 1);
        cluster_sync();  // C: the sweep index is published
        const int s = *(volatile int *)sweep0;
        if (s >= nsweeps) break;
        const int i = s + 1;
        const int J = band_num_chases(n, b, h, i);
        const int Jprev = i > 1 ? band_num_chases(n, b, h, i - 1) : 0;
        if (i > 1 && threadIdx.x == 0 && !wait_progress(progress, s, min(3, Jprev), err)) atomicOr(abort0, 1);
        cluster_sync();  // B of "chase 0": every rank may start chase 1
        if (*(volatile int *)abort0) break;
        for (int j = 1; j <= J; ++j) {
            band_chase_x3<T, RQ, QQ>(AB, ldab, n, b, h, i, j, S, rank, &s_nr, bad);
            __syncthreads();
            if (i > 1 && j < J && threadIdx.x == 0 && !wait_progress(progress, s, min(j + 3, Jprev), err))
                atomicOr(abort0, 1);
            cluster_sync();  // B: chase j is complete on all ranks
            // the release store orders the cluster's writes (made visible to
            // rank 0's thread 0 by the barrier) before the progress flag
            if (rank == 0 && threadIdx.x == 0) st_release(&progress[s], j);
            if (*(volatile int *)abort0) break;
        }
        if (*(volatile int *)abort0) break;
    }
    cluster_sync();  // no rank leaves while a peer may still read its shared memory
    if (__syncthreads_or(bad) && threadIdx.x == 0) latch_error(err, SEV_ERR_INTERNAL);
}

template <typename T, int RQ, int QQ>
__global__ void __launch_bounds__(kThreads) band_chase_kernel(int n, T *AB, int ldab, int b, int h, int nsweeps,
                                                               int *progress, int *sweep_ctr, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    ChaseSmem<T> S(smem, b, h);
    __shared__ int s_sweep, s_abort;
    int bad = 0;  // this thread met an index outside the band
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_sweep = atomicAdd(sweep_ctr, 1);
            s_abort = 0;
        }
        __syncthreads();
        const int s = s_sweep;
        if (s >= nsweeps) break;
        const int i = s + 1;
        const int J = band_num_chases(n, b, h, i);
        const int Jprev = i > 1 ? band_num_chases(n, b, h, i - 1) : 0;
        for (int j = 1; j <= J; ++j) {
            if (i > 1) {
                if (threadIdx.x == 0) {
                    const int need = min(j + 2, Jprev);
                    const long long t0 = clock64();
                    while (ld_acquire(&progress[s - 1]) < need) {
                        if (*(volatile int *)err != 0) {
                            s_abort = 1;
                            break;
                        }
                        if (wait_expired(t0, err)) {
                            latch_error(err, SEV_ERR_TIMEOUT);
                            s_abort = 1;
                            break;
                        }
                    }
                }
                __syncthreads();
                if (s_abort) return;
            }
            band_chase<T, RQ, QQ>(AB, ldab, n, b, h, i, j, S, bad);
            __syncthreads();
            // the release store orders the CTA's writes (made visible to
            // thread 0 by the barrier above) before the progress flag
            if (threadIdx.x == 0) st_release(&progress[s], j);
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) latch_error(err, SEV_ERR_INTERNAL);
}

size_t band_workspace(int n, int b, int h) {
    Carver c(nullptr);
    c.take<int>((size_t)band_num_sweeps(n, h) + 1);
    c.take<int>(1);
    return c.bytes();
}

// The cluster chase for tile (RQ, QQ); SEV_ERR_UNSUPPORTED when no cluster
// of three such CTAs fits on the GPU (the caller then runs one CTA a sweep).
template <typename T>
static int launch_chase_x3(sev_ctx *hd, int n, T *AB, int ldab, int b, int h, int nsweeps, int *progress, int *ctr,
                           int RQ, int QQ) {
    void (*kern)(int, T *, int, int, int, int, int *, int *, int *) = nullptr;
    if (RQ == 2 && QQ == 1) kern = band_chase_x3_kernel<T, 2, 1>;
    if (RQ == 2 && QQ == 2) kern = band_chase_x3_kernel<T, 2, 2>;
    if (RQ == 2 && QQ == 4) kern = band_chase_x3_kernel<T, 2, 4>;
    if (RQ == 2 && QQ == 8) kern = band_chase_x3_kernel<T, 2, 8>;
    if (RQ == 4 && QQ == 1) kern = band_chase_x3_kernel<T, 4, 1>;
    if (RQ == 4 && QQ == 2) kern = band_chase_x3_kernel<T, 4, 2>;
    if (RQ == 4 && QQ == 4) kern = band_chase_x3_kernel<T, 4, 4>;
    if (RQ == 4 && QQ == 8) kern = band_chase_x3_kernel<T, 4, 8>;
    if (RQ == 4 && QQ == 16) kern = band_chase_x3_kernel<T, 4, 16>;
    if (!kern) return SEV_ERR_UNSUPPORTED;
    const size_t smem = band_smem_bytes<T>(b, h);
    if (smem > hd->smem_optin) return SEV_ERR_UNSUPPORTED;
    SEV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int busy = band_num_chases(n, b, h, 0) / 3 + 8;
    int clusters = busy < nsweeps ? busy : nsweeps;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(3 * clusters);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = hd->stream;
    int fit = 0;
    if (cudaOccupancyMaxActiveClusters(&fit, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return SEV_ERR_UNSUPPORTED;
    }
    if (fit < 1) return SEV_ERR_UNSUPPORTED;
    if (clusters > fit) clusters = fit;
    SEV_LAUNCH(hd, K_BAND_CHASE, kern, 3 * clusters, kThreads, smem, n, AB, ldab, b, h, nsweeps, progress, ctr,
               hd->d_err);
    return SEV_OK;
}

template <typename T>
int launch_band_to_band(sev_ctx *hd, int n, T *AB, int ldab, int b, int h, void *ws, size_t ws_bytes) {
    const int nsweeps = band_num_sweeps(n, h);
    if (nsweeps <= 0) return SEV_OK;
    if (ws_bytes < band_workspace(n, b, h)) return SEV_ERR_WORKSPACE;
    size_t smem = band_smem_bytes<T>(b, h);
    if (smem > hd->smem_optin) return SEV_ERR_UNSUPPORTED;
    Carver c(ws);
    int *progress = c.take<int>((size_t)nsweeps + 1);
    int *ctr = c.take<int>(1);
    SEV_CUDA(cudaMemsetAsync(progress, 0, sizeof(int) * ((size_t)nsweeps + 1), hd->stream));
    SEV_CUDA(cudaMemsetAsync(ctr, 0, sizeof(int), hd->stream));
    // register path when its tile and its second block buffer fit
    const int RQ = chase_tile_r(b), QQ = chase_tile_q(h);
    // wide bands: the three-CTA cluster chase when a cluster fits
    if (RQ > 0 && QQ > 0 && b >= hd->chase_x3_min_b) {
        int rc = launch_chase_x3<T>(hd, n, AB, ldab, b, h, nsweeps, progress, ctr, RQ, QQ);
        if (rc != SEV_ERR_UNSUPPORTED) return rc;
    }
    auto kern = band_chase_kernel<T, 0, 0>;
    if (RQ > 0 && QQ > 0 && band_smem_reg<T>(b, h) <= hd->smem_optin) {
        smem = band_smem_reg<T>(b, h);
        if (RQ == 1 && QQ == 1) kern = band_chase_kernel<T, 1, 1>;
        if (RQ == 1 && QQ == 2) kern = band_chase_kernel<T, 1, 2>;
        if (RQ == 1 && QQ == 4) kern = band_chase_kernel<T, 1, 4>;
        if (RQ == 2 && QQ == 1) kern = band_chase_kernel<T, 2, 1>;
        if (RQ == 2 && QQ == 2) kern = band_chase_kernel<T, 2, 2>;
        if (RQ == 2 && QQ == 4) kern = band_chase_kernel<T, 2, 4>;
        if (RQ == 2 && QQ == 8) kern = band_chase_kernel<T, 2, 8>;
        if (RQ == 4 && QQ == 1) kern = band_chase_kernel<T, 4, 1>;
        if (RQ == 4 && QQ == 2) kern = band_chase_kernel<T, 4, 2>;
        if (RQ == 4 && QQ == 4) kern = band_chase_kernel<T, 4, 4>;
        if (RQ == 4 && QQ == 8) kern = band_chase_kernel<T, 4, 8>;
        if (RQ == 4 && QQ == 16) kern = band_chase_kernel<T, 4, 16>;
        if (kern == band_chase_kernel<T, 0, 0>) smem = band_smem_bytes<T>(b, h);
    }
    SEV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SEV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) return SEV_ERR_UNSUPPORTED;
    int grid = hd->sm_count * per_sm;
    // sweep i runs ~3 chases behind sweep i - 1, so about J/3 sweeps (J the
    // chases of the first) progress at once; CTAs beyond that would only poll
    // the progress flags of their predecessors and load the L2 with it
    const int busy = band_num_chases(n, b, h, 0) / 3 + 8;
    if (grid > busy) grid = busy;
    if (grid > nsweeps) grid = nsweeps;
    SEV_LAUNCH(hd, K_BAND_CHASE, kern, grid, kThreads, smem, n, AB, ldab, b, h, nsweeps, progress, ctr, hd->d_err);
    return SEV_OK;
}

template int launch_band_to_band<float>(sev_ctx *, int, float *, int, int, int, void *, size_t);
template int launch_band_to_band<double>(sev_ctx *, int, double *, int, int, int, void *, size_t);
template size_t band_smem_bytes<float>(int, int);
template size_t band_smem_bytes<double>(int, int);

}  // namespace sev
