// regtile.cuh -- register-tile primitives of the Householder kernels: a CTA of
// NW warps holds a (32 R) x (NW Q) block with lane l of warp w keeping
// a[q][t] = M(l + 32 t, w + NW q) (columns dealt to the warps cyclically, the
// rows of a column inside one warp).  reg_qr is a Householder QR with one
// barrier per column and a one-column lookahead; reg_apply_all applies a
// stored sequence of reflectors to warp-private columns without barriers.
// Used by the tree QR of the panel factorisation (panel_reg.cu) and by the
// QR step of every band chase (band.cu).
#pragma once

#include "common.cuh"

#ifdef SEV_TRACE
// per-step clocks of reg_qr in CTA 0 (trace builds only; set by the host)
static __device__ long long *sev_rtrace = nullptr;
#define RTRACE(k, slot)                                                                       \
    do {                                                                                      \
        if (sev_rtrace && blockIdx.x == 0 && blockIdx.y == 0 && (threadIdx.x & 31) == 0 && (k) < 256) \
            sev_rtrace[(k) * 8 + (slot)] = clock64();                                         \
    } while (0)
#else
#define RTRACE(k, slot) \
    do {                \
    } while (0)
#endif

namespace sev {

template <typename T>
__device__ __forceinline__ T fmat(T a, T b, T c);
template <>
__device__ __forceinline__ float fmat<float>(float a, float b, float c) {
    return fmaf(a, b, c);
}
template <>
__device__ __forceinline__ double fmat<double>(double a, double b, double c) {
    return fma(a, b, c);
}

// x[t] for a run-time t without dynamic register indexing.
template <int R, typename T>
__device__ __forceinline__ T rsel(const T (&x)[R], int t) {
    T r = x[0];
#pragma unroll
    for (int i = 1; i < R; ++i)
        if (i == t) r = x[i];
    return r;
}

// The 32-row blocks of the tile that can hold a nonzero of reflector k.
// bstack = 0: a dense block (reflector k lives in rows >= k); bstack = b (a
// multiple of 32): a stack of upper triangles of height b, where reflector k
// is nonzero only in row k of the first triangle and rows 0..k of the others.
// The block offsets are formed once, so the per-step test is a comparison.
template <int R>
struct RowBlocks {
    int toff[R];    // offset of block t's first row inside its triangle
    bool lower[R];  // block t lies in a triangle below the first
    int bstack;
    __device__ __forceinline__ explicit RowBlocks(int bs) : bstack(bs) {
#pragma unroll
        for (int t = 0; t < R; ++t) {
            lower[t] = bs > 0 && 32 * t >= bs;
            toff[t] = bs > 0 ? (32 * t) % bs : 32 * t;
        }
    }
    __device__ __forceinline__ bool active(int t, int k) const {
        if (bstack == 0) return 32 * t + 31 >= k;
        return lower[t] ? toff[t] <= k : (32 * t <= k && k < 32 * t + 32);
    }
};

// a <- H a on every column, H = I - tau v v^T, v given per lane row in vr
// (zero outside the active blocks), each column's update scaled by cm[q]
// (1: apply, 0: leave the column exactly as it is).  The branches are on
// the warp-uniform row blocks only; the dot products of all columns are
// reduced together so their shuffle chains overlap.
template <typename T, int R, int Q>
__device__ __forceinline__ void reg_apply(T (&a)[Q][R], const T (&vr)[R], const bool (&act)[R], T tau,
                                          const T (&cm)[Q], T (&dq)[Q]) {
    T d[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) d[q] = T(0);
#pragma unroll
    for (int t = 0; t < R; ++t)
        if (act[t]) {
#pragma unroll
            for (int q = 0; q < Q; ++q) d[q] = fmat(vr[t], a[q][t], d[q]);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < Q; ++q) d[q] += __shfl_xor_sync(0xffffffffu, d[q], o);
    T sc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        dq[q] = d[q];
        sc[q] = tau * d[q] * cm[q];
    }
#pragma unroll
    for (int t = 0; t < R; ++t)
        if (act[t]) {
#pragma unroll
            for (int q = 0; q < Q; ++q) a[q][t] = fmat(-sc[q], vr[t], a[q][t]);
        }
}

// Two FP32 FMAs in one instruction (fma.rn.f32x2: each lane rounded once,
// the same results as two fmaf).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n"
        " .reg .b64 ra, rb, rc, rd;\n"
        " mov.b64 ra, {%2, %3};\n"
        " mov.b64 rb, {%4, %5};\n"
        " mov.b64 rc, {%6, %7};\n"
        " fma.rn.f32x2 rd, ra, rb, rc;\n"
        " mov.b64 {%0, %1}, rd;\n"
        "}\n"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// Warp sums of Q per-lane values (Q = 2, 4, 8, 16) by a transposing butterfly:
// at each of the first log2 Q levels a lane keeps half of its remaining
// values and sends the other half to its partner, so the shuffles total
// Q - 1 + (5 - log2 Q) + Q (the last Q broadcast the sums) instead of 5 Q.
// On return d[q] holds the sum over the 32 lanes (every lane).
template <int Q>
__device__ __forceinline__ void warp_sums_x(float (&d)[Q]) {
    const int lane = threadIdx.x & 31;
    float c;
    if constexpr (Q == 16) {
        const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4, u2 = lane & 2;
        float a8[8], a4[4], b2[2];
#pragma unroll
        for (int j = 0; j < 8; ++j) a8[j] = (u16 ? d[j + 8] : d[j]) + __shfl_xor_sync(0xffffffffu, u16 ? d[j] : d[j + 8], 16);
#pragma unroll
        for (int j = 0; j < 4; ++j) a4[j] = (u8 ? a8[j + 4] : a8[j]) + __shfl_xor_sync(0xffffffffu, u8 ? a8[j] : a8[j + 4], 8);
#pragma unroll
        for (int j = 0; j < 2; ++j) b2[j] = (u4 ? a4[j + 2] : a4[j]) + __shfl_xor_sync(0xffffffffu, u4 ? a4[j] : a4[j + 2], 4);
        c = (u2 ? b2[1] : b2[0]) + __shfl_xor_sync(0xffffffffu, u2 ? b2[0] : b2[1], 2);
        c += __shfl_xor_sync(0xffffffffu, c, 1);
#pragma unroll
        for (int q = 0; q < 16; ++q)
            d[q] = __shfl_sync(0xffffffffu, c, ((q >> 3) & 1) * 16 + ((q >> 2) & 1) * 8 + ((q >> 1) & 1) * 4 + (q & 1) * 2);
    } else if constexpr (Q == 8) {
        const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
        float a4[4], b2[2];
#pragma unroll
        for (int j = 0; j < 4; ++j) a4[j] = (u16 ? d[j + 4] : d[j]) + __shfl_xor_sync(0xffffffffu, u16 ? d[j] : d[j + 4], 16);
#pragma unroll
        for (int j = 0; j < 2; ++j) b2[j] = (u8 ? a4[j + 2] : a4[j]) + __shfl_xor_sync(0xffffffffu, u8 ? a4[j] : a4[j + 2], 8);
        c = (u4 ? b2[1] : b2[0]) + __shfl_xor_sync(0xffffffffu, u4 ? b2[0] : b2[1], 4);
        c += __shfl_xor_sync(0xffffffffu, c, 2);
        c += __shfl_xor_sync(0xffffffffu, c, 1);
#pragma unroll
        for (int q = 0; q < 8; ++q) d[q] = __shfl_sync(0xffffffffu, c, ((q >> 2) & 1) * 16 + ((q >> 1) & 1) * 8 + (q & 1) * 4);
    } else if constexpr (Q == 4) {
        const bool u16 = lane & 16, u8 = lane & 8;
        float b2[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) b2[j] = (u16 ? d[j + 2] : d[j]) + __shfl_xor_sync(0xffffffffu, u16 ? d[j] : d[j + 2], 16);
        c = (u8 ? b2[1] : b2[0]) + __shfl_xor_sync(0xffffffffu, u8 ? b2[0] : b2[1], 8);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = __shfl_sync(0xffffffffu, c, ((q >> 1) & 1) * 16 + (q & 1) * 8);
    } else {
        static_assert(Q == 2, "warp_sums_x: Q = 2, 4, 8 or 16");
        const bool u16 = lane & 16;
        c = (u16 ? d[1] : d[0]) + __shfl_xor_sync(0xffffffffu, u16 ? d[0] : d[1], 16);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
#pragma unroll
        for (int q = 0; q < 2; ++q) d[q] = __shfl_sync(0xffffffffu, c, q * 16);
    }
}

// reg_apply for FP32 tiles of 2, 4, 8 or 16 columns per warp: the dot products
// and the updates two columns per instruction (ffma2), the column sums by
// warp_sums_x.
template <int R, int Q>
__device__ __forceinline__ void reg_apply_f32x2(float (&a)[Q][R], const float (&vr)[R], const bool (&act)[R],
                                                float tau, const float (&cm)[Q], float (&dq)[Q]) {
    float2 dd[Q / 2];
#pragma unroll
    for (int p = 0; p < Q / 2; ++p) dd[p] = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < R; ++t)
        if (act[t]) {
            const float2 vv = make_float2(vr[t], vr[t]);
#pragma unroll
            for (int p = 0; p < Q / 2; ++p) dd[p] = ffma2(vv, make_float2(a[2 * p][t], a[2 * p + 1][t]), dd[p]);
        }
    float d[Q];
#pragma unroll
    for (int p = 0; p < Q / 2; ++p) {
        d[2 * p] = dd[p].x;
        d[2 * p + 1] = dd[p].y;
    }
    warp_sums_x<Q>(d);
#pragma unroll
    for (int q = 0; q < Q; ++q) dq[q] = d[q];
    float2 ms[Q / 2];
#pragma unroll
    for (int p = 0; p < Q / 2; ++p) ms[p] = make_float2(-tau * d[2 * p] * cm[2 * p], -tau * d[2 * p + 1] * cm[2 * p + 1]);
#pragma unroll
    for (int t = 0; t < R; ++t)
        if (act[t]) {
            const float2 vv = make_float2(vr[t], vr[t]);
#pragma unroll
            for (int p = 0; p < Q / 2; ++p) {
                const float2 r = ffma2(ms[p], vv, make_float2(a[2 * p][t], a[2 * p + 1][t]));
                a[2 * p][t] = r.x;
                a[2 * p + 1][t] = r.y;
            }
        }
}

// x <- column q of a / column q of a <- x (q warp-uniform; one branch taken).
template <typename T, int R, int Q>
__device__ __forceinline__ void reg_col_get(const T (&a)[Q][R], int q, T (&x)[R]) {
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (i == q) {
#pragma unroll
            for (int t = 0; t < R; ++t) x[t] = a[i][t];
        }
}
template <typename T, int R, int Q>
__device__ __forceinline__ void reg_col_put(T (&a)[Q][R], int q, const T (&x)[R]) {
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (i == q) {
#pragma unroll
            for (int t = 0; t < R; ++t) a[i][t] = x[t];
        }
}

// x <- [rows < k unchanged; beta at row k; v below] and vout <- v (0 above
// row k, 1 at k), from the scalars of the reflector.
template <typename T, int R>
__device__ __forceinline__ void reg_house_store(T (&x)[R], int k, T tau, T beta, T inv, T *vout) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int t = 0; t < R; ++t) {
        const int row = lane + 32 * t;
        if (row == k) {
            x[t] = beta;
            vout[row] = T(1);
        } else if (row > k) {
            if (tau != T(0)) x[t] = x[t] * inv;
            vout[row] = x[t];
        } else {
            vout[row] = T(0);
        }
    }
}

// Reflector of rows k..m-1 of the column x (one warp; lane rows lane + 32 t;
// rows >= m are zero).  On return x holds beta at row k and v below it (rows
// < k untouched), vout[0 .. 32R) receives v (0 above k, 1 at k) and the
// return value is tau.  All lanes evaluate the scalars (no broadcast).
template <typename T, int R>
__device__ __forceinline__ T reg_house(T (&x)[R], int k, T *vout) {
    const int lane = threadIdx.x & 31;
    const T alpha = __shfl_sync(0xffffffffu, rsel<R>(x, k >> 5), k & 31);
    T tau, beta, inv;
    if constexpr (sizeof(T) == 4) {
        F2 a0{0.f, 0.f}, a1{0.f, 0.f};
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int row = lane + 32 * t;
            if (row > k) {
                if (t & 1)
                    f2_add_sq(a1, (float)x[t]);
                else
                    f2_add_sq(a0, (float)x[t]);
            }
        }
        RTRACE(k, 4);
        const F2 acc = warp_sum_f2(f2_add(a0, a1));
        RTRACE(k, 5);
        float tf, bf, iv;
        house_scalars_f2((float)alpha, acc, &tf, &bf, &iv);
        RTRACE(k, 6);
        tau = (T)tf;
        beta = (T)bf;
        inv = (T)iv;
    } else {
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int row = lane + 32 * t;
            if (row > k) {
                if (t & 1)
                    s1 = fma((double)x[t], (double)x[t], s1);
                else
                    s0 = fma((double)x[t], (double)x[t], s0);
            }
        }
        const double ssq = warp_sum(s0 + s1);
        const double al = (double)alpha;
        double td, bd, id;
        if ((ssq != 0.0 && ssq < 1e-280) || !(ssq < 1e300) || fabs(al) > 1e150 || (al != 0.0 && fabs(al) < 1e-140)) {
            // rare: rescale by an exact power of two so the squares neither
            // overflow nor underflow
            double amax = fabs(al);
#pragma unroll
            for (int t = 0; t < R; ++t)
                if (lane + 32 * t > k) amax = fmax(amax, fabs((double)x[t]));
            amax = warp_max(amax);
            int e2;
            frexp(amax, &e2);
            const double sc = ldexp(1.0, -e2);
            double a2 = 0.0;
#pragma unroll
            for (int t = 0; t < R; ++t)
                if (lane + 32 * t > k) {
                    const double y = (double)x[t] * sc;
                    a2 = fma(y, y, a2);
                }
            a2 = warp_sum(a2);
            house_scalars(al * sc, a2, &td, &bd, &id);
            bd /= sc;
            id *= sc;
        } else {
            house_scalars(al, ssq, &td, &bd, &id);
        }
        tau = (T)td;
        beta = (T)bd;
        inv = (T)id;
    }
    reg_house_store<T, R>(x, k, tau, beta, inv, vout);
    return tau;
}

// Householder QR of the m x nc block held in `a` (m <= 32R, nc <= NW Q;
// rows >= m and columns >= nc zero), r = min(nc, m - 1) reflectors.  On
// return column c holds R above and on the diagonal and v_c below it (unit
// diagonal implicit); taus[c] = tau_c.  vs: 3 x 32R shared scratch.  With
// Gm and Tm (shared, leading dimension ldg >= r) the compact-WY factor T of
// the r reflectors is formed on the way (into Tm; Gm receives G = V^T V
// above its diagonal): every dot product of a reflector with a finished
// column is an entry of G that the trailing update computes anyway, and
// column k - 2 of T is formed in step k by an otherwise waiting warp.
//
// Step k applies reflector k.  The warp owning column k + 1 first brings
// that column up to date and forms reflector k + 1 from it (lookahead); it
// leaves its other columns for the next step, where it applies reflectors
// k and k + 1 to them back to back while the next owner forms reflector
// k + 2.  So a step lasts one column update plus one reflector, the owner's
// share of the trailing update being off the critical path; every column
// still receives the reflectors in order 0, 1, 2, ... (the same arithmetic
// as applying them one step at a time).  Reflectors rotate through three
// buffers: the deferred warp still reads reflector k - 1 in step k while
// the owner writes k + 1.
// Barrier of the warps running reg_qr: the whole CTA (BAR = 0) or named
// barrier BAR over warps 0 .. NW-1 (the rest of the CTA does other work).
template <int NW, int BAR>
__device__ __forceinline__ void reg_sync() {
    if constexpr (BAR == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NW * 32) : "memory");
}

// The reflector in buffer slot k % 3, restricted to the row blocks it can
// touch, applied to this warp's columns c with lo < c < nc; with Gm, the
// dot products with the finished columns are kept as entries of G.
template <typename T, int R, int Q, int NW>
__device__ __forceinline__ void reg_apply_step(T (&a)[Q][R], const RowBlocks<R> &blk, const T *vs, const T *taus,
                                               int k, int lo, int nc, T *Gm, int ldg) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T tk = taus[k];
    if (tk == T(0)) {
        if (Gm && lane == 0) {  // T's column k is zero then; no stale value reaches it
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int c = warp + NW * q;
                if (c < k) Gm[c + (size_t)k * ldg] = T(0);
            }
        }
        return;
    }
    const T *v = vs + (k % 3) * (32 * R);
    bool act[R];
    T vr[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
        act[t] = blk.active(t, k);
        vr[t] = act[t] ? v[lane + 32 * t] : T(0);
    }
    T cm[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int c = warp + NW * q;
        cm[q] = (c > lo && c < nc) ? T(1) : T(0);
    }
    T dq[Q];
    if constexpr (sizeof(T) == 4 && (Q == 2 || Q == 4 || Q == 8 || Q == 16))
        reg_apply_f32x2<R, Q>(a, vr, act, tk, cm, dq);
    else
        reg_apply<T, R, Q>(a, vr, act, tk, cm, dq);
    // G(c, k) = v_c^T v_k for this warp's finished columns c < k: the dot
    // of reflector k with column c (rows >= k hold v_c there)
    if (Gm && lane == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int c = warp + NW * q;
            if (c < k) Gm[c + (size_t)k * ldg] = dq[q];
        }
    }
}

// Column k of the compact-WY factor T (forward, column-wise: Q = I - V T V^T,
// T upper triangular, r x r) by one warp: T(k, k) = tau_k, for a < k
// T(a, k) = -tau_k sum_{q = a}^{k-1} T(a, q) G(q, k) with G = V^T V, and
// zeros below the diagonal.
template <typename T>
__device__ __forceinline__ void reg_t_column(int k, int r, const T *taus, const T *Gm, T *Tm, int ldg) {
    const int lane = threadIdx.x & 31;
    const T tk = taus[k];
    for (int a = k + 1 + lane; a < r; a += 32) Tm[a + (size_t)k * ldg] = T(0);
    for (int a = lane; a <= k; a += 32) {
        T s0 = 0, s1 = 0;
        int q = a;
        for (; q + 1 < k; q += 2) {
            s0 += Tm[a + (size_t)q * ldg] * Gm[q + (size_t)k * ldg];
            s1 += Tm[a + (size_t)(q + 1) * ldg] * Gm[q + 1 + (size_t)k * ldg];
        }
        if (q < k) s0 += Tm[a + (size_t)q * ldg] * Gm[q + (size_t)k * ldg];
        Tm[a + (size_t)k * ldg] = a == k ? tk : -tk * (s0 + s1);
    }
}

template <typename T, int R, int Q, int NW, int BAR = 0>
__device__ int reg_qr(T (&a)[Q][R], int m, int nc, int bstack, T *vs, T *taus, T *Gm = nullptr,
                      T *Tm = nullptr, int ldg = 0) {
    static_assert(NW >= 2, "reg_qr: the owner of a column and of the next one must differ");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = nc < m - 1 ? nc : m - 1;
    if (r <= 0) {
        reg_sync<NW, BAR>();
        return 0;
    }
    const RowBlocks<R> blk(bstack);
    if (warp == 0) {
        const T t0 = reg_house<T, R>(a[0], 0, vs);
        if (lane == 0) taus[0] = t0;
    }
    reg_sync<NW, BAR>();
    // k = r: no step, only the last owner's deferred share (reflector r - 1
    // on its columns past r)
    for (int k = 0; k <= r; ++k) {
        const int k1 = k + 1;
        const bool step = k < r;
        if (warp == 0 && step) RTRACE(k, 0);
        if (step && k1 < nc && (k1 % NW) == warp) {
            // owner of column k + 1: that column only (taken out of the tile,
            // so the reflector code is emitted once), then reflector k + 1
            const T tk = taus[k];
            const T *v = vs + (k % 3) * (32 * R);
            bool act[R];
            T vr[R];
#pragma unroll
            for (int t = 0; t < R; ++t) {
                act[t] = blk.active(t, k);
                vr[t] = act[t] ? v[lane + 32 * t] : T(0);
            }
            const int q1 = k1 / NW;
            T x[1][R];
            reg_col_get<T, R, Q>(a, q1, x[0]);
            if (tk != T(0)) {
                const T one[1] = {T(1)};
                T d1[1];
                reg_apply<T, R, 1>(x, vr, act, tk, one, d1);
            }
            RTRACE(k, 1);
            if (k1 < r) {
                const T t1 = reg_house<T, R>(x[0], k1, vs + (k1 % 3) * (32 * R));
                if (lane == 0) taus[k1] = t1;
            }
            RTRACE(k, 2);
            reg_col_put<T, R, Q>(a, q1, x[0]);
        } else {
            // the previous owner (column k is its own) catches up on
            // reflector k - 1 first (column k already has it); one loop, so
            // the update code is emitted once
            const bool deferred = k >= 1 && k < nc && (k % NW) == warp;
            const int kend = step ? k : k - 1;
            for (int kk = deferred ? k - 1 : k; kk <= kend; ++kk)
                reg_apply_step<T, R, Q, NW>(a, blk, vs, taus, kk, k, nc, Gm, ldg);
            // T's column k - 2 (G(., k - 2) is complete since the last
            // barrier) by a warp that neither owns column k + 1 nor is
            // catching up (warp k mod NW): warp (k + 2) mod NW
            if (Tm && NW >= 3 && step && k >= 2 && warp == (k + 2) % NW) reg_t_column<T>(k - 2, r, taus, Gm, Tm, ldg);
        }
        if (step) {
            if (k1 < nc && (k1 % NW) == warp) RTRACE(k, 3);
            reg_sync<NW, BAR>();
        }
    }
    if (Tm) {
        // the last columns of T (all of them with two warps), in order
        reg_sync<NW, BAR>();
        if (warp == 0)
            for (int k = (NW >= 3 ? (r - 2 > 0 ? r - 2 : 0) : 0); k < r; ++k) {
                reg_t_column<T>(k, r, taus, Gm, Tm, ldg);
                __syncwarp();
            }
        reg_sync<NW, BAR>();
    }
    return r;
}

// Householder QR of an m x nc block (m <= 32, nc <= Q) held by ONE warp:
// lane l keeps row l of every column (a[q] = M(l, q)).  No barrier: each
// step forms reflector k from column k (reg_house; v through the 32-entry
// scratch vs) and applies it to the later columns, the dot products of all
// columns summed together (transposing butterfly); the sums for the
// finished columns are G(q, k) = v_q^T v_k, from which lane a forms row a
// of the compact-WY factor T (forward, column-wise) in registers:
// T(a, k) = -tau_k sum_{q = a}^{k-1} T(a, q) G(q, k), T(k, k) = tau_k.  On
// return column c holds R on and above the diagonal and v_c below; taus[c]
// and T (r x r, leading dimension ldt, zeros below the diagonal) are in
// shared memory; returns r = min(nc, m - 1).
template <typename T, int Q>
__device__ int warp_qr(T (&a)[Q], int m, int nc, T *vs, T *taus, T *Tm, int ldt) {
    const int lane = threadIdx.x & 31;
    int r = nc < m - 1 ? nc : m - 1;
    if (r < 0) r = 0;
    T trow[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) trow[q] = T(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        if (k < r) {
            T x[1] = {a[k]};
            const T tk = reg_house<T, 1>(x, k, vs);
            a[k] = x[0];
            __syncwarp();
            const T v = vs[lane];
            __syncwarp();
            T d[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) d[q] = q == k ? T(0) : v * a[q];
            if constexpr (sizeof(T) == 4 && (Q == 2 || Q == 4 || Q == 8 || Q == 16)) {
                warp_sums_x<Q>(d);
            } else {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int q = 0; q < Q; ++q) d[q] += __shfl_xor_sync(0xffffffffu, d[q], o);
            }
#pragma unroll
            for (int q = k + 1; q < Q; ++q) a[q] = fmat(-tk * d[q], v, a[q]);
            T sacc = T(0);
#pragma unroll
            for (int q = 0; q < k; ++q) sacc = fmat(trow[q], d[q], sacc);
            trow[k] = lane < k ? -tk * sacc : (lane == k ? tk : T(0));
            if (lane == 0) taus[k] = tk;
        }
    }
    if (lane < r) {
#pragma unroll
        for (int q = 0; q < Q; ++q)
            if (q < r) Tm[lane + (size_t)q * ldt] = trow[q];
    }
    __syncwarp();
    return r;
}

// M <- H_0 H_1 ... H_{nr-1} M: reflectors explicit in Vs (column k at
// Vs[k * ldv], rows 0 .. 32R), scalars in taus; columns of M with cm[q] = 1.
template <typename T, int R, int Q>
__device__ void reg_apply_all(T (&m)[Q][R], const T *Vs, int ldv, const T *taus, int nr, int bstack,
                              const T (&cm)[Q]) {
    const int lane = threadIdx.x & 31;
    const RowBlocks<R> blk(bstack);
    for (int k = nr - 1; k >= 0; --k) {
        const T tk = taus[k];
        if (tk == T(0)) continue;
        bool act[R];
        T vr[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            act[t] = blk.active(t, k);
            vr[t] = act[t] ? Vs[(size_t)k * ldv + lane + 32 * t] : T(0);
        }
        T dq[Q];
        if constexpr (sizeof(T) == 4 && (Q == 2 || Q == 4 || Q == 8 || Q == 16))
            reg_apply_f32x2<R, Q>(m, vr, act, tk, cm, dq);
        else
            reg_apply<T, R, Q>(m, vr, act, tk, cm, dq);
    }
}

}  // namespace sev
