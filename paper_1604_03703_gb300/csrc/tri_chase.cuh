// tri_chase.cuh -- one b -> 1 bulge-chase step (Algorithm 4.2 with h = 1)
// performed by a single warp on a column window of the packed band, shared
// by the sliding-window kernel (band_tri.cu) and the batched kernel
// (batched.cu).  See band_tri.cu for the index sets of a chase.
#pragma once
#include "common.cuh"

#ifndef TRACEP
#define TRACEP(k) \
    do {          \
    } while (0)
#endif

namespace sev {

constexpr int kTriInf = 1 << 30;

__device__ __forceinline__ int ld_acquire_i(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_i(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__host__ __device__ __forceinline__ int tri_chases(int n, int b, int i) {
    const int r = n - i;
    return r < 2 ? 0 : (n - 2 - i) / b + 1;
}

template <typename T, int B>
struct TriWin {
    T *w;      // ring of WCAP columns x LDW diagonals
    int wcap;  // columns in the ring
    static constexpr int LDW = 2 * B;
    __device__ __forceinline__ T &at(int r, int c) const {  // r >= c, r - c < 2B
        return w[(c % wcap) * LDW + (r - c)];
    }
    __device__ __forceinline__ T &sym(int u, int q) const { return u >= q ? at(u, q) : at(q, u); }
};

// Reflector scalars from this lane's x (lanes t < nr hold x_t), computed by
// every lane (no divergence): FP32 data -- pair-float sum of squares over the
// B-lane group and pair-float scalars (house_scalars_f2); FP64 data -- FP64.
template <typename T, int B>
__device__ __forceinline__ void tri_reflector(T x, int nr, T &v, T &tau, T &beta) {
    constexpr int W = B < 32 ? B : 32;
    const int lane = threadIdx.x & 31;
    if constexpr (sizeof(T) == 4) {
        F2 acc{0.f, 0.f};
        if (lane >= 1 && lane < nr) f2_add_sq(acc, (float)x);
        acc = warp_sum_f2<W>(acc);
        float tf, bf, inf;
        house_scalars_f2(__shfl_sync(0xffffffffu, (float)x, 0), acc, &tf, &bf, &inf);
        tau = (T)tf;
        beta = (T)bf;
        v = lane == 0 ? T(1) : (lane < nr ? x * (T)inf : T(0));
    } else {
        const double xd = (lane >= 1 && lane < nr) ? (double)x : 0.0;
        double a = xd * xd;
#pragma unroll
        for (int off = W / 2; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        const double alpha = (double)__shfl_sync(0xffffffffu, x, 0);
        double td, bd, id;
        house_scalars(alpha, a, &td, &bd, &id);
        tau = (T)td;
        beta = (T)bd;
        v = lane == 0 ? T(1) : (lane < nr ? x * (T)id : T(0));
    }
}

// One chase (i, j), h = 1, by one warp on the shared window, with the rows a
// lane owns held in registers: lane l owns update row up0 + l above the qr
// rows, qr row o + l and row o + n_r + l below them.  The reflector (v in
// lane t, tau, beta) arrives in registers; if the sweep has a next chase,
// its reflector -- a function of column o after this chase only -- is formed
// here and returned the same way (its column gets [beta'; 0]).
// FULL: an interior chase (j > 1, o + 3b <= n, a next chase follows), where
// every block has its full size: the sizes are compile-time constants and
// the per-lane bounds tests on n drop out.
// A chase is compiled as a function of its own: inlined into the
// sliding-window kernel, whose loader and writer code shares the register
// allocation, its stores alone took ~2.8K cycles against ~0.5K (16 -> 1
// stage 222 -> 180 ms at n = 16384).
#ifndef SEV_TRI_CHASE_INLINE
#define SEV_TRI_CHASE_INLINE __noinline__
#endif
template <typename T, int B, bool FULL = false>
__device__ __forceinline__ void tri_chase_body(int n, int o, int j, bool has_next_rt, const TriWin<T, B> &W,
                                               T *vbuf, T *wbuf, T &v, T &tau, T &beta) {
    constexpr int LDW = 2 * B;
    const int lane = threadIdx.x & 31;
    const int wcap = W.wcap;
    T *const w = W.w;
    const bool has_next = FULL ? true : has_next_rt;
    const int n_r = FULL ? B : min(n - o, B);
    int up0, nc, ov;
    if (FULL) {
        up0 = o - B + 1;
        nc = 3 * B - 1;
        ov = B - 1;
    } else if (j == 1) {
        up0 = o;
        nc = min(n - o, 2 * B);
        ov = 0;
    } else {
        up0 = o - B + 1;
        nc = min(n - up0, 3 * B - 1);
        ov = B - 1;
    }
    const int so = o % wcap;
    auto cslot = [&](int q) {  // slot of column o + q (q < B)
        const int sl = so + q;
        return sl >= wcap ? sl - wcap : sl;
    };
    TRACEP(0);
    // broadcast v
    if (lane < B) vbuf[lane] = v;
    __syncwarp();
    T vv[B];
#pragma unroll
    for (int q = 0; q < B; ++q) vv[q] = q < n_r ? vbuf[q] : T(0);
    const T tt = tau;
    // load the owned rows (all loads in flight before any use)
    const bool has_a = lane < ov;
    const int ua = up0 + lane;  // above: entries (o + q, ua), column ua
    T *rowa = w + (size_t)((has_a ? ua : o) % wcap) * LDW + (o - (has_a ? ua : o));
    const int ub = o + n_r + lane;  // below: entries (ub, o + q)
    const bool has_b = lane < B && ub < up0 + nc;
    const bool has_d = lane < n_r;  // diag: entries of qr row o + lane
    const int sd = cslot(lane < B ? lane : 0);
    T ra[B], rb[B], rd[B];
#pragma unroll
    for (int q = 0; q < B; ++q) {
        ra[q] = (has_a && q < n_r) ? rowa[q] : T(0);
        rb[q] = (has_b && q < n_r) ? w[(size_t)cslot(q) * LDW + (ub - o - q)] : T(0);
        T dv = T(0);
        if (has_d && q < n_r) dv = q <= lane ? w[(size_t)cslot(q) * LDW + (lane - q)] : w[(size_t)sd * LDW + (q - lane)];
        rd[q] = dv;
    }
    TRACEP(1);
    // off rows: X <- X (I - tau v v^T)
    T sa = 0, sb = 0, p = 0;
#pragma unroll
    for (int q = 0; q < B; ++q) {
        sa = fma(ra[q], vv[q], sa);
        sb = fma(rb[q], vv[q], sb);
        p = fma(rd[q], vv[q], p);
    }
    sa *= tt;
    sb *= tt;
    p *= tt;
#pragma unroll
    for (int q = 0; q < B; ++q) {
        ra[q] = fma(-sa, vv[q], ra[q]);
        rb[q] = fma(-sb, vv[q], rb[q]);
    }
    TRACEP(2);
    // the next chase's reflector: column o of the rows below, x_t = rb[0] of lane t
    T nv = T(0), ntau = T(0), nbeta = T(0);
    const int n_r_next = FULL ? B : (has_next ? min(n - (o + B), B) : 0);
    if (has_next) tri_reflector<T, B>(rb[0], n_r_next, nv, ntau, nbeta);
    TRACEP(3);
    // qr-row block: H X H = X - v w^T - w v^T, w = p - (tau/2)(p^T v) v
    const T vl = lane < n_r ? v : T(0);  // this lane's own v (a runtime index into vv would spill)
    T ptv = has_d ? p * vl : T(0);
#pragma unroll
    for (int off = (B < 32 ? B : 32) / 2; off > 0; off >>= 1) ptv += __shfl_xor_sync(0xffffffffu, ptv, off);
    const T wl = p - T(0.5) * tt * ptv * vl;
    if (lane < B) wbuf[lane] = wl;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const T wq = wbuf[q];
        rd[q] = fma(-vl, wq, fma(-wl, vv[q], rd[q]));
    }
    TRACEP(4);
    // store back (the next reflector's column gets [beta'; 0])
#pragma unroll
    for (int q = 0; q < B; ++q) {
        if (has_a && q < n_r) rowa[q] = ra[q];
        if (has_b && q < n_r) {
            T val = rb[q];
            if (q == 0 && has_next && lane < n_r_next) val = lane == 0 ? nbeta : T(0);
            w[(size_t)cslot(q) * LDW + (ub - o - q)] = val;
        }
        if (has_d && q < n_r && q <= lane) w[(size_t)cslot(q) * LDW + (lane - q)] = rd[q];
    }
    __syncwarp();
    TRACEP(5);
    v = nv;
    tau = ntau;
    beta = nbeta;
}

// The chase as the sliding-window kernel calls it (see SEV_TRI_CHASE_INLINE);
// the batched kernel inlines tri_chase_body, which is faster there.
template <typename T, int B, bool FULL = false>
__device__ SEV_TRI_CHASE_INLINE void tri_chase(int n, int o, int j, bool has_next_rt, const TriWin<T, B> &W, T *vbuf,
                                               T *wbuf, T &v, T &tau, T &beta) {
    tri_chase_body<T, B, FULL>(n, o, j, has_next_rt, W, vbuf, wbuf, v, tau, beta);
}

}  // namespace sev
