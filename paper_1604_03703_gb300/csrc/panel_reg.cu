// panel_reg.cu -- the panel factorisation of the full-to-band reduction (the
// QR step of Algorithm 4.1: tree QR of Algorithm 3.2, then Householder
// reconstruction of Cor. 3.7) with the matrix blocks held in REGISTERS.
//
// Register tile.  A CTA of NW warps holds a (32 R) x (NW Q) block: lane l
// of warp w keeps a[q][t] = M(l + 32 t, w + NW q).  Columns are dealt to the
// warps cyclically, so the active (not yet factorised) columns stay spread
// over all warps as the factorisation proceeds, and every row of a column
// sits in one warp, so a column's dot product is a lane-local sum followed
// by one warp butterfly.  The leaf and node QRs of FP32 panels run on 8
// warps (fewer warps share each scheduler with the column owner), the
// applies and the reconstruction on 16.
//
// QR (reg_qr, regtile.cuh).  Householder QR, one reflector per column, one
// barrier per column.  At step k the warp owning column k+1 applies H_k to
// that column and forms reflector k+1 from it (lookahead), leaving its other
// columns to the next step; every other warp applies H_k = I - tau_k v_k
// v_k^T to its columns c > k.  v_k travels through three shared buffers.
// Scalars: the "always reflect" rule, beta = -sgn(alpha) ||x||,
// tau = (beta - alpha)/beta (FP64-accurate for FP32 data through the
// pair-float routine, see common.cuh).  Stacked triangles (the tree nodes)
// are handled with their structure: reflector k is nonzero only in row k of
// the top triangle and rows 0..k of the lower ones (the other entries are
// exact zeros), so 32-row blocks without such a row are skipped -- bit for
// bit the same result as the dense loop.
//
// Apply (reg_apply_all).  M <- H_0 H_1 ... H_{r-1} M with all reflectors in
// shared memory and M's columns private to their warps: no barrier at all.
//
// Reconstruction (recon_reg_kernel).  Unpivoted LU of Q1 - S with the sign
// S_kk = -sgn(current pivot) chosen during the elimination (|pivot| >= 1),
// W1^{-1} and U1^{-1} by column sweeps, T = -(W1 S) U1^{-T}: every
// elimination step is a rank-1 update of register tiles with the pivot
// column broadcast through shared memory and the pivot row through a shuffle.
#include "regtile.cuh"

#ifdef SEV_TRACE
extern "C" int sev_trace_set_reg(void *p) {
    return cudaMemcpyToSymbol(sev_rtrace, &p, sizeof(p)) == cudaSuccess ? 0 : 1;
}
#endif

namespace sev {

constexpr int kRegWarps = 16;
constexpr int kRegThreads = kRegWarps * 32;

// ------------------------------------------------------------- tree plan
// Leaf l covers panel rows [l N / L, (l + 1) N / L).
__host__ __device__ __forceinline__ int rleaf_row0(int N, int L, int l) { return (int)((long long)l * N / L); }

// --------------------------------------------------------------- kernels
// Leaf QR: CTA l factorises its rows of the N x b panel P (ldp).  Writes the
// explicit unit lower trapezoidal V into Y (rows of the leaf, ldy), tau,
// the number of reflectors and R (b x b, upper) into Rbuf[l].
template <typename T, int R, int Q, int NW>
__global__ void __launch_bounds__(NW * 32, 1)
    rtsqr_leaf_qr_kernel(const T *__restrict__ P, int ldp, int N, int b, int L, T *__restrict__ Y, int ldy,
                         T *__restrict__ tau, int *__restrict__ nref, T *__restrict__ Rbuf) {
    __shared__ __align__(16) T vs[3 * 32 * R];
    __shared__ T taus[NW * Q];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int l = blockIdx.x;
    const int row0 = rleaf_row0(N, L, l);
    const int rows = rleaf_row0(N, L, l + 1) - row0;
    T a[Q][R];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int c = warp + NW * q, r = lane + 32 * t;
            a[q][t] = (c < b && r < rows) ? P[(size_t)(row0 + r) + (size_t)c * ldp] : T(0);
        }
    const int nr = reg_qr<T, R, Q, NW>(a, rows, b, 0, vs, taus);
    T *Rl = Rbuf + (size_t)l * b * b;
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int c = warp + NW * q, r = lane + 32 * t;
            if (c >= b) continue;
            if (r < rows) {
                T v = T(0);
                if (c < nr) v = r < c ? T(0) : (r == c ? T(1) : a[q][t]);
                Y[(size_t)(row0 + r) + (size_t)c * ldy] = v;
            }
            if (r < b) Rl[r + (size_t)c * b] = (r <= c && r < rows) ? a[q][t] : T(0);
        }
    for (int c = threadIdx.x; c < b; c += blockDim.x) tau[(size_t)l * b + c] = c < nr ? taus[c] : T(0);
    if (threadIdx.x == 0) nref[l] = nr;
}

// Node QR: CTA p of a level stacks the R's of its two children (one child:
// pass-through) and factorises the 2b x b stack of upper triangles.
template <typename T, int R, int Q, int NW>
__global__ void __launch_bounds__(NW * 32, 1)
    rtsqr_node_qr_kernel(int b, int cnt_child, int off_child, int off_node, T *__restrict__ Rbuf,
                         T *__restrict__ Ylev, size_t ystride, T *__restrict__ tau, int *__restrict__ nref) {
    __shared__ __align__(16) T vs[3 * 32 * R];
    __shared__ T taus[NW * Q];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x;
    const int c0 = 2 * p, nc = min(2, cnt_child - c0);
    const int node = off_node + p;
    T *Rn = Rbuf + (size_t)node * b * b;
    if (nc == 1) {
        const T *Rc = Rbuf + (size_t)(off_child + c0) * b * b;
        for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) Rn[idx] = Rc[idx];
        if (threadIdx.x == 0) nref[node] = 0;
        return;
    }
    const int rows = 2 * b;
    T a[Q][R];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int c = warp + NW * q, r = lane + 32 * t;
            const int i = r % b;
            a[q][t] = (c < b && r < rows && i <= c) ? Rbuf[(size_t)(off_child + c0 + r / b) * b * b + i + (size_t)c * b]
                                                     : T(0);
        }
    const int nr = reg_qr<T, R, Q, NW>(a, rows, b, b % 32 == 0 ? b : 0, vs, taus);
    T *Y = Ylev + (size_t)p * ystride;
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int c = warp + NW * q, r = lane + 32 * t;
            if (c >= b) continue;
            if (r < rows) {
                T v = T(0);
                if (c < nr) v = r < c ? T(0) : (r == c ? T(1) : a[q][t]);
                Y[r + (size_t)c * rows] = v;
            }
            if (r < b) Rn[r + (size_t)c * b] = r <= c ? a[q][t] : T(0);
        }
    for (int c = threadIdx.x; c < b; c += blockDim.x) tau[(size_t)node * b + c] = c < nr ? taus[c] : T(0);
    if (threadIdx.x == 0) nref[node] = nr;
}

// Node apply (the way down): CTA (p, slice) pushes columns
// [slice 16Q, slice 16Q + 16Q) of the node's Z (identity at the root)
// through the node's reflectors, [Z; 0] -> H [Z; 0], and scatters the b-row
// blocks of the result to the children's Z.
template <typename T, int R, int Q>
__global__ void __launch_bounds__(kRegThreads, 1)
    rtsqr_node_apply_kernel(int b, int cnt_child, int off_child, int off_node, const T *__restrict__ Ylev,
                            size_t ystride, const T *__restrict__ tau, const int *__restrict__ nref,
                            T *__restrict__ Zbuf, int root_identity) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Vs = (T *)smem_raw;  // nr x 32R
    T *taus = Vs + (size_t)32 * R * b;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x, col0 = blockIdx.y * kRegWarps * Q;
    const int c0 = 2 * p, nc = min(2, cnt_child - c0);
    const int node = off_node + p;
    const int rows = nc * b;
    const int nr = nref[node];
    const T *Y = Ylev + (size_t)p * ystride;
    if (rows == 32 * R && ((uintptr_t)Y & 15) == 0) {
        // the node's reflectors fill whole 32R-row columns: one contiguous
        // block, copied in 16-byte pieces, 8 in flight per thread
        const uint4 *src = reinterpret_cast<const uint4 *>(Y);
        uint4 *dst = reinterpret_cast<uint4 *>(Vs);
        batched_copy<uint4, 8>(
            (int)(((size_t)nr * rows * sizeof(T)) / 16), threadIdx.x, blockDim.x, [&](int i) { return __ldg(src + i); },
            [&](int i, uint4 v) { dst[i] = v; });
    } else {
        batched_copy<T>(
            nr * 32 * R, threadIdx.x, blockDim.x,
            [&](int idx) {
                const int k = idx / (32 * R), r = idx % (32 * R);
                return r < rows ? Y[r + (size_t)k * rows] : T(0);
            },
            [&](int idx, T v) { Vs[idx] = v; });
    }
    for (int k = threadIdx.x; k < nr; k += blockDim.x) taus[k] = tau[(size_t)node * b + k];
    const T *Zn = Zbuf + (size_t)node * b * b;
    T m[Q][R], cm[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int c = col0 + warp + kRegWarps * q;
        cm[q] = c < b ? T(1) : T(0);
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int r = lane + 32 * t;
            T z = T(0);
            if (c < b && r < b) z = root_identity ? T(r == c ? 1 : 0) : Zn[r + (size_t)c * b];
            m[q][t] = z;
        }
    }
    __syncthreads();
    reg_apply_all<T, R, Q>(m, Vs, 32 * R, taus, nr, (b % 32 == 0 && nc == 2) ? b : 0, cm);
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int c = col0 + warp + kRegWarps * q, r = lane + 32 * t;
            if (c < b && r < rows)
                Zbuf[(size_t)(off_child + c0 + r / b) * b * b + r % b + (size_t)c * b] = m[q][t];
        }
}

// Leaf apply: the rows of the explicit thin Q owned by leaf l,
// Q_l = H_l [Z_l; 0], for columns [slice 16Q, slice 16Q + 16Q).
template <typename T, int R, int Q>
__global__ void __launch_bounds__(kRegThreads, 1)
    rtsqr_leaf_apply_kernel(int N, int b, int L, const T *__restrict__ Y, int ldy, const T *__restrict__ tau,
                            const int *__restrict__ nref, const T *__restrict__ Zbuf, T *__restrict__ Qout,
                            int ldq) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Vs = (T *)smem_raw;
    T *taus = Vs + (size_t)32 * R * b;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int l = blockIdx.x, col0 = blockIdx.y * kRegWarps * Q;
    const int row0 = rleaf_row0(N, L, l);
    const int rows = rleaf_row0(N, L, l + 1) - row0;
    const int nr = nref[l];
    batched_copy<T>(
        nr * 32 * R, threadIdx.x, blockDim.x,
        [&](int idx) {
            const int k = idx / (32 * R), r = idx % (32 * R);
            return r < rows ? Y[(size_t)(row0 + r) + (size_t)k * ldy] : T(0);
        },
        [&](int idx, T v) { Vs[idx] = v; });
    for (int k = threadIdx.x; k < nr; k += blockDim.x) taus[k] = tau[(size_t)l * b + k];
    const T *Zl = Zbuf + (size_t)l * b * b;
    T m[Q][R], cm[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int c = col0 + warp + kRegWarps * q;
        cm[q] = c < b ? T(1) : T(0);
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int r = lane + 32 * t;
            m[q][t] = (c < b && r < b) ? Zl[r + (size_t)c * b] : T(0);
        }
    }
    __syncthreads();
    reg_apply_all<T, R, Q>(m, Vs, 32 * R, taus, nr, 0, cm);
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int c = col0 + warp + kRegWarps * q, r = lane + 32 * t;
            if (c < b && r < rows) Qout[(size_t)(row0 + r) + (size_t)c * ldq] = m[q][t];
        }
}

// Reconstruction (single CTA; b <= 32R, b <= 16Q).  Reads Q1 = Q[0:b, 0:b]
// and the root R; writes U[0:b, :] (unit lower U1), T (b x b), W1^{-1} and
// the band block S R over the panel's top b rows (zeros below the diagonal).
template <typename T, int R, int Q>
__global__ void __launch_bounds__(kRegThreads, 1)
    recon_reg_kernel(int b, const T *__restrict__ Qm, int ldq, const T *__restrict__ Rroot, T *__restrict__ U,
                     int ldu, T *__restrict__ Tm, T *__restrict__ Winv, T *__restrict__ Apanel, int lda) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ld = b + 1;
    T *WS = (T *)smem_raw;            // W1 S (b x b, ld)
    T *Yi = WS + (size_t)ld * b;      // U1^{-1} (b x b, ld)
    T *cb = Yi + (size_t)ld * b;      // 2 x 32R column broadcast buffers
    T *Sg = cb + 2 * 32 * R;          // signs S_kk
    T *dg = Sg + b;                   // W1 diagonal
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T m[Q][R];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int c = warp + kRegWarps * q, r = lane + 32 * t;
            m[q][t] = (c < b && r < b) ? Qm[r + (size_t)c * ldq] : T(0);
        }
    // ---- LU of Q1 - S: step k scales column k below the pivot (the
    // multipliers, broadcast through cb), then every column c > k loses
    // l_i * m[k, c] in rows i > k
    for (int k = 0; k < b; ++k) {
        T *l = cb + (k & 1) * (32 * R);
        if (warp == k % kRegWarps) {
            const int qk = k / kRegWarps;
#pragma unroll
            for (int q = 0; q < Q; ++q)
                if (q == qk) {
                    const T v = __shfl_sync(0xffffffffu, rsel<R>(m[q], k >> 5), k & 31);
                    const T s = v < T(0) ? T(1) : T(-1);  // S_kk = -sgn(v), sgn(0) = +1
                    const T piv = v - s;
                    const T rp = T(1) / piv;  // |piv| >= 1
#pragma unroll
                    for (int t = 0; t < R; ++t) {
                        const int row = lane + 32 * t;
                        if (row == k) m[q][t] = piv;
                        if (row > k) m[q][t] *= rp;
                        l[row] = row > k ? m[q][t] : T(0);
                    }
                    if (lane == 0) {
                        Sg[k] = s;
                        dg[k] = piv;
                    }
                }
        }
        __syncthreads();
        // rows <= k have l = 0 and columns <= k a zero scale: every update is
        // an unconditional FMA (x - 0 * u leaves x unchanged)
        T lr[R];
#pragma unroll
        for (int t = 0; t < R; ++t) lr[t] = l[lane + 32 * t];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int c = warp + kRegWarps * q;
            const T u = __shfl_sync(0xffffffffu, rsel<R>(m[q], k >> 5), k & 31) * ((c > k && c < b) ? T(1) : T(0));
#pragma unroll
            for (int t = 0; t < R; ++t) m[q][t] = fmat(-lr[t], u, m[q][t]);
        }
    }
    __syncthreads();
    // U[0:b] = U1 (unit lower), W1 S into shared memory, band block S R
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int c = warp + kRegWarps * q, r = lane + 32 * t;
            if (c < b && r < b) {
                U[r + (size_t)c * ldu] = r < c ? T(0) : (r == c ? T(1) : m[q][t]);
                WS[r + (size_t)c * ld] = r <= c ? m[q][t] * Sg[c] : T(0);
            }
        }
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
        const int i = idx % b, c = idx / b;
        Apanel[i + (size_t)c * lda] = i <= c ? Sg[i] * Rroot[idx] : T(0);
    }
    // ---- W1^{-1} (upper) by back substitution, all columns at once: x = I;
    // for q = b-1 .. 0: row q of x is divided by W1[q, q], then rows i < q
    // lose W1[i, q] times it.  Column q of W1 is broadcast through cb.
    T x[Q][R];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) x[q][t] = (warp + kRegWarps * q == lane + 32 * t) ? T(1) : T(0);
    for (int qq = b - 1; qq >= 0; --qq) {
        T *w = cb + (qq & 1) * (32 * R);
        if (warp == qq % kRegWarps) {
            const int qk = qq / kRegWarps;
#pragma unroll
            for (int q = 0; q < Q; ++q)
                if (q == qk) {
#pragma unroll
                    for (int t = 0; t < R; ++t) {
                        const int row = lane + 32 * t;
                        w[row] = row < qq ? m[q][t] : T(0);
                    }
                }
        }
        __syncthreads();
        const T rdq = T(1) / dg[qq];
        T wr[R];
#pragma unroll
        for (int t = 0; t < R; ++t) wr[t] = w[lane + 32 * t];  // 0 on rows >= qq
        const int tq = qq >> 5;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            // columns c < qq have x[qq, c] = 0 and stay unchanged; row qq is scaled
            const T xq = __shfl_sync(0xffffffffu, rsel<R>(x[q], tq), qq & 31) * rdq;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                x[q][t] = fmat(-wr[t], xq, x[q][t]);
                if (t == tq && lane == (qq & 31)) x[q][t] = xq;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int c = warp + kRegWarps * q, r = lane + 32 * t;
            if (c < b && r < b) Winv[r + (size_t)c * b] = x[q][t];
        }
    // ---- U1^{-1} (unit lower) by forward substitution: y = I; for
    // q = 0 .. b-2: rows i > q lose U1[i, q] times row q (columns c <= q).
    __syncthreads();  // the broadcast buffers are read until the last sweep step ends
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) x[q][t] = (warp + kRegWarps * q == lane + 32 * t) ? T(1) : T(0);
    for (int qq = 0; qq + 1 < b; ++qq) {
        T *l = cb + (qq & 1) * (32 * R);
        if (warp == qq % kRegWarps) {
            const int qk = qq / kRegWarps;
#pragma unroll
            for (int q = 0; q < Q; ++q)
                if (q == qk) {
#pragma unroll
                    for (int t = 0; t < R; ++t) {
                        const int row = lane + 32 * t;
                        l[row] = row > qq ? m[q][t] : T(0);
                    }
                }
        }
        __syncthreads();
        T lr[R];
#pragma unroll
        for (int t = 0; t < R; ++t) lr[t] = l[lane + 32 * t];  // 0 on rows <= qq
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            // columns c > qq have y[qq, c] = 0: the update leaves them unchanged
            const T yq = __shfl_sync(0xffffffffu, rsel<R>(x[q], qq >> 5), qq & 31);
#pragma unroll
            for (int t = 0; t < R; ++t) x[q][t] = fmat(-lr[t], yq, x[q][t]);
        }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int c = warp + kRegWarps * q, r = lane + 32 * t;
            if (c < b && r < b) Yi[r + (size_t)c * ld] = x[q][t];
        }
    __syncthreads();
    // T = -(W1 S) U1^{-T} (upper: the product of two upper triangular factors)
    cta_gemm<T, false, true>(b, b, b, T(-1), WS, ld, Yi, ld, T(0), Tm, b);
}

// ---------------------------------------------------------------- driver
// (R, Q) by element type and panel width: rows per leaf <= 32R, b <= 16Q.
// FP32: 256-row leaves for every width up to 128; FP64: up to b = 64.
template <typename T>
int reg_panel_supported(int b) {
    if (b < 8) return 0;
    return sizeof(T) == 4 ? b <= 128 : b <= 64;
}

// Q, RR: columns per warp of the 16-warp kernels (applies, reconstruction);
// QW, NWQ: columns per warp and warps of the leaf and node QRs.
#ifndef SEV_QR128_QW
#define SEV_QR128_QW 16  // b = 128 FP32: 8 warps x 16 columns for the tree QR
#endif
template <typename T, int R, int Q, int RR, int QW = Q, int NWQ = kRegWarps>
static int reg_panel_run(sev_ctx *h, int N, int b, T *P, int lda, T *U, T *Tm, const RegPanelBufs<T> &B) {
    static_assert(NWQ * QW == kRegWarps * Q, "the QR kernels hold the same columns");
    // leaves: as many as 256-row blocks need (each >= b rows when there are
    // two or more), or rows of about SEV_LEAF_ROWS (tests: deep trees)
    int L = (N + 32 * R - 1) / (32 * R);
    if (h->leaf_rows_override > 0) {
        const int ov = h->leaf_rows_override < b ? b : h->leaf_rows_override;
        const int Lo = N / ov;
        if (Lo > L) L = Lo;
    }
    if (L > 1 && N / L < b) L = N / b;
    if (L < 1) L = 1;
    if (L == 1) {
        // one leaf: its Householder QR already is (U, T); T by the forward recurrence
        SEV_LAUNCH(h, K_TSQR_LEAF, (rtsqr_leaf_qr_kernel<T, R, QW, NWQ>), 1, NWQ * 32, 0, P, lda, N, b, 1, U, N, B.tau,
                   B.nref, B.Rbuf);
        return panel_finish_single_leaf<T>(h, N, b, U, B.tau, B.nref, B.Rbuf, Tm, P, lda);
    }
    SEV_LAUNCH(h, K_TSQR_LEAF, (rtsqr_leaf_qr_kernel<T, R, QW, NWQ>), L, NWQ * 32, 0, P, lda, N, b, L, B.Yleaf, N, B.tau,
               B.nref, B.Rbuf);
    int cnt[32], off[32], nlev = 0;
    for (int c = L, o = 0;; c = (c + 1) / 2) {
        cnt[nlev] = c;
        off[nlev] = o;
        o += c;
        ++nlev;
        if (c == 1) break;
    }
    const size_t ystride = (size_t)2 * b * b;
    for (int lev = 1; lev < nlev; ++lev) {
        T *Ylev = B.Ynode + (size_t)(off[lev] - L) * ystride;
        SEV_LAUNCH(h, K_TSQR_TREE, (rtsqr_node_qr_kernel<T, R, QW, NWQ>), cnt[lev], NWQ * 32, 0, b, cnt[lev - 1],
                   off[lev - 1], off[lev], B.Rbuf, Ylev, ystride, B.tau, B.nref);
    }
    // the way down: the upper levels have few nodes, so 32-column slices
    // (more CTAs); the leaves are many, so 64-column slices (V loaded fewer times)
    constexpr int QN = 2, QL = 4;
    const int slices_n = (b + kRegWarps * QN - 1) / (kRegWarps * QN);
    const int slices_l = (b + kRegWarps * QL - 1) / (kRegWarps * QL);
    const size_t s_apply = sizeof(T) * ((size_t)32 * R * b + b);
    SEV_CUDA(cudaFuncSetAttribute(rtsqr_node_apply_kernel<T, R, QN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)s_apply));
    SEV_CUDA(cudaFuncSetAttribute(rtsqr_leaf_apply_kernel<T, R, QL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)s_apply));
    for (int lev = nlev - 1; lev >= 1; --lev) {
        T *Ylev = B.Ynode + (size_t)(off[lev] - L) * ystride;
        SEV_LAUNCH(h, K_TSQR_DOWN, (rtsqr_node_apply_kernel<T, R, QN>), dim3(cnt[lev], slices_n), kRegThreads,
                   s_apply, b, cnt[lev - 1], off[lev - 1], off[lev], Ylev, ystride, B.tau, B.nref, B.Zbuf,
                   lev == nlev - 1 ? 1 : 0);
    }
    SEV_LAUNCH(h, K_TSQR_LEAF_Q, (rtsqr_leaf_apply_kernel<T, R, QL>), dim3(L, slices_l), kRegThreads, s_apply, N, b,
               L, B.Yleaf, N, B.tau, B.nref, B.Zbuf, B.Q, N);
    const T *Rroot = B.Rbuf + (size_t)(off[nlev - 1]) * b * b;
    const size_t s_rec = sizeof(T) * (2 * (size_t)(b + 1) * b + 2 * 32 * RR + 2 * b);
    SEV_CUDA(cudaFuncSetAttribute(recon_reg_kernel<T, RR, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_rec));
    SEV_LAUNCH(h, K_RECON_LU, (recon_reg_kernel<T, RR, Q>), 1, kRegThreads, s_rec, b, B.Q, N, Rroot, U, N, Tm, B.Winv,
               P, lda);
    return panel_form_u2<T>(h, N, b, B.Q, B.Winv, U, P, lda);
}

template <typename T>
int reg_panel_factor(sev_ctx *h, int N, int b, T *P, int lda, T *U, T *Tm, const RegPanelBufs<T> &B) {
    if constexpr (sizeof(T) == 4) {  // FP32: the QRs on 8 warps (twice the columns each)
        if (b <= 32) return reg_panel_run<T, 8, 2, 1, 4, 8>(h, N, b, P, lda, U, Tm, B);
        if (b <= 64) return reg_panel_run<T, 8, 4, 2, 8, 8>(h, N, b, P, lda, U, Tm, B);
    } else {
        if (b <= 32) return reg_panel_run<T, 8, 2, 1>(h, N, b, P, lda, U, Tm, B);
        if (b <= 64) return reg_panel_run<T, 8, 4, 2>(h, N, b, P, lda, U, Tm, B);
    }
    if constexpr (sizeof(T) == 4) return reg_panel_run<T, 8, 8, 4, SEV_QR128_QW, 128 / SEV_QR128_QW>(h, N, b, P, lda, U, Tm, B);
    return SEV_ERR_UNSUPPORTED;
}

template int reg_panel_supported<float>(int);
template int reg_panel_supported<double>(int);
template int reg_panel_factor<float>(sev_ctx *, int, int, float *, int, float *, float *, const RegPanelBufs<float> &);
template int reg_panel_factor<double>(sev_ctx *, int, int, double *, int, double *, double *,
                                      const RegPanelBufs<double> &);

}  // namespace sev
