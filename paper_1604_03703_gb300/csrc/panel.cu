// panel.cu -- QR of the N x b trailing panel of the full-to-band reduction
// (the QR step of Algorithm 4.1) as a tree of small QRs over row blocks
// (Algorithm 3.2), then the compact-WY form (U, T) of its Q by Householder
// reconstruction (Cor. 3.7).
//
// Tree QR.  The panel's rows are split into L leaves of at least r_leaf rows
// (the last leaf takes the remainder).  Leaf l is QR'd in one CTA:
// A_l = W_l R_l (blocked Householder QR, cta_qr_blocked, keeping the
// compact-WY factor of every 32-column block for the way down).  Going up, a node stacks the R's of its (up to F) children
// and QRs the stack: [R_c0; ...; R_ck] = Z R.  Going down (Algorithm 3.2's
// Q_i = W_i Z_i), a node's Z block is pushed through its reflectors,
// [Z; 0] -> H [Z; 0], and the row blocks of the result are its children's
// Z blocks; at a leaf, Q_l = H_l [Z_l; 0] gives the rows of the explicit
// thin Q.  The root's Z is the identity.  Both pushes apply the reflectors
// a block at a time, M <- M - V (T (V^T M)) (cta_apply_blocked).
//
// Reconstruction (Cor. 3.7).  Q1 - S = U1 W1 (unpivoted LU, U1 unit lower,
// W1 upper) with S a diagonal sign matrix chosen during the LU: at step k,
// S_kk = -sgn(current pivot), sgn(0) = +1, so every pivot has magnitude
// >= 1.  Then U = [U1; Q2 W1^{-1}], T = -W1 S U1^{-T} and
// (I - U T U^T)[:, 0:b] = Q S, so the band block is S R.  This S makes each
// tau lie in [1, 2], the same reflectors a column-by-column Householder QR
// with beta = -sgn(alpha)||x|| produces.
//
// A panel with a single leaf skips the tree: its Householder QR already is
// (U, T) (T by the forward recurrence).
#include "common.cuh"

namespace sev {

// ------------------------------------------------------------- tree layout
struct TreePlan {
    int N = 0, b = 0, r_leaf = 0, L = 0, F = 2, cs = 1;
    int nlev = 0;              // number of levels incl. the leaf level
    int cnt[32] = {};          // nodes per level
    int off[32] = {};          // first flat node id of each level
    int total = 0;             // total nodes
    size_t ynode_stride = 0;   // elements per internal-node Y slot (F b x b)
};

static int col_slices(int b) { return b >= 64 && b % 32 == 0 ? b / 32 : 1; }  // apply slices of 32 columns

template <typename T>
static size_t smem_leaf_qr(int r_leaf, int b);
template <typename T>
static size_t smem_leaf_apply(int r_leaf, int b, int cs);

// Rows per leaf: the largest multiple of 32 (>= b, <= 1024) whose leaf QR
// and leaf apply both fit the shared-memory budget.
template <typename T>
static int pick_r_leaf(int b, size_t budget) {
    int best = b;
    for (int r = 32; r <= 1024; r += 32) {
        if (r < b) continue;
        if (smem_leaf_qr<T>(r, b) <= budget && smem_leaf_apply<T>(r, b, col_slices(b)) <= budget) best = r;
    }
    return best;
}

static void make_plan(TreePlan &p, int N, int b, int r_leaf, int F) {
    p.N = N;
    p.b = b;
    p.r_leaf = r_leaf;
    p.F = F;
    p.L = N / r_leaf;
    if (p.L < 1) p.L = 1;
    p.nlev = 0;
    int c = p.L, o = 0;
    for (;;) {
        p.cnt[p.nlev] = c;
        p.off[p.nlev] = o;
        o += c;
        ++p.nlev;
        if (c == 1) break;
        c = (c + F - 1) / F;
    }
    p.total = o;
    p.ynode_stride = (size_t)F * b * b;
    p.cs = col_slices(b);
}

__host__ __device__ __forceinline__ int leaf_rows(int N, int r_leaf, int L, int l) {
    return l == L - 1 ? N - l * r_leaf : r_leaf;
}

// --------------------------------------------------------- QR kernels (up)
// Leaf QR: CTA l factorises panel rows [l r_leaf, l r_leaf + rows_l).
// Writes Y (explicit unit lower trapezoidal, rows_l x b) into Yleaf at the
// leaf's row offset, tau, nref and R (b x b, upper; rows >= rows_l zero).
template <typename T>
__global__ void __launch_bounds__(kThreads)
    tsqr_leaf_qr_kernel(const T *__restrict__ P, int ldp, int N, int b, int r_leaf, int L, T *__restrict__ Yleaf,
                        int ldy, T *__restrict__ tau, int *__restrict__ nref, T *__restrict__ Rbuf,
                        T *__restrict__ Tbuf) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int l = blockIdx.x;
    const int row0 = l * r_leaf;
    const int rows = leaf_rows(N, r_leaf, L, l);
    const int ld = (2 * r_leaf) | 1;
    T *S = (T *)smem;
    T *tl = S + (size_t)ld * b;
    T *Tblk = tl + b;
    T *Wk = Tblk + (size_t)kQrNB * b;
    T *Gb = Wk + (size_t)kQrNB * b;
    T *Rs = Gb + kQrNB * kQrNB;
    batched_copy<T>(
        rows * b, threadIdx.x, blockDim.x, [&](int k) { return P[(size_t)(row0 + k % rows) + (size_t)(k / rows) * ldp]; },
        [&](int k, T v) { S[k % rows + (size_t)(k / rows) * ld] = v; });
    __syncthreads();
    const int r = cta_qr_blocked(rows, b, S, ld, tl, Tblk, Wk, Gb, Rs);
    for (int idx = threadIdx.x; idx < rows * b; idx += blockDim.x) {
        const int i = idx % rows, c = idx / rows;
        T v = 0;
        if (c < r) v = (i < c) ? T(0) : (i == c ? T(1) : S[i + (size_t)c * ld]);
        Yleaf[(size_t)(row0 + i) + (size_t)c * ldy] = v;
    }
    for (int idx = threadIdx.x; idx < kQrNB * b; idx += blockDim.x) Tbuf[(size_t)l * kQrNB * b + idx] = Tblk[idx];
    T *R = Rbuf + (size_t)l * b * b;
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
        const int i = idx % b, c = idx / b;
        R[idx] = (i <= c && i < rows) ? S[i + (size_t)c * ld] : T(0);
    }
    for (int c = threadIdx.x; c < b; c += blockDim.x) tau[(size_t)l * b + c] = c < r ? tl[c] : T(0);
    if (threadIdx.x == 0) nref[l] = r;
}

// Internal node QR: CTA p of level lev stacks the R's of its children.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    tsqr_node_qr_kernel(int b, int F, int cnt_child, int off_child, int off_node, T *__restrict__ Rbuf,
                        T *__restrict__ Ynode, size_t ynode_stride, T *__restrict__ tau, int *__restrict__ nref,
                        T *__restrict__ Tbuf) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int p = blockIdx.x;
    const int c0 = F * p, c1 = min(F * p + F, cnt_child);
    const int nc = c1 - c0;
    const int node = off_node + p;
    T *Rn = Rbuf + (size_t)node * b * b;
    if (nc == 1) {  // pass-through
        const T *Rc = Rbuf + (size_t)(off_child + c0) * b * b;
        for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) Rn[idx] = Rc[idx];
        if (threadIdx.x == 0) nref[node] = 0;
        return;
    }
    const int rows = nc * b;
    const int ld = (F * b) | 1;
    T *S = (T *)smem;
    T *tl = S + (size_t)ld * b;
    T *Tblk = tl + b;
    T *Wk = Tblk + (size_t)kQrNB * b;
    T *Gb = Wk + (size_t)kQrNB * b;
    T *Rs = Gb + kQrNB * kQrNB;
    batched_copy<T>(
        rows * b, threadIdx.x, blockDim.x,
        [&](int k) {
            const int r = k % rows, c = k / rows;
            return Rbuf[(size_t)(off_child + c0 + r / b) * b * b + r % b + (size_t)c * b];
        },
        [&](int k, T v) { S[k % rows + (size_t)(k / rows) * ld] = v; });
    __syncthreads();
    const int r = cta_qr_blocked(rows, b, S, ld, tl, Tblk, Wk, Gb, Rs);
    T *Y = Ynode + (size_t)p * ynode_stride;
    for (int idx = threadIdx.x; idx < kQrNB * b; idx += blockDim.x) Tbuf[(size_t)node * kQrNB * b + idx] = Tblk[idx];
    for (int idx = threadIdx.x; idx < rows * b; idx += blockDim.x) {
        const int i = idx % rows, c = idx / rows;
        T v = 0;
        if (c < r) v = (i < c) ? T(0) : (i == c ? T(1) : S[i + (size_t)c * ld]);
        Y[i + (size_t)c * rows] = v;
    }
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
        const int i = idx % b, c = idx / b;
        Rn[idx] = (i <= c) ? S[i + (size_t)c * ld] : T(0);
    }
    for (int c = threadIdx.x; c < b; c += blockDim.x) tau[(size_t)node * b + c] = c < r ? tl[c] : T(0);
    if (threadIdx.x == 0) nref[node] = r;
}

// ------------------------------------------------------- apply kernels (down)
// Node level: CTA (p, slice) pushes the node's Z (columns of the slice)
// through its reflectors and scatters the row blocks to the children's Z.
// Z_root (lev = top) is the identity when root_identity != 0.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    tsqr_node_apply_kernel(int b, int F, int cs, int cnt_child, int off_child, int off_node, const T *__restrict__ Ynode,
                           size_t ynode_stride, const T *__restrict__ tau, const int *__restrict__ nref,
                           T *__restrict__ Zbuf, int root_identity, const T *__restrict__ Tbuf) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int p = blockIdx.x, slice = blockIdx.y;
    const int w = b / cs, col0 = slice * w;
    const int c0 = F * p, c1 = min(F * p + F, cnt_child);
    const int nc = c1 - c0;
    const int node = off_node + p;
    const T *Zn = Zbuf + (size_t)node * b * b;
    const int rows = nc * b;
    const int ld = (F * b) | 1;
    T *Ys = (T *)smem;
    T *Ms = Ys + (size_t)ld * b;
    T *tl = Ms + (size_t)ld * w;
    T *Tblk = tl + b;
    T *Wk = Tblk + (size_t)kQrNB * b;
    const int nr = nref[node];
    batched_copy<T>(
        rows * w, threadIdx.x, blockDim.x,
        [&](int k) {
            const int r = k % rows, c = k / rows;
            T z = 0;
            if (r < b) z = root_identity ? T(r == col0 + c ? 1 : 0) : Zn[r + (size_t)(col0 + c) * b];
            return z;
        },
        [&](int k, T v) { Ms[k % rows + (size_t)(k / rows) * ld] = v; });
    if (nr > 0) {
        const T *Y = Ynode + (size_t)p * ynode_stride;
        batched_copy<T>(
            rows * nr, threadIdx.x, blockDim.x, [&](int k) { return Y[k]; },
            [&](int k, T v) { Ys[k % rows + (size_t)(k / rows) * ld] = v; });
        for (int idx = threadIdx.x; idx < kQrNB * nr; idx += blockDim.x)
            Tblk[idx] = Tbuf[(size_t)node * kQrNB * b + idx];
    }
    __syncthreads();
    if (nr > 0) cta_apply_blocked(rows, w, nr, Ys, ld, Tblk, Ms, Wk);
    for (int idx = threadIdx.x; idx < rows * w; idx += blockDim.x) {
        const int r = idx % rows, c = idx / rows;
        const int k = r / b, rr = r % b;
        Zbuf[(size_t)(off_child + c0 + k) * b * b + rr + (size_t)(col0 + c) * b] = Ms[r + (size_t)c * ld];
    }
}

// Leaf level: Q_l = H_l [Z_l; 0] written to the explicit Q (N x b, ldq).
template <typename T>
__global__ void __launch_bounds__(kThreads)
    tsqr_leaf_apply_kernel(int N, int b, int r_leaf, int L, int cs, const T *__restrict__ Yleaf, int ldy,
                           const T *__restrict__ tau, const int *__restrict__ nref, const T *__restrict__ Zbuf,
                           T *__restrict__ Q, int ldq, const T *__restrict__ Tbuf) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int l = blockIdx.x, slice = blockIdx.y;
    const int w = b / cs, col0 = slice * w;
    const int row0 = l * r_leaf;
    const int rows = leaf_rows(N, r_leaf, L, l);
    const int ld = (2 * r_leaf) | 1;
    T *Ys = (T *)smem;
    T *Ms = Ys + (size_t)ld * b;
    T *tl = Ms + (size_t)ld * w;
    T *Tblk = tl + b;
    T *Wk = Tblk + (size_t)kQrNB * b;
    const int nr = nref[l];
    const T *Zl = Zbuf + (size_t)l * b * b;
    batched_copy<T>(
        rows * w, threadIdx.x, blockDim.x,
        [&](int k) {
            const int r = k % rows, c = k / rows;
            return r < b ? Zl[r + (size_t)(col0 + c) * b] : T(0);
        },
        [&](int k, T v) { Ms[k % rows + (size_t)(k / rows) * ld] = v; });
    batched_copy<T>(
        rows * nr, threadIdx.x, blockDim.x,
        [&](int k) { return Yleaf[(size_t)(row0 + k % rows) + (size_t)(k / rows) * ldy]; },
        [&](int k, T v) { Ys[k % rows + (size_t)(k / rows) * ld] = v; });
    for (int idx = threadIdx.x; idx < kQrNB * nr; idx += blockDim.x) Tblk[idx] = Tbuf[(size_t)l * kQrNB * b + idx];
    __syncthreads();
    cta_apply_blocked(rows, w, nr, Ys, ld, Tblk, Ms, Wk);
    for (int idx = threadIdx.x; idx < rows * w; idx += blockDim.x) {
        const int r = idx % rows, c = idx / rows;
        Q[(size_t)(row0 + r) + (size_t)(col0 + c) * ldq] = Ms[r + (size_t)c * ld];
    }
}

// ------------------------------------------------------------ reconstruction
// Single CTA.  Reads Q1 = Q[0:b, 0:b] and the root R; writes U[0:b, :]
// (unit lower), T (b x b), W1^{-1} (b x b, for U2 = Q2 W1^{-1}) and the band
// block S R into the panel's top b rows of A (zeros below the diagonal).
template <typename T>
__global__ void __launch_bounds__(kThreads)
    recon_lu_kernel(int b, const T *__restrict__ Q, int ldq, const T *__restrict__ Rroot, T *__restrict__ U, int ldu,
                    T *__restrict__ Tm, T *__restrict__ Winv, T *__restrict__ Apanel, int lda) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = b + 1;
    T *M = (T *)smem;                 // LU in place: U1 strictly lower, W1 upper
    T *Inv = M + (size_t)ld * b;      // W1^{-1}, then U1^{-1}
    T *WS = Inv + (size_t)ld * b;     // W1 S
    T *Sg = WS + (size_t)ld * b;      // signs
    batched_copy<T>(
        b * b, threadIdx.x, blockDim.x, [&](int k) { return Q[k % b + (size_t)(k / b) * ldq]; },
        [&](int k, T v) { M[k % b + (size_t)(k / b) * ld] = v; });
    __syncthreads();
    for (int k = 0; k < b; ++k) {
        if (threadIdx.x == 0) {
            const T v = M[k + (size_t)k * ld];
            const T s = v < T(0) ? T(1) : T(-1);  // S_kk = -sgn(v), sgn(0) = +1
            Sg[k] = s;
            M[k + (size_t)k * ld] = v - s;
        }
        __syncthreads();
        const T rpiv = T(1) / M[k + (size_t)k * ld];  // |pivot| >= 1 by the choice of S
        for (int i = k + 1 + threadIdx.x; i < b; i += blockDim.x) M[i + (size_t)k * ld] *= rpiv;
        __syncthreads();
        const int m = b - k - 1;
        for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
            const int i = k + 1 + idx % m, c = k + 1 + idx / m;
            M[i + (size_t)c * ld] -= M[i + (size_t)k * ld] * M[k + (size_t)c * ld];
        }
        __syncthreads();
    }
    // W1^{-1} (upper) by column-sweep back substitution, all columns at once:
    // Inv = I; for q = b-1 .. 0: row q /= W1[q,q], then rows i < q lose
    // W1[i,q] times row q (columns c >= q).
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
        const int i = idx % b, c = idx / b;
        Inv[i + (size_t)c * ld] = i == c ? T(1) : T(0);
    }
    __syncthreads();
    for (int q = b - 1; q >= 0; --q) {
        const T piv = M[q + (size_t)q * ld];
        for (int c = q + threadIdx.x; c < b; c += blockDim.x) Inv[q + (size_t)c * ld] /= piv;
        __syncthreads();
        const int w = b - q;
        for (int idx = threadIdx.x; idx < q * w; idx += blockDim.x) {
            const int i = idx % q, c = q + idx / q;
            Inv[i + (size_t)c * ld] -= M[i + (size_t)q * ld] * Inv[q + (size_t)c * ld];
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) Winv[idx] = Inv[idx % b + (size_t)(idx / b) * ld];
    // U[0:b, :] = U1 (unit lower); W1 S (upper, zeros below) into WS
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
        const int i = idx % b, c = idx / b;
        U[i + (size_t)c * ldu] = i < c ? T(0) : (i == c ? T(1) : M[i + (size_t)c * ld]);
        WS[i + (size_t)c * ld] = i <= c ? M[i + (size_t)c * ld] * Sg[c] : T(0);
    }
    // band block S R (rows scaled by S), zeros below the diagonal
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
        const int i = idx % b, c = idx / b;
        Apanel[i + (size_t)c * lda] = i <= c ? Sg[i] * Rroot[idx] : T(0);
    }
    __syncthreads();
    // U1^{-1} (unit lower) by column-sweep forward substitution: Inv = I; for
    // q = 0 .. b-1: rows i > q lose U1[i,q] times row q (columns c <= q).
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
        const int i = idx % b, c = idx / b;
        Inv[i + (size_t)c * ld] = i == c ? T(1) : T(0);
    }
    __syncthreads();
    for (int q = 0; q < b - 1; ++q) {
        const int h = b - 1 - q, w = q + 1;
        for (int idx = threadIdx.x; idx < h * w; idx += blockDim.x) {
            const int i = q + 1 + idx % h, c = idx / h;
            Inv[i + (size_t)c * ld] -= M[i + (size_t)q * ld] * Inv[q + (size_t)c * ld];
        }
        __syncthreads();
    }
    // T = -(W1 S) U1^{-T} (upper: the product of the two triangular factors)
    cta_gemm<T, false, true>(b, b, b, T(-1), WS, ld, Inv, ld, T(0), Tm, b);
}

// U[b:N, :] = Q[b:N, :] W1^{-1}; also zeroes the panel of A below its top b
// rows (those entries are outside the band after the reduction).
template <typename T>
__global__ void __launch_bounds__(kThreads)
    recon_u2_kernel(int N, int b, const T *__restrict__ Q, int ldq, const T *__restrict__ Winv, T *__restrict__ U,
                    int ldu, T *__restrict__ Apanel, int lda) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = b + 1;
    T *Wi = (T *)smem;
    batched_copy<T>(
        b * b, threadIdx.x, blockDim.x, [&](int k) { return Winv[k]; },
        [&](int k, T v) { Wi[k % b + (size_t)(k / b) * ld] = v; });
    __syncthreads();
    const int rows_per = 64;
    const int r0 = b + blockIdx.x * rows_per;
    for (int idx = threadIdx.x; idx < rows_per * b; idx += blockDim.x) {
        const int r = r0 + idx % rows_per, c = idx / rows_per;
        if (r >= N) continue;
        T s = 0;
        for (int q = 0; q <= c; ++q) s += Q[r + (size_t)q * ldq] * Wi[q + (size_t)c * ld];
        U[r + (size_t)c * ldu] = s;
        Apanel[r + (size_t)c * lda] = T(0);
    }
}

// Single-leaf panels: T by the forward recurrence from the explicit Y (= U),
// R into the panel's top rows, zeros below.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    single_leaf_finish_kernel(int N, int b, const T *__restrict__ U, int ldu, const T *__restrict__ tau,
                              const int *__restrict__ nref, const T *__restrict__ R, T *__restrict__ Tm,
                              T *__restrict__ Apanel, int lda) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = b + 1;
    T *G = (T *)smem;
    T *Ts = G + (size_t)ld * b;
    const int r = nref[0];
    // G = U^T U (strict upper part)
    for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
        const int a = idx % r, c = idx / r;
        if (a >= c) continue;
        T s = 0;
        for (int i = c; i < N; ++i) s += U[i + (size_t)a * ldu] * U[i + (size_t)c * ldu];
        G[a + (size_t)c * ld] = s;
    }
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
        const int a = idx % b, c = idx / b;
        Ts[a + (size_t)c * ld] = (a == c && c < r) ? tau[c] : T(0);
    }
    __syncthreads();
    for (int k = 1; k < r; ++k) {
        for (int a = threadIdx.x; a < k; a += blockDim.x) {
            T s = 0;
            for (int q = a; q < k; ++q) s += Ts[a + (size_t)q * ld] * G[q + (size_t)k * ld];
            Ts[a + (size_t)k * ld] = -tau[k] * s;
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) Tm[idx] = Ts[idx % b + (size_t)(idx / b) * ld];
    for (long idx = threadIdx.x; idx < (long)N * b; idx += blockDim.x) {
        const int i = (int)(idx % N), c = (int)(idx / N);
        T v = 0;
        if (i < b && i <= c) v = R[i + (size_t)c * b];
        Apanel[i + (size_t)c * lda] = v;
    }
}

// ---------------------------------------------------------------- driver
template <typename T>
static size_t smem_leaf_qr(int r_leaf, int b) {
    // block, tau, T blocks, GEMM scratch, R save, reduction scratch
    return sizeof(T) * ((size_t)((2 * r_leaf) | 1) * b + b + 2 * (size_t)kQrNB * b + 2 * kQrNB * kQrNB) + 16 +
           32 * sizeof(double);
}
template <typename T>
static size_t smem_node_qr(int F, int b) {
    return sizeof(T) * ((size_t)((F * b) | 1) * b + b + 2 * (size_t)kQrNB * b + 2 * kQrNB * kQrNB) + 16 +
           32 * sizeof(double);
}
template <typename T>
static size_t smem_leaf_apply(int r_leaf, int b, int cs) {
    const size_t ld = (2 * r_leaf) | 1, w = b / cs;
    return sizeof(T) * (ld * b + ld * w + b + (size_t)kQrNB * b + kQrNB * w);
}
template <typename T>
static size_t smem_node_apply(int F, int b, int cs) {
    const size_t ld = (F * b) | 1, w = b / cs;
    return sizeof(T) * (ld * b + ld * w + b + (size_t)kQrNB * b + kQrNB * w);
}

struct PanelWs {
    void *base;
};

template <typename T>
struct PanelBuffers {
    T *Yleaf, *Ynode, *tau, *Rbuf, *Zbuf, *Q, *Winv, *Tbuf;
    int *nref;
};

template <typename T>
static void carve_panel(Carver &c, PanelBuffers<T> &B, int n, int b, int r_leaf, int F) {
    const int Lmax = n / r_leaf + 1;
    const int nodes = 2 * Lmax + 64;
    B.Yleaf = c.take<T>((size_t)n * b);
    B.Ynode = c.take<T>((size_t)(Lmax + 64) * F * b * b);
    B.tau = c.take<T>((size_t)nodes * b);
    B.Rbuf = c.take<T>((size_t)nodes * b * b);
    B.Zbuf = c.take<T>((size_t)nodes * b * b);
    B.Q = c.take<T>((size_t)n * b);
    B.Winv = c.take<T>((size_t)b * b);
    B.Tbuf = c.take<T>((size_t)nodes * kQrNB * b);
    B.nref = c.take<int>((size_t)nodes);
}

// Register path: leaves of at least b rows, binary tree.
template <typename T>
static void carve_reg_panel(Carver &c, RegPanelBufs<T> &B, int n, int b) {
    const int Lmax = n / b + 1;
    const int nodes = 2 * Lmax + 64;
    B.Yleaf = c.take<T>((size_t)n * b);
    B.Ynode = c.take<T>((size_t)(Lmax + 64) * 2 * b * b);
    B.tau = c.take<T>((size_t)nodes * b);
    B.Rbuf = c.take<T>((size_t)nodes * b * b);
    B.Zbuf = c.take<T>((size_t)nodes * b * b);
    B.Q = c.take<T>((size_t)n * b);
    B.Winv = c.take<T>((size_t)b * b);
    B.nref = c.take<int>((size_t)nodes);
}

template <typename T>
size_t panel_workspace(sev_ctx *h, int n, int b) {
    Carver c(nullptr);
    PanelBuffers<T> B;
    carve_panel<T>(c, B, n, b, pick_r_leaf<T>(b, (size_t)h->smem_optin - 1024), 2);
    Carver c2(nullptr);
    RegPanelBufs<T> B2;
    carve_reg_panel<T>(c2, B2, n, b);
    return c.bytes() > c2.bytes() ? c.bytes() : c2.bytes();
}

template <typename T>
int panel_finish_single_leaf(sev_ctx *h, int N, int b, const T *U, const T *tau, const int *nref, const T *R, T *Tm,
                             T *P, int lda) {
    const size_t s_fin = sizeof(T) * 2 * (size_t)(b + 1) * b;
    SEV_CUDA(cudaFuncSetAttribute(single_leaf_finish_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)s_fin));
    SEV_LAUNCH(h, K_RECON_LU, single_leaf_finish_kernel<T>, 1, kThreads, s_fin, N, b, U, N, tau, nref, R, Tm, P, lda);
    return SEV_OK;
}

template <typename T>
int panel_form_u2(sev_ctx *h, int N, int b, const T *Q, const T *Winv, T *U, T *P, int lda) {
    const size_t s_u2 = sizeof(T) * (size_t)(b + 1) * b;
    SEV_CUDA(cudaFuncSetAttribute(recon_u2_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_u2));
    const int g2 = (N - b + 63) / 64;
    if (g2 > 0) SEV_LAUNCH(h, K_RECON_U2, recon_u2_kernel<T>, g2, kThreads, s_u2, N, b, Q, N, Winv, U, N, P, lda);
    return SEV_OK;
}

// Factorise the N x b panel P (lda) and produce U (N x b, ldu = N), T (b x b)
// and the band block (written over the panel in A).
template <typename T>
int panel_factor(sev_ctx *h, int N, int b, T *P, int lda, T *U, T *Tm, void *ws) {
    if (reg_panel_supported<T>(b)) {
        Carver c(ws);
        RegPanelBufs<T> B;
        carve_reg_panel<T>(c, B, N, b);
        return reg_panel_factor<T>(h, N, b, P, lda, U, Tm, B);
    }
    const size_t budget = (size_t)h->smem_optin - 1024;
    int r_leaf = pick_r_leaf<T>(b, budget);
    if (h->leaf_rows_override > 0) {
        r_leaf = h->leaf_rows_override < r_leaf ? h->leaf_rows_override : r_leaf;
        if (r_leaf < b) r_leaf = b;
    }
    const int F = 2;
    TreePlan plan;
    make_plan(plan, N, b, r_leaf, F);
    Carver c(ws);
    PanelBuffers<T> B;
    carve_panel<T>(c, B, N, b, r_leaf, F);
    const int cs = plan.cs;
    if (smem_leaf_qr<T>(r_leaf, b) > h->smem_optin || smem_node_qr<T>(F, b) > h->smem_optin ||
        smem_leaf_apply<T>(r_leaf, b, cs) > h->smem_optin || smem_node_apply<T>(F, b, cs) > h->smem_optin ||
        sizeof(T) * (3 * (size_t)(b + 1) * b + b) > h->smem_optin)
        return SEV_ERR_UNSUPPORTED;

    const size_t s_leaf = smem_leaf_qr<T>(r_leaf, b);
    SEV_CUDA(cudaFuncSetAttribute(tsqr_leaf_qr_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_leaf));
    if (plan.L == 1) {
        // single leaf: Householder QR of the whole panel gives (U, T) directly
        SEV_LAUNCH(h, K_TSQR_LEAF, tsqr_leaf_qr_kernel<T>, 1, kThreads, s_leaf, P, lda, N, b, r_leaf, 1, U, N, B.tau,
                   B.nref, B.Rbuf, B.Tbuf);
        const size_t s_fin = sizeof(T) * 2 * (size_t)(b + 1) * b;
        SEV_CUDA(cudaFuncSetAttribute(single_leaf_finish_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)s_fin));
        SEV_LAUNCH(h, K_RECON_LU, single_leaf_finish_kernel<T>, 1, kThreads, s_fin, N, b, U, N, B.tau, B.nref, B.Rbuf,
                   Tm, P, lda);
        return SEV_OK;
    }
    SEV_LAUNCH(h, K_TSQR_LEAF, tsqr_leaf_qr_kernel<T>, plan.L, kThreads, s_leaf, P, lda, N, b, r_leaf, plan.L,
               B.Yleaf, N, B.tau, B.nref, B.Rbuf, B.Tbuf);
    // up the tree
    const size_t s_node = smem_node_qr<T>(F, b);
    SEV_CUDA(cudaFuncSetAttribute(tsqr_node_qr_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_node));
    for (int lev = 1; lev < plan.nlev; ++lev) {
        // internal-node Y slots are indexed by the node's position in its level
        // level by level; reuse one slot array per level (levels run in order
        // and the down-sweep needs every level, so give each level its own)
        T *Ylev = B.Ynode + (size_t)(plan.off[lev] - plan.L) * plan.ynode_stride;
        SEV_LAUNCH(h, K_TSQR_TREE, tsqr_node_qr_kernel<T>, plan.cnt[lev], kThreads, s_node, b, F, plan.cnt[lev - 1],
                   plan.off[lev - 1], plan.off[lev], B.Rbuf, Ylev, plan.ynode_stride, B.tau, B.nref, B.Tbuf);
    }
    // down the tree
    const size_t s_napply = smem_node_apply<T>(F, b, cs);
    SEV_CUDA(
        cudaFuncSetAttribute(tsqr_node_apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_napply));
    for (int lev = plan.nlev - 1; lev >= 1; --lev) {
        T *Ylev = B.Ynode + (size_t)(plan.off[lev] - plan.L) * plan.ynode_stride;
        dim3 grid(plan.cnt[lev], cs);
        SEV_LAUNCH(h, K_TSQR_DOWN, tsqr_node_apply_kernel<T>, grid, kThreads, s_napply, b, F, cs, plan.cnt[lev - 1],
                   plan.off[lev - 1], plan.off[lev], Ylev, plan.ynode_stride, B.tau, B.nref, B.Zbuf,
                   lev == plan.nlev - 1 ? 1 : 0, B.Tbuf);
    }
    const size_t s_lapply = smem_leaf_apply<T>(r_leaf, b, cs);
    SEV_CUDA(
        cudaFuncSetAttribute(tsqr_leaf_apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_lapply));
    SEV_LAUNCH(h, K_TSQR_LEAF_Q, tsqr_leaf_apply_kernel<T>, dim3(plan.L, cs), kThreads, s_lapply, N, b, r_leaf, plan.L,
               cs, B.Yleaf, N, B.tau, B.nref, B.Zbuf, B.Q, N, B.Tbuf);
    // reconstruction
    const T *Rroot = B.Rbuf + (size_t)(plan.total - 1) * b * b;
    const size_t s_lu = sizeof(T) * (3 * (size_t)(b + 1) * b + b);
    SEV_CUDA(cudaFuncSetAttribute(recon_lu_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_lu));
    SEV_LAUNCH(h, K_RECON_LU, recon_lu_kernel<T>, 1, kThreads, s_lu, b, B.Q, N, Rroot, U, N, Tm, B.Winv, P, lda);
    const size_t s_u2 = sizeof(T) * (size_t)(b + 1) * b;
    SEV_CUDA(cudaFuncSetAttribute(recon_u2_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_u2));
    const int g2 = (N - b + 63) / 64;
    if (g2 > 0)
        SEV_LAUNCH(h, K_RECON_U2, recon_u2_kernel<T>, g2, kThreads, s_u2, N, b, B.Q, N, B.Winv, U, N, P, lda);
    return SEV_OK;
}

template int panel_factor<float>(sev_ctx *, int, int, float *, int, float *, float *, void *);
template int panel_factor<double>(sev_ctx *, int, int, double *, int, double *, double *, void *);
template size_t panel_workspace<float>(sev_ctx *, int, int);
template int panel_finish_single_leaf<float>(sev_ctx *, int, int, const float *, const float *, const int *,
                                             const float *, float *, float *, int);
template int panel_finish_single_leaf<double>(sev_ctx *, int, int, const double *, const double *, const int *,
                                              const double *, double *, double *, int);
template int panel_form_u2<float>(sev_ctx *, int, int, const float *, const float *, float *, float *, int);
template int panel_form_u2<double>(sev_ctx *, int, int, const double *, const double *, double *, double *, int);
template size_t panel_workspace<double>(sev_ctx *, int, int);

}  // namespace sev
