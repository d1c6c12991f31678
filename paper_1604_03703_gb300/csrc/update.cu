// update.cu -- the two-sided trailing update of the full-to-band reduction
// (Eq. 4.1 as used in Algorithm 4.1) and the full-to-band driver.
//
// Per panel, with U (N x b) and T (b x b) from panel.cu and A22 the lower-
// stored trailing matrix:
//   Y  = A22 U                       (symm: reads A22 symmetrically)
//   X  = Y T                         (= W T in the algorithm's notation)
//   Zm = T^T (U^T X)
//   V  = 1/2 U Zm - X                (the V_1 line of Algorithm 4.1)
//   A22 <- A22 + U V^T + V U^T       (syr2k, lower tiles only)
//
// The FP64 form runs all of it on SIMT tiles (64 x 64 outputs, 4 x 4 per
// thread, DFMA); the mixed form's symm runs on larger FP32 tiles
// (symm_f32_kernel) and its syr2k on the tensor cores (update_tc.cu).
#include "common.cuh"

namespace sev {

template <typename T>
int panel_factor(sev_ctx *h, int N, int b, T *P, int lda, T *U, T *Tm, void *ws);
template <typename T>
size_t panel_workspace(sev_ctx *h, int n, int b);
template <typename T>
int tc_update_supported(sev_ctx *h, int N, int b);
template <typename T>
int tc_syr2k(sev_ctx *h, int N, int b, T *A22, int lda, const T *U, const T *V, void *ws);
template <typename T>
size_t tc_workspace(int n, int b);
template <typename T>
int tc_symm_supported(sev_ctx *h, int N, int b, const T *A22, int lda);
template <typename T>
int tc_symm(sev_ctx *h, int N, int b, const T *A22, int lda, const T *U, T *Y, T *ypart, int max_splits, void *ws);

constexpr int BM = 64, BN = 64, BK = 16, PADT = 4;

template <typename T>
struct Tile {
    T As[BK][BM + PADT];
    T Bs[BK][BN + PADT];
};

template <typename T>
__device__ __forceinline__ void tile_mma(const Tile<T> &t, T (&acc)[4][4]) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int k = 0; k < BK; ++k) {
        T a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = t.As[k][tx + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = t.Bs[k][ty + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
    }
}

// A slab (BM x BK) where element (m, k) = src[m + k*ld] (m contiguous).
template <typename T>
__device__ __forceinline__ void load_a_mcont(Tile<T> &t, const T *src, int ld, int m0, int k0, int M, int K) {
    for (int idx = threadIdx.x; idx < BM * BK; idx += blockDim.x) {
        const int m = idx % BM, k = idx / BM;
        const int gm = m0 + m, gk = k0 + k;
        t.As[k][m] = (gm < M && gk < K) ? src[(size_t)gm + (size_t)gk * ld] : T(0);
    }
}
// A slab where element (m, k) = src[k + m*ld] (k contiguous).
template <typename T>
__device__ __forceinline__ void load_a_kcont(Tile<T> &t, const T *src, int ld, int m0, int k0, int M, int K) {
    for (int idx = threadIdx.x; idx < BM * BK; idx += blockDim.x) {
        const int k = idx % BK, m = idx / BK;
        const int gm = m0 + m, gk = k0 + k;
        t.As[k][m] = (gm < M && gk < K) ? src[(size_t)gk + (size_t)gm * ld] : T(0);
    }
}
// B slab (BK x BN) where element (k, n) = src[k + n*ld] (k contiguous).
template <typename T>
__device__ __forceinline__ void load_b_kcont(Tile<T> &t, const T *src, int ld, int k0, int n0, int K, int N) {
    for (int idx = threadIdx.x; idx < BK * BN; idx += blockDim.x) {
        const int k = idx % BK, n = idx / BK;
        const int gk = k0 + k, gn = n0 + n;
        t.Bs[k][n] = (gk < K && gn < N) ? src[(size_t)gk + (size_t)gn * ld] : T(0);
    }
}
// B slab where element (k, n) = src[n + k*ld] (n contiguous).
template <typename T>
__device__ __forceinline__ void load_b_ncont(Tile<T> &t, const T *src, int ld, int k0, int n0, int K, int N) {
    for (int idx = threadIdx.x; idx < BK * BN; idx += blockDim.x) {
        const int n = idx % BN, k = idx / BN;
        const int gk = k0 + k, gn = n0 + n;
        t.Bs[k][n] = (gk < K && gn < N) ? src[(size_t)gn + (size_t)gk * ld] : T(0);
    }
}

// Y = A22 U, A22 symmetric N x N stored in its lower triangle.
template <typename T>
__global__ void __launch_bounds__(256) symm_kernel(int N, int b, const T *__restrict__ A, int lda,
                                                   const T *__restrict__ U, int ldu, T *__restrict__ Y, int ldy) {
    __shared__ Tile<T> t;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    T acc[4][4] = {};
    for (int k0 = 0; k0 < N; k0 += BK) {
        if (k0 + BK <= m0) {
            load_a_mcont(t, A, lda, m0, k0, N, N);  // strictly below the diagonal
        } else if (k0 >= m0 + BM) {
            load_a_kcont(t, A, lda, m0, k0, N, N);  // strictly above: A(m,k) = A(k,m)
        } else {
            for (int idx = threadIdx.x; idx < BM * BK; idx += blockDim.x) {
                const int m = idx % BM, k = idx / BM;
                const int gm = m0 + m, gk = k0 + k;
                T v = 0;
                if (gm < N && gk < N) v = gm >= gk ? A[(size_t)gm + (size_t)gk * lda] : A[(size_t)gk + (size_t)gm * lda];
                t.As[k][m] = v;
            }
        }
        load_b_kcont(t, U, ldu, k0, n0, N, b);
        __syncthreads();
        tile_mma(t, acc);
        __syncthreads();
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + tx + 16 * i, n = n0 + ty + 16 * j;
            if (m < N && n < b) Y[(size_t)m + (size_t)n * ldy] = acc[i][j];
        }
}

// Y = A22 U for FP32 data: 128 x 64 output tiles, 8 x 4 outputs per thread,
// K in steps of 16 through double-buffered shared memory (the next step's
// loads in registers while this one is multiplied), float4 loads of A22 in
// whichever orientation is contiguous (columns below the diagonal block,
// rows -- A(m, k) = A(k, m) -- above it, transposed into shared memory),
// and the K range split over blockIdx.z with per-split partial tiles
// (summed in a fixed order by symm_reduce_kernel) so that every SM has work.
// Needs lda % 4 == 0 and a 16-byte-aligned A22.
constexpr int SBM = 128, SBN = 64, SBK = 16;

struct SymmSmem {
    float As[2][SBK][SBM + 4];
    float Bs[2][SBK][SBN + 4];
};

__device__ __forceinline__ void symm_load_a(float4 (&ra)[2], float (&rs)[8], bool &vec, int &mode, const float *A,
                                            int lda, int N, int m0, int k0) {
    const int tid = threadIdx.x;
    const bool inside = m0 + SBM <= N && k0 + SBK <= N;
    if (inside && k0 + SBK <= m0) {  // strictly below: columns are contiguous
        mode = 0;
        vec = true;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = tid + r * 256, k = idx >> 5, mq = idx & 31;
            ra[r] = *reinterpret_cast<const float4 *>(A + (size_t)(m0 + 4 * mq) + (size_t)(k0 + k) * lda);
        }
    } else if (inside && k0 >= m0 + SBM) {  // strictly above: A(m, k) = A(k, m), rows contiguous
        mode = 1;
        vec = true;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = tid + r * 256, m = idx >> 2, kq = idx & 3;
            ra[r] = *reinterpret_cast<const float4 *>(A + (size_t)(k0 + 4 * kq) + (size_t)(m0 + m) * lda);
        }
    } else {  // crosses the diagonal block or the matrix edge: element by element
        mode = 2;
        vec = false;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int idx = tid + r * 256, m = idx & (SBM - 1), k = idx >> 7;
            const int gm = m0 + m, gk = k0 + k;
            float v = 0.f;
            if (gm < N && gk < N) v = gm >= gk ? A[(size_t)gm + (size_t)gk * lda] : A[(size_t)gk + (size_t)gm * lda];
            rs[r] = v;
        }
    }
}

__device__ __forceinline__ void symm_store_a(SymmSmem &S, int buf, const float4 (&ra)[2], const float (&rs)[8],
                                             int mode) {
    const int tid = threadIdx.x;
    if (mode == 0) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = tid + r * 256, k = idx >> 5, mq = idx & 31;
            *reinterpret_cast<float4 *>(&S.As[buf][k][4 * mq]) = ra[r];
        }
    } else if (mode == 1) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = tid + r * 256, m = idx >> 2, kq = idx & 3;
            S.As[buf][4 * kq + 0][m] = ra[r].x;
            S.As[buf][4 * kq + 1][m] = ra[r].y;
            S.As[buf][4 * kq + 2][m] = ra[r].z;
            S.As[buf][4 * kq + 3][m] = ra[r].w;
        }
    } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int idx = tid + r * 256, m = idx & (SBM - 1), k = idx >> 7;
            S.As[buf][k][m] = rs[r];
        }
    }
}

__device__ __forceinline__ void symm_load_b(float (&rb)[4], const float *U, int ldu, int N, int b, int k0, int n0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int idx = threadIdx.x + r * 256, k = idx & (SBK - 1), n = idx >> 4;
        const int gk = k0 + k, gn = n0 + n;
        rb[r] = (gk < N && gn < b) ? U[(size_t)gk + (size_t)gn * ldu] : 0.f;
    }
}

__device__ __forceinline__ void symm_store_b(SymmSmem &S, int buf, const float (&rb)[4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int idx = threadIdx.x + r * 256, k = idx & (SBK - 1), n = idx >> 4;
        S.Bs[buf][k][n] = rb[r];
    }
}

__global__ void __launch_bounds__(256) symm_f32_kernel(int N, int b, const float *__restrict__ A, int lda,
                                                       const float *__restrict__ U, int ldu, int kchunk,
                                                       float *__restrict__ Yout, int ldy, size_t split_stride) {
    __shared__ __align__(16) SymmSmem S;
    const int m0 = blockIdx.x * SBM, n0 = blockIdx.y * SBN;
    const int kbeg = blockIdx.z * kchunk, kend = min(N, kbeg + kchunk);
    float *Y = Yout + (size_t)blockIdx.z * split_stride;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    float4 ra[2];
    float rs[8], rb[4];
    bool vec;
    int mode;
    int buf = 0;
    if (kbeg < kend) {
        symm_load_a(ra, rs, vec, mode, A, lda, N, m0, kbeg);
        symm_load_b(rb, U, ldu, N, b, kbeg, n0);
        symm_store_a(S, 0, ra, rs, mode);
        symm_store_b(S, 0, rb);
    }
    __syncthreads();
    for (int k0 = kbeg; k0 < kend; k0 += SBK) {
        const bool more = k0 + SBK < kend;
        if (more) {
            symm_load_a(ra, rs, vec, mode, A, lda, N, m0, k0 + SBK);
            symm_load_b(rb, U, ldu, N, b, k0 + SBK, n0);
        }
        // rows beyond kend in this step are zero-padded only at the matrix
        // edge; split boundaries are multiples of SBK
#pragma unroll
        for (int k = 0; k < SBK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&S.As[buf][k][4 * tx]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&S.As[buf][k][64 + 4 * tx]);
            const float4 bv = *reinterpret_cast<const float4 *>(&S.Bs[buf][k][4 * ty]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bw[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bw[j], acc[i][j]);
        }
        if (more) {
            symm_store_a(S, buf ^ 1, ra, rs, mode);
            symm_store_b(S, buf ^ 1, rb);
        }
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + (i < 4 ? 4 * tx + i : 64 + 4 * tx + i - 4);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + 4 * ty + j;
            if (m < N && n < b) Y[(size_t)m + (size_t)n * ldy] = acc[i][j];
        }
    }
}

// Y = sum over the splits of the partial tiles, in split order.
__global__ void symm_reduce_kernel(int N, int b, int splits, const float *__restrict__ part, size_t split_stride,
                                   float *__restrict__ Y, int ldy) {
    const size_t total = (size_t)N * b;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(idx % N), n = (int)(idx / N);
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[(size_t)z * split_stride + idx];
        Y[(size_t)m + (size_t)n * ldy] = s;
    }
}

int launch_symm_reduce(sev_ctx *h, int N, int b, int splits, const float *part, float *Y) {
    int g = (int)(((size_t)N * b + 255) / 256);
    if (g > h->sm_count * 8) g = h->sm_count * 8;
    SEV_LAUNCH(h, K_SYMM, symm_reduce_kernel, g, 256, 0, N, b, splits, part, (size_t)N * b, Y, N);
    return SEV_OK;
}

// C = alpha * A B + beta * D, A (M x K, m contiguous), B (K x Nc, k contiguous, ld ldb).
// Used for X = Y T and V = 1/2 U Zm - X.
template <typename T>
__global__ void __launch_bounds__(256) gemm_nn_kernel(int M, int Nc, int K, T alpha, const T *__restrict__ A, int lda,
                                                      const T *__restrict__ B, int ldb, T beta,
                                                      const T *__restrict__ D, int ldd, T *__restrict__ C, int ldc) {
    __shared__ Tile<T> t;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    T acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += BK) {
        load_a_mcont(t, A, lda, m0, k0, M, K);
        load_b_kcont(t, B, ldb, k0, n0, K, Nc);
        __syncthreads();
        tile_mma(t, acc);
        __syncthreads();
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + tx + 16 * i, n = n0 + ty + 16 * j;
            if (m < M && n < Nc) {
                T v = alpha * acc[i][j];
                if (beta != T(0)) v += beta * D[(size_t)m + (size_t)n * ldd];
                C[(size_t)m + (size_t)n * ldc] = v;
            }
        }
}

// Partial products P_s = U[rows_s]^T X[rows_s] (b x b) for row chunk s.
template <typename T>
__global__ void __launch_bounds__(256) utx_partial_kernel(int N, int b, int chunk, const T *__restrict__ U, int ldu,
                                                          const T *__restrict__ X, int ldx, T *__restrict__ part) {
    __shared__ Tile<T> t;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN, s = blockIdx.z;
    const int kbeg = s * chunk, kend = min(N, kbeg + chunk);
    T acc[4][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        // A(m = a, k = i) = U[i, a] (k contiguous); B(k = i, n = c) = X[i, c]
        for (int idx = threadIdx.x; idx < BM * BK; idx += blockDim.x) {
            const int k = idx % BK, m = idx / BK;
            const int gm = m0 + m, gk = k0 + k;
            t.As[k][m] = (gm < b && gk < kend) ? U[(size_t)gk + (size_t)gm * ldu] : T(0);
        }
        for (int idx = threadIdx.x; idx < BK * BN; idx += blockDim.x) {
            const int k = idx % BK, n = idx / BK;
            const int gk = k0 + k, gn = n0 + n;
            t.Bs[k][n] = (gk < kend && gn < b) ? X[(size_t)gk + (size_t)gn * ldx] : T(0);
        }
        __syncthreads();
        tile_mma(t, acc);
        __syncthreads();
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T *P = part + (size_t)s * b * b;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + tx + 16 * i, n = n0 + ty + 16 * j;
            if (m < b && n < b) P[m + (size_t)n * b] = acc[i][j];
        }
}

// M = sum_s P_s, entry by entry, the partials in a fixed order (deterministic).
template <typename T>
__global__ void __launch_bounds__(256) utx_sum_kernel(int bb, int nparts, const T *__restrict__ part, T *__restrict__ M) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= bb) return;
    T s = 0;
    for (int p = 0; p < nparts; ++p) s += part[(size_t)p * bb + idx];
    M[idx] = s;
}

// Zm = T^T M (M = sum_s P_s, b x b; T upper triangular): CTA handles 4
// columns; Zm(a, c) = sum_{q <= a} T(q, a) M(q, c), summed in q order.
template <typename T>
__global__ void __launch_bounds__(256) utx_tmul_kernel(int b, const T *__restrict__ M, const T *__restrict__ Tm,
                                                       T *__restrict__ Zm) {
    extern __shared__ __align__(16) unsigned char smem[];
    T *Ms = (T *)smem;  // b x 4
    const int c0 = blockIdx.x * 4;
    const int nc = min(4, b - c0);
    for (int idx = threadIdx.x; idx < b * nc; idx += blockDim.x) Ms[idx] = M[idx % b + (size_t)(c0 + idx / b) * b];
    __syncthreads();
    for (int idx = threadIdx.x; idx < b * nc; idx += blockDim.x) {
        const int a = idx % b, c = idx / b;
        T s = 0;
        for (int q = 0; q <= a; ++q) s += Tm[q + (size_t)a * b] * Ms[q + (size_t)c * b];
        Zm[a + (size_t)(c0 + c) * b] = s;
    }
}

// A22 += U V^T + V U^T on the lower tiles (tile (I, J), I >= J).
template <typename T>
__global__ void __launch_bounds__(256) syr2k_kernel(int N, int b, T *__restrict__ A, int lda, const T *__restrict__ U,
                                                    int ldu, const T *__restrict__ V, int ldv) {
    __shared__ Tile<T> t;
    const long x = blockIdx.x;
    int I = (int)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
    while ((long)(I + 1) * (I + 2) / 2 <= x) ++I;
    while ((long)I * (I + 1) / 2 > x) --I;
    const int J = (int)(x - (long)I * (I + 1) / 2);
    const int m0 = I * BM, n0 = J * BN;
    T acc[4][4] = {};
    const int K2 = 2 * b;
    for (int k0 = 0; k0 < K2; k0 += BK) {
        for (int idx = threadIdx.x; idx < BM * BK; idx += blockDim.x) {
            const int m = idx % BM, k = idx / BM;
            const int gm = m0 + m, gk = k0 + k;
            T v = 0;
            if (gm < N && gk < K2) v = gk < b ? U[(size_t)gm + (size_t)gk * ldu] : V[(size_t)gm + (size_t)(gk - b) * ldv];
            t.As[k][m] = v;
        }
        for (int idx = threadIdx.x; idx < BK * BN; idx += blockDim.x) {
            const int n = idx % BN, k = idx / BN;
            const int gk = k0 + k, gn = n0 + n;
            T v = 0;
            if (gn < N && gk < K2) v = gk < b ? V[(size_t)gn + (size_t)gk * ldv] : U[(size_t)gn + (size_t)(gk - b) * ldu];
            t.Bs[k][n] = v;
        }
        __syncthreads();
        tile_mma(t, acc);
        __syncthreads();
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + tx + 16 * i, n = n0 + ty + 16 * j;
            if (m < N && n < N && m >= n) A[(size_t)m + (size_t)n * lda] += acc[i][j];
        }
}

// --------------------------------------------------------------- driver
template <typename T>
struct F2BBuffers {
    T *U, *Y, *X, *V, *Tm, *Zm, *part, *ypart;
    void *panel_ws, *tc_ws;
};

constexpr int kSymmMaxSplits = 8;

// Row chunks of U^T X: 256 rows or more each, at most 64 (a wave of CTAs at
// b = 128: 2 x 2 tiles x 64 chunks).
static int utx_parts(int N) {
    int p = (N + 255) / 256;
    return p < 1 ? 1 : (p > 64 ? 64 : p);
}

template <typename T>
static void carve_f2b(Carver &c, F2BBuffers<T> &B, sev_ctx *h, int n, int b, bool tc) {
    B.U = c.take<T>((size_t)n * b);
    B.Y = c.take<T>((size_t)n * b);
    B.X = c.take<T>((size_t)n * b);
    B.V = c.take<T>((size_t)n * b);
    B.Tm = c.take<T>((size_t)b * b);
    B.Zm = c.take<T>((size_t)b * b);
    B.part = c.take<T>((size_t)(utx_parts(n) + 1) * b * b);  // the chunks' partial products, then their sum
    B.ypart = c.take<T>((size_t)kSymmMaxSplits * n * b);
    B.tc_ws = tc ? (void *)c.take<char>(tc_workspace<T>(n, b)) : nullptr;
    B.panel_ws = c.take<char>(panel_workspace<T>(h, n, b));
}

template <typename T>
size_t full_to_band_workspace(sev_ctx *h, int n, int b) {
    Carver c(nullptr);
    F2BBuffers<T> B;
    carve_f2b<T>(c, B, h, n, b, true);
    return c.bytes();
}

template <typename T>
int launch_full_to_band(sev_ctx *h, int n, T *A, int lda, int b, T *AB, int ldab, void *ws, size_t ws_bytes) {
    if (n <= 0) return SEV_OK;
    if (ws_bytes < full_to_band_workspace<T>(h, n, b)) return SEV_ERR_WORKSPACE;
    Carver c(ws);
    F2BBuffers<T> B;
    carve_f2b<T>(c, B, h, n, b, true);
    for (int k = 0;; ++k) {
        const int c0 = k * b, r0 = c0 + b;
        if (r0 >= n) break;
        const int N = n - r0;
        if (N < 2) break;
        T *P = A + (size_t)r0 + (size_t)c0 * lda;
        T *A22 = A + (size_t)r0 + (size_t)r0 * lda;
        int rc = panel_factor<T>(h, N, b, P, lda, B.U, B.Tm, B.panel_ws);
        if (rc) return rc;
        const bool tc = tc_update_supported<T>(h, N, b);
        // Y = A22 U
        if (tc_symm_supported<T>(h, N, b, A22, lda)) {
            rc = tc_symm<T>(h, N, b, A22, lda, B.U, B.Y, B.ypart, kSymmMaxSplits, B.tc_ws);
            if (rc) return rc;
        } else if (sizeof(T) == 4 && lda % 4 == 0 && ((uintptr_t)A22 & 15) == 0) {
            // split K until the grid covers ~2 CTAs per SM
            const int mt = (N + SBM - 1) / SBM, nt = (b + SBN - 1) / SBN;
            int splits = 1;
            while (splits < kSymmMaxSplits && mt * nt * splits < 2 * h->sm_count && N / (splits * 2) >= 256) splits *= 2;
            const int kchunk = ((N + splits - 1) / splits + SBK - 1) / SBK * SBK;
            float *dst = splits > 1 ? (float *)B.ypart : (float *)B.Y;
            SEV_LAUNCH(h, K_SYMM, symm_f32_kernel, dim3(mt, nt, splits), 256, 0, N, b, (const float *)A22, lda,
                       (const float *)B.U, N, kchunk, dst, N, (size_t)N * b);
            if (splits > 1) {
                int g = (int)(((size_t)N * b + 255) / 256);
                if (g > h->sm_count * 8) g = h->sm_count * 8;
                SEV_LAUNCH(h, K_SYMM, symm_reduce_kernel, g, 256, 0, N, b, splits, (const float *)B.ypart,
                           (size_t)N * b, (float *)B.Y, N);
            }
        } else {
            SEV_LAUNCH(h, K_SYMM, symm_kernel<T>, dim3((N + BM - 1) / BM, (b + BN - 1) / BN), 256, 0, N, b, A22, lda,
                       B.U, N, B.Y, N);
        }
        // X = Y T
        SEV_LAUNCH(h, K_VFORM_XT, gemm_nn_kernel<T>, dim3((N + BM - 1) / BM, (b + BN - 1) / BN), 256, 0, N, b, b, T(1),
                   B.Y, N, B.Tm, b, T(0), (const T *)nullptr, N, B.X, N);
        // Zm = T^T (U^T X)
        const int parts = utx_parts(N);
        const int chunk = (((N + parts - 1) / parts) + BK - 1) / BK * BK;
        SEV_LAUNCH(h, K_VFORM_UTX, utx_partial_kernel<T>, dim3((b + BM - 1) / BM, (b + BN - 1) / BN, parts), 256, 0, N,
                   b, chunk, B.U, N, B.X, N, B.part);
        {
            // the chunks summed by b^2 threads, then T^T applied (4 columns a CTA)
            T *Msum = B.part + (size_t)parts * b * b;
            SEV_LAUNCH(h, K_VFORM_REDUCE, utx_sum_kernel<T>, (b * b + 255) / 256, 256, 0, b * b, parts, B.part, Msum);
            SEV_LAUNCH(h, K_VFORM_REDUCE, utx_tmul_kernel<T>, (b + 3) / 4, 256, sizeof(T) * (size_t)b * 4, b, Msum,
                       B.Tm, B.Zm);
        }
        // V = 1/2 U Zm - X
        SEV_LAUNCH(h, K_VFORM_V, gemm_nn_kernel<T>, dim3((N + BM - 1) / BM, (b + BN - 1) / BN), 256, 0, N, b, b,
                   T(0.5), B.U, N, B.Zm, b, T(-1), B.X, N, B.V, N);
        // A22 += U V^T + V U^T
        if (tc) {
            rc = tc_syr2k<T>(h, N, b, A22, lda, B.U, B.V, B.tc_ws);
            if (rc) return rc;
        } else {
            const long nt = (N + BM - 1) / BM;
            SEV_LAUNCH(h, K_SYR2K, syr2k_kernel<T>, (unsigned)(nt * (nt + 1) / 2), 256, 0, N, b, A22, lda, B.U, N, B.V,
                       N);
        }
    }
    return launch_band_from_dense<T>(h, n, A, lda, b, AB, ldab);
}

template int launch_full_to_band<float>(sev_ctx *, int, float *, int, int, float *, int, void *, size_t);
template int launch_full_to_band<double>(sev_ctx *, int, double *, int, int, double *, int, void *, size_t);
template size_t full_to_band_workspace<float>(sev_ctx *, int, int);
template size_t full_to_band_workspace<double>(sev_ctx *, int, int);

}  // namespace sev
