// update_tc.cu -- the trailing syr2k update of the full-to-band reduction,
// A22 <- A22 + U V^T + V U^T (Eq. 4.1), on the 5th-generation tensor cores
// (tcgen05) in BF16x3 form, for the mixed precision (FP32 data).
//
// Split.  Each FP32 operand x is written as x_hi + x_lo with x_hi = bf16(x)
// and x_lo = bf16(x - x_hi); the product x y is approximated by
// x_hi y_hi + x_hi y_lo + x_lo y_hi (the x_lo y_lo term, ~2^-16 relative, is
// dropped), accumulated in FP32.  With the row-major (K-contiguous) BF16
// operands
//   P = [U_hi | V_hi | U_hi | V_hi | U_lo | V_lo]   (N x 6b, padded to 64)
//   Q = [V_hi | U_hi | V_lo | U_lo | V_hi | U_hi]
// one GEMM P Q^T with K = 6b gives U V^T + V U^T in that form.
//
// GEMM.  One CTA (4 warps) per 128 x 128 lower tile (I >= J) of A22.  Warp 0
// lane 0 loads K-steps of 64 (a 128 x 64 BF16 tile of P and of Q, 128-byte
// swizzle) with TMA into a 3-stage ring guarded by mbarriers; warp 1 lane 0
// issues tcgen05.mma (M = 128, N = 128, K = 16, kind::f16, FP32 accumulate in
// TMEM) and frees each stage with tcgen05.commit; the 4 warps then read the
// 128 x 128 accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31,
// i.e. tile rows) and add it to A22's lower triangle.  Every mbarrier wait
// is time-capped: on expiry the kernel latches SEV_ERR_TIMEOUT, skips its
// epilogue and still frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace sev {

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Wait on an mbarrier phase for at most `cap` SM cycles; false on timeout.
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t phase, long long cap) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase))
        if (clock64() - t0 > cap) return false;
    return true;
}
// The same with the handle's wait limit.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase, const int *err) {
    return mbar_wait_for(bar, phase, wait_cap(err));
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte rows in the
// 128-byte swizzled layout TMA writes (8-row atoms of 1024 bytes): start
// address >> 4, stride between 8-row groups 1024 bytes, descriptor version 1,
// layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t desc_sw128(const void *tile) {
    const uint32_t addr = smem_u32(tile);
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major,
// N = 128, M = 128.
constexpr uint32_t kIdescBF16_128x128 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

constexpr int kTcStages = 3;
constexpr int kTcStageBytes = 2 * 128 * 64 * 2;  // A + B tile

// ----------------------------------------------------------- split kernel
__global__ void split_bf16x3_kernel(int N, int b, int K6p, const float *__restrict__ U, const float *__restrict__ V,
                                    __nv_bfloat16 *__restrict__ P, __nv_bfloat16 *__restrict__ Q) {
    const long total = (long)N * K6p;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / K6p), k = (int)(idx % K6p);
        __nv_bfloat16 p = __float2bfloat16_rn(0.f), q = p;
        if (k < 6 * b) {
            const int seg = k / b, c = k % b;
            const float u = U[(size_t)r + (size_t)c * N], v = V[(size_t)r + (size_t)c * N];
            const __nv_bfloat16 uh = __float2bfloat16_rn(u), vh = __float2bfloat16_rn(v);
            const __nv_bfloat16 ul = __float2bfloat16_rn(u - __bfloat162float(uh));
            const __nv_bfloat16 vl = __float2bfloat16_rn(v - __bfloat162float(vh));
            switch (seg) {
                case 0: p = uh; q = vh; break;
                case 1: p = vh; q = uh; break;
                case 2: p = uh; q = vl; break;
                case 3: p = vh; q = ul; break;
                case 4: p = ul; q = vh; break;
                default: p = vl; q = uh; break;
            }
        }
        P[idx] = p;
        Q[idx] = q;
    }
}

// ------------------------------------------------------------ GEMM kernel
__global__ void __launch_bounds__(128, 1)
    syr2k_tc_kernel(const __grid_constant__ CUtensorMap mapP, const __grid_constant__ CUtensorMap mapQ, int N,
                    int ksteps, float *__restrict__ A, int lda, int *err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail, s_issued, s_waited;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // lower tile (I, J), I >= J, from the linear block index
    const long x = blockIdx.x;
    int I = (int)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
    while ((long)(I + 1) * (I + 2) / 2 <= x) ++I;
    while ((long)I * (I + 1) / 2 > x) --I;
    const int J = (int)(x - (long)I * (I + 1) / 2);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
        s_issued = 0;
        s_waited = 0;
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base, 128);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // TMA producer
        int issued = 0;
        for (int ks = 0; ks < ksteps; ++ks) {
            const int s = ks % kTcStages, round = ks / kTcStages;
            if (ks >= kTcStages && !mbar_wait(&empty[s], (round - 1) & 1, err)) {
                s_fail = 1;
                break;
            }
            unsigned char *st = smem + (size_t)s * kTcStageBytes;
            mbar_expect_tx(&full[s], kTcStageBytes);
            tma_load_2d(st, &mapP, ks * 64, I * 128, &full[s]);
            tma_load_2d(st + kTcStageBytes / 2, &mapQ, ks * 64, J * 128, &full[s]);
            ++issued;
        }
        s_issued = issued;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        bool ok = true;
        int waited = 0;
        for (int ks = 0; ks < ksteps; ++ks) {
            const int s = ks % kTcStages, round = ks / kTcStages;
            if (!mbar_wait(&full[s], round & 1, err)) {
                ok = false;
                s_fail = 1;
                break;
            }
            tc_fence_after();
            unsigned char *st = smem + (size_t)s * kTcStageBytes;
            const uint64_t ad = desc_sw128(st), bd = desc_sw128(st + kTcStageBytes / 2);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)  // K = 16 per instruction: +32 bytes = +2 in the address field
                umma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, kIdescBF16_128x128, (ks | kk) != 0);
            umma_commit(&empty[s]);
            ++waited;
        }
        s_waited = waited;
        if (ok) umma_commit(&done);
    }
    __syncwarp();
    // epilogue: every thread waits for the accumulator
    // warp-uniform decision: tcgen05.ld is .sync.aligned
    const bool have = __all_sync(0xffffffffu, mbar_wait(&done, 0, err) ? 1 : 0) && !s_fail;
    tc_fence_after();
    if (have) {
        const int row = I * 128 + warp * 32 + lane;
        const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int cc = 0; cc < 4; ++cc) {
            float acc[32];
            tmem_ld32(tbase + cc * 32, acc);
            if (row < N) {
                // All 32 loads are issued before any store: the compiler cannot
                // prove arow[j * lda] distinct across j (lda is a runtime
                // value), so a fused load-add-store loop would wait one memory
                // latency per column.
                float *arow = A + row;
                float old[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int j = J * 128 + cc * 32 + c;
                    old[c] = (j < N && row >= j) ? arow[(size_t)j * lda] : 0.0f;
                }
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int j = J * 128 + cc * 32 + c;
                    if (j < N && row >= j) arow[(size_t)j * lda] = old[c] + acc[c];
                }
            }
        }
    } else if (threadIdx.x == 0) {
        latch_error(err, SEV_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (s_fail && threadIdx.x == 0) {
        // a wait ran out: before the CTA frees its TMEM and leaves, let the
        // copies it issued land and the MMAs it committed finish (each with
        // the default limit, whatever the handle's limit is)
        for (int ks = s_waited; ks < s_issued; ++ks)
            mbar_wait_for(&full[ks % kTcStages], (ks / kTcStages) & 1, kWaitCyclesDefault);
        if (s_waited > 0) {
            const int last = s_waited - 1;
            mbar_wait_for(&empty[last % kTcStages], (last / kTcStages) & 1, kWaitCyclesDefault);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

// -------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2D map of a row-major BF16 matrix rows x cols (cols contiguous), 128 x 64 boxes.
static int make_map(CUtensorMap *m, void *base, int rows, int cols) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return SEV_ERR_CUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {64, 128};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SEV_OK : SEV_ERR_CUDA;
}

static int k6p_of(int b) { return (6 * b + 63) / 64 * 64; }

template <typename T>
int tc_update_supported(sev_ctx *h, int N, int b) {
    if (sizeof(T) != 4) return 0;
    static int disabled = -1;
    if (disabled < 0) disabled = getenv("SEV_NO_TC") ? 1 : 0;
    if (disabled) return 0;
    (void)h;
    return N >= 2 && b >= 1 && encode_fn() != nullptr;
}

template <typename T>
size_t tc_workspace(int n, int b) {
    if (sizeof(T) != 4) return 0;
    Carver c(nullptr);
    c.take<__nv_bfloat16>((size_t)n * k6p_of(b));
    c.take<__nv_bfloat16>((size_t)n * k6p_of(b));
    return c.bytes();
}

template <typename T>
int tc_syr2k(sev_ctx *h, int N, int b, T *A22, int lda, const T *U, const T *V, void *ws) {
    if constexpr (sizeof(T) != 4) {
        return SEV_ERR_UNSUPPORTED;
    } else {
        const int K6p = k6p_of(b);
        Carver c(ws);
        __nv_bfloat16 *P = c.take<__nv_bfloat16>((size_t)N * K6p);
        __nv_bfloat16 *Q = c.take<__nv_bfloat16>((size_t)N * K6p);
        const long total = (long)N * K6p;
        int g = (int)((total + 255) / 256);
        if (g > h->sm_count * 32) g = h->sm_count * 32;
        SEV_LAUNCH(h, K_SPLIT_BF16, split_bf16x3_kernel, g, 256, 0, N, b, K6p, U, V, P, Q);
        CUtensorMap mP, mQ;
        int rc = make_map(&mP, P, N, K6p);
        if (rc) return rc;
        rc = make_map(&mQ, Q, N, K6p);
        if (rc) return rc;
        const size_t smem = (size_t)kTcStages * kTcStageBytes + 1024;
        SEV_CUDA(cudaFuncSetAttribute(syr2k_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const long nt = (N + 127) / 128;
        SEV_LAUNCH(h, K_SYR2K_TC, syr2k_tc_kernel, (unsigned)(nt * (nt + 1) / 2), 128, smem, mP, mQ, N, K6p / 64,
                   (float *)A22, lda, h->d_err);
        return SEV_OK;
    }
}

template int tc_update_supported<float>(sev_ctx *, int, int);
template int tc_update_supported<double>(sev_ctx *, int, int);
template int tc_syr2k<float>(sev_ctx *, int, int, float *, int, const float *, const float *, void *);
template int tc_syr2k<double>(sev_ctx *, int, int, double *, int, const double *, const double *, void *);
template size_t tc_workspace<float>(int, int);
template size_t tc_workspace<double>(int, int);

}  // namespace sev
