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

// ------------------------------------------------------ symmetric product
// Y = A22 U, the first product of the V formation (W = A22 U in Eq. 4.1 /
// Algorithm 4.1), for FP32 data on the tensor cores in BF16x3:
// Y ~ Ah Uh + Ah Ul + Al Uh (hi/lo splits as in split_bf16x3_kernel; the
// Al Ul term, ~2^-16 relative, dropped).
//
// CTA (I, s) computes rows [128 I, 128 I + 128) of Y over the 64-wide
// K-blocks of split s.  A22 is stored in its lower triangle only, so the A
// tile of K-block kb comes from whichever triangle holds it: below the
// diagonal block, a 128 (rows) x 64 box of its columns (TMA, rows
// contiguous); above it, a 64 x 128 box of the stored lower part read as
// rows (A(i, k) = A(k, i); TMA, k contiguous); the two K-blocks that meet the
// diagonal are loaded element by element.  Converter warps split every FP32
// tile into BF16 hi and lo tiles in the K-major, 128-byte-swizzled layout
// of the MMA operand (16-byte chunk c of row i at chunk c ^ (i mod 8)); the
// U tiles, split once per panel, arrive by TMA in that layout.
//
// Accumulation.  The tensor core sums at most kSyChunk K-blocks (512 terms)
// in TMEM; the chunks alternate between two TMEM accumulators, and four
// accumulator warps add each finished chunk into an FP32 register sum (IEEE
// round-to-nearest) while the next chunk is being multiplied.  Summing all
// N terms in TMEM made the error grow with N (measured: 5.8e-5 ||A|| at
// n = 16384 against 3.7e-6 at n = 4096).
//
// Warps: 0 TMA producer, 1-4 converters, 5 MMA issuer, 6-9 accumulators
// (TMEM lanes 32 (warp mod 4) .. + 31, i.e. tile rows).  Every wait is
// time-capped; a CTA whose wait runs out latches SEV_ERR_TIMEOUT, lets the
// copies and MMAs it issued finish, frees its TMEM and returns.
constexpr int kSyRaw = 2;                   // FP32 tile stages
constexpr int kSyCvt = 2;                   // converted operand stages
constexpr int kSyRawBytes = 128 * 64 * 4;   // one FP32 tile
constexpr int kSyChunk = 8;                 // K-blocks summed in TMEM before the register sum
constexpr int kSyThreads = 320;
__host__ __device__ constexpr int sy_cvt_bytes(int bn) { return 2 * 128 * 128 + 2 * bn * 128; }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Eight FP32 values of row i, K-chunk ch: BF16 hi and lo parts into the
// swizzled hi / lo tiles (128-byte rows).
__device__ __forceinline__ void sy_store_chunk(unsigned char *hi_t, unsigned char *lo_t, int i, int ch,
                                               const float (&v)[8]) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * j]), h1 = __float2bfloat16_rn(v[2 * j + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * j] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * j + 1] - __bfloat162float(h1));
        h[j] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        l[j] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    const int off = i * 128 + ((ch ^ (i & 7)) << 4);
    *reinterpret_cast<uint4 *>(hi_t + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(lo_t + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

template <int BN>
__global__ void __launch_bounds__(kSyThreads, 1)
    symm_tc_kernel(const __grid_constant__ CUtensorMap mapAc, const __grid_constant__ CUtensorMap mapAr,
                   const __grid_constant__ CUtensorMap mapUh, const __grid_constant__ CUtensorMap mapUl,
                   const float *__restrict__ A, int lda, int N, int kb_per_split, float *__restrict__ Ypart,
                   size_t split_stride, int *err) {
    constexpr int kCvt = sy_cvt_bytes(BN);
    constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((128u >> 4) << 24);
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *raw = smem;
    unsigned char *cvt = raw + kSyRaw * kSyRawBytes;
    __shared__ __align__(8) uint64_t raw_full[kSyRaw], raw_empty[kSyRaw], u_full[kSyCvt], a_full[kSyCvt],
        cvt_empty[kSyCvt], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail, s_raw_issued, s_u_issued, s_mma_done;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = blockIdx.x, s = blockIdx.y;
    const int nkb = (N + 63) / 64;
    const int kb0 = s * kb_per_split, kb1 = min(nkb, kb0 + kb_per_split);
    const int nblk = kb1 - kb0, nchunk = (nblk + kSyChunk - 1) / kSyChunk;
    // 0: below the diagonal block, 1: above it, 2: meets the diagonal
    auto kind = [&](int kb) { return 64 * kb + 64 <= 128 * I ? 0 : (64 * kb >= 128 * I + 128 ? 1 : 2); };

    if (threadIdx.x == 0) {
        for (int q = 0; q < kSyRaw; ++q) {
            mbar_init(&raw_full[q], 1);
            mbar_init(&raw_empty[q], 4);
        }
        for (int q = 0; q < kSyCvt; ++q) {
            mbar_init(&u_full[q], 1);
            mbar_init(&a_full[q], 4);
            mbar_init(&cvt_empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&acc_full[q], 1);
            mbar_init(&acc_empty[q], 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
        s_raw_issued = 0;
        s_u_issued = 0;
        s_mma_done = 0;
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base, 2 * BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer: FP32 A tiles (off-diagonal K-blocks), U hi/lo tiles
        int r = 0, c = 0;
        for (int kb = kb0; kb < kb1; ++kb, ++c) {
            const int k = kind(kb);
            if (k != 2) {
                const int sr = r % kSyRaw, ur = r / kSyRaw;
                if (ur > 0 && !mbar_wait(&raw_empty[sr], (ur - 1) & 1, err)) {
                    s_fail = 1;
                    break;
                }
                mbar_expect_tx(&raw_full[sr], kSyRawBytes);
                if (k == 0)
                    tma_load_2d(raw + sr * kSyRawBytes, &mapAc, 128 * I, 64 * kb, &raw_full[sr]);
                else
                    tma_load_2d(raw + sr * kSyRawBytes, &mapAr, 64 * kb, 128 * I, &raw_full[sr]);
                ++r;
                s_raw_issued = r;
            }
            const int sc = c % kSyCvt, uc = c / kSyCvt;
            if (uc > 0 && !mbar_wait(&cvt_empty[sc], (uc - 1) & 1, err)) {
                s_fail = 1;
                break;
            }
            unsigned char *cs = cvt + sc * kCvt;
            mbar_expect_tx(&u_full[sc], 2 * BN * 128);
            tma_load_2d(cs + 32768, &mapUh, 64 * kb, 0, &u_full[sc]);
            tma_load_2d(cs + 32768 + BN * 128, &mapUl, 64 * kb, 0, &u_full[sc]);
            s_u_issued = c + 1;
        }
    } else if (warp >= 1 && warp <= 4) {
        // ---- converters: FP32 tile -> BF16 hi / lo operand tiles
        const int t = threadIdx.x - 32;  // 0 .. 127
        int r = 0, c = 0;
        for (int kb = kb0; kb < kb1; ++kb, ++c) {
            const int k = kind(kb);
            const int sc = c % kSyCvt, uc = c / kSyCvt;
            if (uc > 0 && !mbar_wait(&cvt_empty[sc], (uc - 1) & 1, err)) {
                s_fail = 1;
                break;
            }
            unsigned char *ah = cvt + sc * kCvt, *al = ah + 16384;
            if (k == 2) {
                const int gi = 128 * I + t;
#pragma unroll 1
                for (int ch = 0; ch < 8; ++ch) {
                    float v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int gk = 64 * kb + 8 * ch + j;
                        float x = 0.f;
                        if (gi < N && gk < N) x = gi >= gk ? A[(size_t)gi + (size_t)gk * lda] : A[(size_t)gk + (size_t)gi * lda];
                        v[j] = x;
                    }
                    sy_store_chunk(ah, al, t, ch, v);
                }
            } else {
                const int sr = r % kSyRaw, ur = r / kSyRaw;
                if (!mbar_wait(&raw_full[sr], ur & 1, err)) {
                    s_fail = 1;
                    break;
                }
                const float *rw = reinterpret_cast<const float *>(raw + sr * kSyRawBytes);
                if (k == 0) {  // tile stored [k][i] (128 rows per k): thread t takes row t
#pragma unroll 2
                    for (int ch = 0; ch < 8; ++ch) {
                        float v[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) v[j] = rw[(8 * ch + j) * 128 + t];
                        sy_store_chunk(ah, al, t, ch, v);
                    }
                } else {  // tile stored [i][k] (64 k per row): 8 threads per row, 16 rows per pass
#pragma unroll 2
                    for (int pass = 0; pass < 8; ++pass) {
                        const int i = pass * 16 + (t >> 3), ch = t & 7;
                        const float4 x0 = *reinterpret_cast<const float4 *>(rw + i * 64 + 8 * ch);
                        const float4 x1 = *reinterpret_cast<const float4 *>(rw + i * 64 + 8 * ch + 4);
                        const float v[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                        sy_store_chunk(ah, al, i, ch, v);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&raw_empty[sr]);
                ++r;
            }
            fence_proxy_async_smem();  // the tensor core reads these tiles through the async proxy
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_full[sc]);
        }
    } else if (warp == 5 && lane == 0) {
        // ---- MMA issuer: chunk ch of kSyChunk K-blocks into TMEM buffer ch & 1
        int c = 0;
        for (int kb = kb0; kb < kb1; ++kb, ++c) {
            const int ch = c / kSyChunk, buf = ch & 1;
            const bool first = c % kSyChunk == 0, last = c % kSyChunk == kSyChunk - 1 || kb + 1 == kb1;
            if (first && ch >= 2 && !mbar_wait(&acc_empty[buf], ((ch >> 1) - 1) & 1, err)) {
                s_fail = 1;
                break;
            }
            const int sc = c % kSyCvt, uc = c / kSyCvt;
            if (!mbar_wait(&u_full[sc], uc & 1, err) || !mbar_wait(&a_full[sc], uc & 1, err)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            unsigned char *cs = cvt + sc * kCvt;
            const uint64_t dah = desc_sw128(cs), dal = desc_sw128(cs + 16384);
            const uint64_t duh = desc_sw128(cs + 32768), dul = desc_sw128(cs + 32768 + BN * 128);
            const uint32_t dt = tmem + (uint32_t)(buf * BN);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {  // K = 16 per instruction: +32 bytes = +2 in the address field
                umma_bf16(dt, dah + 2 * kk, duh + 2 * kk, kIdesc, (first && kk == 0) ? 0u : 1u);
                umma_bf16(dt, dah + 2 * kk, dul + 2 * kk, kIdesc, 1);
                umma_bf16(dt, dal + 2 * kk, duh + 2 * kk, kIdesc, 1);
            }
            umma_commit(&cvt_empty[sc]);
            if (last) umma_commit(&acc_full[buf]);
            s_mma_done = c + 1;
        }
    } else if (warp >= 6) {
        // ---- accumulators: register sum of the chunks, then the rows of Y
        const int quarter = warp & 3;
        const uint32_t tb = tmem + ((uint32_t)(32 * quarter) << 16);
        float sum[BN];
#pragma unroll
        for (int j = 0; j < BN; ++j) sum[j] = 0.f;
        bool ok = true;
        for (int ch = 0; ch < nchunk; ++ch) {
            const int buf = ch & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (ch >> 1) & 1, err) ? 1 : 0)) {
                ok = false;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int cc = 0; cc < BN / 32; ++cc) {
                float acc[32];
                tmem_ld32(tb + (uint32_t)(buf * BN + cc * 32), acc);
#pragma unroll
                for (int j = 0; j < 32; ++j) sum[cc * 32 + j] += acc[j];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
        if (ok && !s_fail) {
            const int row = 128 * I + 32 * quarter + lane;
            float *Y = Ypart + (size_t)s * split_stride;
            if (row < N) {
#pragma unroll
                for (int j = 0; j < BN; ++j) Y[(size_t)row + (size_t)j * N] = sum[j];
            }
        } else if (lane == 0) {
            latch_error(err, SEV_ERR_TIMEOUT);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (s_fail && threadIdx.x == 0) {
        // a wait ran out: let the copies this CTA issued land and its MMAs
        // finish before the TMEM is freed (the last phase of each stage)
        const long long cap = kWaitCyclesDefault;
        for (int q = 0; q < kSyRaw; ++q) {
            int last = -1;
            for (int r = 0; r < s_raw_issued; ++r)
                if (r % kSyRaw == q) last = r;
            if (last >= 0) mbar_wait_for(&raw_full[q], (last / kSyRaw) & 1, cap);
        }
        for (int q = 0; q < kSyCvt; ++q) {
            int last = -1;
            for (int c = 0; c < s_u_issued; ++c)
                if (c % kSyCvt == q) last = c;
            if (last >= 0) mbar_wait_for(&u_full[q], (last / kSyCvt) & 1, cap);
        }
        if (s_mma_done > 0) {
            const int last = s_mma_done - 1;
            mbar_wait_for(&cvt_empty[last % kSyCvt], (last / kSyCvt) & 1, cap);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 2 * BN);
}

// U (N x b FP32, column-major, ld N) -> Uh, Ul (BF16, column-major, ld ldh).
__global__ void split_u_kernel(int N, int b, int ldh, const float *__restrict__ U, __nv_bfloat16 *__restrict__ Uh,
                               __nv_bfloat16 *__restrict__ Ul) {
    const long total = (long)ldh * b;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int r = (int)(idx % ldh), c = (int)(idx / ldh);
        const float u = r < N ? U[(size_t)r + (size_t)c * N] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(u);
        Uh[idx] = h;
        Ul[idx] = __float2bfloat16_rn(u - __bfloat162float(h));
    }
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

// 2D map of a column-major FP32 matrix (rows x cols, leading dimension ld
// elements), boxes of box_r rows x box_c columns, no swizzle, zero fill.
static int make_map_f32(CUtensorMap *m, const void *base, int rows, int cols, int ld, int box_r, int box_c) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return SEV_ERR_CUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {(cuuint32_t)box_r, (cuuint32_t)box_c};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SEV_OK : SEV_ERR_CUDA;
}

// 2D map of a column-major BF16 matrix (rows x cols, ld elements, rows
// contiguous), boxes of 64 rows x box_c columns, 128-byte swizzle.
static int make_map_bf16_cm(CUtensorMap *m, const void *base, int rows, int cols, int ld, int box_c) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return SEV_ERR_CUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)box_c};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
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

template <typename T>
int tc_symm_supported(sev_ctx *h, int N, int b, const T *A22, int lda) {
    if (sizeof(T) != 4 || !tc_update_supported<T>(h, N, b)) return 0;
    static int disabled = -1;
    if (disabled < 0) disabled = getenv("SEV_NO_TC_SYMM") ? 1 : 0;
    if (disabled) return 0;
    return (b == 32 || b == 64 || b == 128) && N >= 256 && lda % 4 == 0 && ((uintptr_t)A22 & 15) == 0;
}

// Y = A22 U on the tensor cores; partial products of the K splits go to
// ypart (kSymmMaxSplits x N x b) and are summed in split order into Y.
template <typename T>
int tc_symm(sev_ctx *h, int N, int b, const T *A22, int lda, const T *U, T *Y, T *ypart, int max_splits, void *ws) {
    if constexpr (sizeof(T) != 4) {
        return SEV_ERR_UNSUPPORTED;
    } else {
        const int ldh = (N + 7) / 8 * 8;
        Carver c(ws);
        __nv_bfloat16 *Uh = c.take<__nv_bfloat16>((size_t)ldh * b);
        __nv_bfloat16 *Ul = c.take<__nv_bfloat16>((size_t)ldh * b);
        int g = (int)(((long)ldh * b + 255) / 256);
        if (g > h->sm_count * 16) g = h->sm_count * 16;
        SEV_LAUNCH(h, K_SPLIT_BF16, split_u_kernel, g, 256, 0, N, b, ldh, U, Uh, Ul);
        CUtensorMap mAc, mAr, mUh, mUl;
        int rc = make_map_f32(&mAc, A22, N, N, lda, 128, 64);
        if (!rc) rc = make_map_f32(&mAr, A22, N, N, lda, 64, 128);
        if (!rc) rc = make_map_bf16_cm(&mUh, Uh, N, b, ldh, b);
        if (!rc) rc = make_map_bf16_cm(&mUl, Ul, N, b, ldh, b);
        if (rc) return rc;
        const int nkb = (N + 63) / 64, rb = (N + 127) / 128;
        // split K so that the grid covers about one wave of CTAs (one per SM)
        int S = (h->sm_count + rb / 2) / rb;
        S = S < 1 ? 1 : (S > max_splits ? max_splits : S);
        const int per = (nkb + S - 1) / S;
        S = (nkb + per - 1) / per;  // every split gets at least one K-block
        const size_t smem = (size_t)kSyRaw * kSyRawBytes + (size_t)kSyCvt * sy_cvt_bytes(b) + 1024;
        auto kern = b == 128 ? symm_tc_kernel<128> : (b == 64 ? symm_tc_kernel<64> : symm_tc_kernel<32>);
        SEV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        float *dst = S > 1 ? (float *)ypart : (float *)Y;
        SEV_LAUNCH(h, K_SYMM, kern, dim3(rb, S), kSyThreads, smem, mAc, mAr, mUh, mUl, (const float *)A22, lda, N, per,
                   dst, (size_t)N * b, h->d_err);
        if (S > 1) {
            rc = launch_symm_reduce(h, N, b, S, (const float *)ypart, (float *)Y);
            if (rc) return rc;
        }
        return SEV_OK;
    }
}

template int tc_update_supported<float>(sev_ctx *, int, int);
template int tc_update_supported<double>(sev_ctx *, int, int);
template int tc_syr2k<float>(sev_ctx *, int, int, float *, int, const float *, const float *, void *);
template int tc_syr2k<double>(sev_ctx *, int, int, double *, int, const double *, const double *, void *);
template size_t tc_workspace<float>(int, int);
template int tc_symm_supported<float>(sev_ctx *, int, int, const float *, int);
template int tc_symm_supported<double>(sev_ctx *, int, int, const double *, int);
template int tc_symm<float>(sev_ctx *, int, int, const float *, int, const float *, float *, float *, int, void *);
template int tc_symm<double>(sev_ctx *, int, int, const double *, int, const double *, double *, double *, int,
                             void *);
template size_t tc_workspace<double>(int, int);

}  // namespace sev
