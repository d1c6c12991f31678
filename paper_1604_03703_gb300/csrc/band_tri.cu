// band_tri.cu -- the last band reduction, b -> 1 (Algorithm 4.2 with k = b,
// h = 1), for b <= 32, as a sliding-window bulge chase.
//
// With h = 1 every chase (i, j) is ONE Householder reflector: it
// annihilates the single column o_qr.c below row o_qr.r (o_qr.r =
// i + (j-1) b, o_qr.c = o_qr.r - 1 for j = 1, o_qr.r - b for j > 1) and
// applies H two-sidedly to the qr rows [o_qr.r, o_qr.r + n_r) against the
// update rows [o_up.c, o_up.c + n_c) (o_up.c = o_qr.r for j = 1,
// o_qr.r - b + 1 for j > 1; n_c = min(n - o_up.c, 2b) resp. 3b - 1).  One
// warp performs a chase: lane l owns one update row above, in, and below
// the qr rows; off rows get X <- X H (row-local), the qr-row block gets
// H X H = X - v w^T - w v^T with p = tau X v, w = p - (tau/2)(p^T v) v.
//
// Schedule.  A CTA takes G consecutive sweeps (compute warp g -> sweep
// i0 + g) and steps them together: at step t warp g performs chase t - 3g,
// so sweep i runs 3 chases behind sweep i - 1 -- the rule that chase (i, j)
// follows (i - 1, j + 2) -- and the chases of one step are independent.
// Steps are separated by a named barrier among the compute warps.  The band
// columns the group touches live in a shared-memory ring of (3G + 3) b + 2
// columns (2b diagonals each): a loader warp brings columns in (16-byte
// asynchronous copies) ahead of warp 0, and a writer warp writes them back
// once the group's last sweep has passed them (after its chase j, columns
// below o_qr.r(i_last, j) are final).  The writer then publishes j with a
// release store; the next group's loader waits (acquire, capped) for j + 2
// before loading a column range -- the only global synchronisation, once
// per step per group boundary.  Groups are handed out in order by a global
// counter and each CTA finishes its group before taking another, so every
// awaited group is held by a running CTA.
#include "common.cuh"

#ifdef SEV_TRACE
static __device__ long long *sev_trace_buf = nullptr;
static __device__ int sev_trace_phase_on = 0;
static __device__ long long sev_trace_phase[8];
extern "C" int sev_trace_set(void *p) {
    return cudaMemcpyToSymbol(sev_trace_buf, &p, sizeof(p)) == cudaSuccess ? 0 : 1;
}
#define TRACE(gi, t, k, v)                                                                    \
    do {                                                                                      \
        if (sev_trace_buf && (gi) < 4 && (t) < 4096) sev_trace_buf[((gi) * 4096 + (t)) * 8 + (k)] = (v); \
    } while (0)
#define TRACEP(k)                                                                      \
    do {                                                                               \
        if (sev_trace_phase_on == (int)blockIdx.x + 1 && (threadIdx.x & 31) == 0 && (threadIdx.x >> 5) == 0) \
            sev_trace_phase[(k)] = clock64();                                          \
    } while (0)
#else
#define TRACEP(k) \
    do {          \
    } while (0)
#define TRACE(gi, t, k, v) \
    do {                   \
    } while (0)
#endif

#include "tri_chase.cuh"

namespace sev {

// G compute warps + one loader warp + one writer warp, decoupled through
// shared-memory flags.  Compute warps step together (named barrier 1): at
// step t warp g performs chase t - 3g once the loader has made step t's
// columns available (s_avail >= t).  The loader runs ahead: it polls the
// previous group (acquire, capped, cached), waits for ring space (columns
// written back, s_wblo) and loads each step's new columns.  The writer runs
// behind: once compute has finished a step (s_done), it writes back every
// column that became final, advances s_wblo and publishes the group's
// progress (release store).  Flags are ordered with block-scope fences; each
// wait is capped and an abort turns the remaining steps into no-ops so that
// every warp still reaches its barriers.  The ring holds (3G + 3) b + 2
// columns.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int B, int G>
__host__ __device__ constexpr int tri_wcap() {
    return (3 * G + 3) * B + 2;
}

__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <typename T, int B, int G>
__global__ void __launch_bounds__((G + 2) * 32, 1)
    band_tri_kernel(int n, T *AB, int ldab, int nsweeps, int ngroups, int *progress, int *group_ctr, int *err,
                    int async_ok) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int LDW = 2 * B;
    constexpr int wcap = tri_wcap<B, G>();
    TriWin<T, B> W;
    W.w = (T *)smem;
    W.wcap = wcap;
    T *vb = W.w + (size_t)wcap * LDW;  // G x 32
    T *wb = vb + G * 32;               // G x 32
    __shared__ int s_group;
    __shared__ volatile int s_abort, s_avail, s_done, s_wblo;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool loader = warp == G, writer = warp == G + 1;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int g = atomicAdd(group_ctr, 1);
            s_group = g;
            s_abort = 0;
            s_avail = 0;
            s_done = 0;
            s_wblo = 1 + g * G - 1;
        }
        __syncthreads();
        const int gi = s_group;
        if (gi >= ngroups) break;
        const int i0 = 1 + gi * G;
        const int nact = min(G, nsweeps - i0 + 1);
        const int il = i0 + nact - 1;
        const int Jf = tri_chases(n, B, i0), Jl = tri_chases(n, B, il);
        const int Jprev = gi > 0 ? tri_chases(n, B, i0 - 1) : 0;
        const int tmax = Jl + 3 * (nact - 1);
        auto hi_of = [&](int ts) { return (ts >= Jf) ? n : min(n, i0 + ts * B); };

        if (warp < G) {
            // ------------------------------------------------------ compute
            T rv = T(0), rtau = T(0), rbeta = T(0);  // this warp's pending reflector
            for (int t = 1; t <= tmax; ++t) {
                if (warp == 0 && lane == 0) TRACE(gi, t, 0, clock64());
                if (warp == 0 && lane == 0 && !s_abort) {
                    const int need = min(t, Jf);
                    const long long t0 = clock64();
                    while (s_avail < need && !s_abort) {
                        if (wait_expired(t0, err)) {
                            latch_error(err, SEV_ERR_TIMEOUT);
                            s_abort = 1;
                        }
                    }
                    __threadfence_block();
                }
                named_bar(1, G * 32);
                if (warp == 0 && lane == 0) TRACE(gi, t, 1, clock64());
                if (!s_abort) {
                    const int j = t - 3 * warp;
                    const int i = i0 + warp;
                    const int Ji = tri_chases(n, B, i);
                    if (warp < nact && j >= 1 && j <= Ji) {
                        const int o = i + (j - 1) * B;
                        if (j == 1) {
                            // the sweep's first reflector: column i - 1, rows [i, i + n_r)
                            const int nr1 = min(n - o, B);
                            T *xcol = W.w + (size_t)((o - 1) % wcap) * LDW + 1;
                            const T x = lane < nr1 ? xcol[lane] : T(0);
                            tri_reflector<T, B>(x, nr1, rv, rtau, rbeta);
                            if (lane < nr1) xcol[lane] = lane == 0 ? rbeta : T(0);
                            __syncwarp();
                        }
#ifdef SEV_TRACE
                        if (warp == 0 && lane == 0 && gi == 1 && j == 40) sev_trace_phase_on = blockIdx.x + 1;
                        __syncwarp();
#endif
                        if (j > 1 && j < Ji && o + 3 * B <= n)
                            tri_chase<T, B, true>(n, o, j, true, W, vb + warp * 32, wb + warp * 32, rv, rtau, rbeta);
                        else
                            tri_chase<T, B>(n, o, j, j < Ji, W, vb + warp * 32, wb + warp * 32, rv, rtau, rbeta);
#ifdef SEV_TRACE
                        if (warp == 0 && lane == 0 && gi == 1 && j == 40 && sev_trace_buf)
                            for (int k = 0; k < 6; ++k) sev_trace_buf[3 * 4096 * 8 + 4000 * 8 + k] = sev_trace_phase[k];
                        if (warp == 0 && lane == 0 && gi == 1 && j == 40) sev_trace_phase_on = 0;
#endif
                    }
                }
                if (lane == 0) TRACE(gi, t, 3 + (warp < 3 ? warp : 2), clock64());
                named_bar(1, G * 32);
                if (warp == 0 && lane == 0) {
                    TRACE(gi, t, 2, clock64());
                    __threadfence_block();
                    s_done = t;
                }
            }
        } else if (loader) {
            // ------------------------------------------------------- loader
            int loaded_hi = i0 - 1, seen = 0;
            for (int ts = 1; ts <= Jf && !s_abort; ++ts) {
                if (async_ok && ts > 1) {
                    // the previous step's copies land and are published before
                    // this step waits for anything (the ring-space wait depends
                    // on compute having consumed them)
                    cp_async_wait_all();
                    __syncwarp();
                    if (lane == 0) {
                        __threadfence_block();
                        s_avail = ts - 1;
                    }
                }
                if (gi > 0 && ts + 2 > seen) {
                    const int need = (ts + 2 <= Jprev) ? ts + 2 : kTriInf;
                    int pv = 0;
                    if (lane == 0) {
                        const long long t0 = clock64();
                        while ((pv = ld_acquire_i(&progress[gi - 1])) < need) {
                            if (*(volatile int *)err != 0 || s_abort) {
                                pv = -1;
                                break;
                            }
                            if (wait_expired(t0, err)) {
                                latch_error(err, SEV_ERR_TIMEOUT);
                                pv = -1;
                                break;
                            }

                        }
                    }
                    pv = __shfl_sync(0xffffffffu, pv, 0);
                    if (pv < 0) {
                        if (lane == 0) s_abort = 1;
                        break;
                    }
                    seen = pv;
                    if (lane == 0) TRACE(gi, ts, 6, clock64());
                }
                const int hi = hi_of(ts);
                // ring space: columns below hi - wcap must have been written back
                if (lane == 0) {
                    const long long t0 = clock64();
                    while (s_wblo < hi - wcap && !s_abort) {
                        if (wait_expired(t0, err)) {
                            latch_error(err, SEV_ERR_TIMEOUT);
                            s_abort = 1;
                        }
                    }
                    __threadfence_block();
                }
                __syncwarp();
                if (s_abort) break;
                const int c0 = loaded_hi;
                if (async_ok) {
                    // asynchronous 16-byte copies (zero-filled past the matrix
                    // end), all issued at once: a step costs one memory latency
                    // instead of one per batch of loads; published at the top of
                    // the next iteration (or after the loop)
                    constexpr int EPC = 16 / (int)sizeof(T);  // elements per chunk
                    constexpr int CH = LDW / EPC;             // chunks per column
                    for (int q = lane; q < (hi - c0) * CH; q += 32) {
                        const int c = c0 + q / CH, d0 = (q % CH) * EPC;
                        int valid = n - c - d0;
                        valid = valid < 0 ? 0 : (valid > EPC ? EPC : valid);
                        const T *src = valid > 0 ? AB + d0 + (size_t)c * ldab : AB;
                        cp_async16(W.w + (size_t)(c % wcap) * LDW + d0, src, valid * (int)sizeof(T));
                    }
                    cp_async_commit();
                } else {
                    batched_copy<T, 16>(
                        (hi - c0) * LDW, lane, 32,
                        [&](int k) {
                            const int c = c0 + k / LDW, d = k % LDW;
                            return (c + d < n) ? __ldcg(AB + d + (size_t)c * ldab) : T(0);
                        },
                        [&](int k, T v) { W.w[((c0 + k / LDW) % wcap) * LDW + k % LDW] = v; });
                    __syncwarp();
                    if (lane == 0) {
                        __threadfence_block();
                        s_avail = ts;
                    }
                }
                loaded_hi = max(loaded_hi, hi);
                if (lane == 0) TRACE(gi, ts, 7, clock64());
            }
            if (async_ok) {
                // every copy in flight lands before the loader publishes or leaves
                cp_async_wait_all();
                __syncwarp();
                if (lane == 0 && !s_abort) {
                    __threadfence_block();
                    s_avail = Jf;
                }
            }
        } else if (writer) {
            // ------------------------------------------------------- writer
            int wb_lo = i0 - 1, written = 0;
            while (written < tmax) {
                int ts = 0;
                if (lane == 0) {
                    const long long t0 = clock64();
                    while ((ts = s_done) <= written && !s_abort) {
                        if (wait_expired(t0, err)) {
                            latch_error(err, SEV_ERR_TIMEOUT);
                            s_abort = 1;
                        }
                    }
                    __threadfence_block();
                }
                ts = __shfl_sync(0xffffffffu, ts, 0);
                if (s_abort) break;
                written = ts;
                const int jl = ts - 3 * (nact - 1);
                if (jl < 1) continue;
                const bool done = jl >= Jl;
                const int fin = done ? n : min(n, il + (jl - 1) * B);
                for (int idx = lane; idx < (fin - wb_lo) * LDW; idx += 32) {
                    const int c = wb_lo + idx / LDW, d = idx % LDW;
                    if (c + d < n) AB[d + (size_t)c * ldab] = W.w[(c % wcap) * LDW + d];
                }
                if (fin > wb_lo) wb_lo = fin;
                __syncwarp();
                if (lane == 0) {
                    __threadfence_block();
                    s_wblo = wb_lo;
                    // the release store orders the warp's write-back before the flag
                    st_release_i(&progress[gi], done ? kTriInf : jl);
                }
            }
        }
        __syncthreads();
        if (s_abort) return;
    }
}

template <typename T, int B, int G>
static int launch_tri(sev_ctx *h, int n, T *AB, int ldab, int *progress, int *ctr, int nsweeps) {
    const int ngroups = (nsweeps + G - 1) / G;
    constexpr int wcap = tri_wcap<B, G>();
    const size_t smem = sizeof(T) * ((size_t)wcap * 2 * B + 2 * G * 32);
    if (smem > h->smem_optin) return SEV_ERR_UNSUPPORTED;
    SEV_CUDA(cudaMemsetAsync(progress, 0, sizeof(int) * (size_t)ngroups, h->stream));
    SEV_CUDA(cudaMemsetAsync(ctr, 0, sizeof(int), h->stream));
    auto kern = band_tri_kernel<T, B, G>;
    SEV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SEV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (G + 2) * 32, smem));
    if (per_sm < 1) return SEV_ERR_UNSUPPORTED;
    // groups start ~3G steps apart and each runs ~J + 3G steps, so about
    // J / (3G) of them are busy at once; more CTAs would only poll
    const int J1 = tri_chases(n, B, 1);
    int grid = h->sm_count * per_sm;
    const int busy = J1 / (3 * G) + 16;
    if (grid > busy) grid = busy;
    if (grid > ngroups) grid = ngroups;
    // 16-byte asynchronous copies need a 16-byte-aligned band and column stride
    const int async_ok = ((uintptr_t)AB % 16 == 0) && ((size_t)ldab * sizeof(T)) % 16 == 0;
    SEV_LAUNCH(h, K_BAND_TRI, kern, grid, (G + 2) * 32, smem, n, AB, ldab, nsweeps, ngroups, progress, ctr,
               h->d_err, async_ok);
    return SEV_OK;
}

// Compute warps (sweeps) per CTA: fewer per CTA spreads the concurrently
// active sweeps over more SMs.
#ifndef SEV_TRI_G_SMALL
#define SEV_TRI_G_SMALL 8
#endif
#ifndef SEV_TRI_G16
#define SEV_TRI_G16 4
#endif
#ifndef SEV_TRI_G32
#define SEV_TRI_G32 4
#endif

int band_tri_supported(int b, int elem) { return b == 2 || b == 4 || b == 8 || b == 16 || (b == 32 && elem == 4); }

size_t band_tri_workspace(int n) {
    Carver c(nullptr);
    c.take<int>((size_t)n + 1);
    c.take<int>(1);
    return c.bytes();
}

template <typename T>
int launch_band_tri(sev_ctx *h, int n, T *AB, int ldab, int b, void *ws, size_t ws_bytes) {
    const int nsweeps = n >= 3 ? n - 2 : 0;
    if (nsweeps <= 0) return SEV_OK;
    if (ws_bytes < band_tri_workspace(n)) return SEV_ERR_WORKSPACE;
    Carver c(ws);
    int *progress = c.take<int>((size_t)n + 1);
    int *ctr = c.take<int>(1);
    switch (b) {
        case 2: return launch_tri<T, 2, SEV_TRI_G_SMALL>(h, n, AB, ldab, progress, ctr, nsweeps);
        case 4: return launch_tri<T, 4, SEV_TRI_G_SMALL>(h, n, AB, ldab, progress, ctr, nsweeps);
        case 8: return launch_tri<T, 8, SEV_TRI_G_SMALL>(h, n, AB, ldab, progress, ctr, nsweeps);
        case 16: return launch_tri<T, 16, SEV_TRI_G16>(h, n, AB, ldab, progress, ctr, nsweeps);
        case 32:
            if constexpr (sizeof(T) == 4) return launch_tri<T, 32, SEV_TRI_G32>(h, n, AB, ldab, progress, ctr, nsweeps);
            return SEV_ERR_UNSUPPORTED;
        default: return SEV_ERR_UNSUPPORTED;
    }
}

template int launch_band_tri<float>(sev_ctx *, int, float *, int, int, void *, size_t);
template int launch_band_tri<double>(sev_ctx *, int, double *, int, int, void *, size_t);

}  // namespace sev
