// autotune.cu -- choice of the first band width b0 and of the band-to-band
// stage widths for sev_eigvalsh (Algorithm 4.3 reduces to band width b0 and
// then through successively narrower bands; the paper fixes neither b0 nor
// the stages for a machine, and Algorithm 4.2 holds for any h dividing b).
//
// The cost of the path is the sum of its parts, each measured once at the
// order n on this GPU: the full-to-band reduction for every candidate b0,
// and every band stage b -> h (b, h powers of two, h | b) that the kernels
// support.  The cheapest way from each width down to 1 follows by dynamic
// programming over the measured stage costs; the chosen b0 minimises
// full-to-band + band path.  The result is kept in the handle per bucket
// of n (orders within a factor sqrt 2) and precision, and optionally in a
// cache file (environment variable SEV_TUNE_CACHE) keyed by the GPU name.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "common.cuh"

namespace sev {

__device__ __forceinline__ unsigned long long tune_mix(unsigned long long z) {  // splitmix64 finaliser
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double tune_unit(unsigned long long r) {  // uniform in [-1, 1)
    return (double)(r >> 11) * 0x1.0p-52 - 1.0;
}

// Lower triangle of a symmetric n x n matrix, entries uniform in [-1, 1) / sqrt(n).
template <typename T>
__global__ void tune_fill_sym_kernel(int n, T *A, int lda, unsigned long long seed) {
    const double s = 1.0 / sqrt((double)n);
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)n * n; idx += (long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % n), j = (int)(idx / n);
        if (i >= j) A[i + (size_t)j * lda] = (T)(s * tune_unit(tune_mix(seed ^ (unsigned long long)idx)));
    }
}

// Packed band of half-bandwidth b (ldab rows), zeros beyond it.
template <typename T>
__global__ void tune_fill_band_kernel(int n, int b, T *AB, int ldab, unsigned long long seed) {
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)ldab * n; idx += (long)gridDim.x * blockDim.x) {
        const int d = (int)(idx % ldab), j = (int)(idx / ldab);
        AB[idx] = (d <= b && j + d < n) ? (T)tune_unit(tune_mix(seed ^ (unsigned long long)idx)) : T(0);
    }
}

int tune_bucket(int n) { return n <= 1 ? 0 : (int)std::lround(2.0 * std::log2((double)n)); }

static int wlog(int w) {  // log2 of a power of two in 1..128, else -1
    for (int k = 0; k < kTuneWidths; ++k)
        if ((1 << k) == w) return k;
    return -1;
}

const TunedBands *tuned_for(const sev_ctx *h, int n, int prec) {
    const int bk = tune_bucket(n);
    for (const TunedBands &t : h->tuned)
        if (t.bucket == bk && t.prec == prec) return &t;
    return nullptr;
}

// The stage widths from b0 (b0 first, 1 last) by the tuned table; 0 if the
// table does not reach 1 from b0.
int tuned_schedule(const TunedBands &t, int b0, int *out, int max_out) {
    int k = 0, b = b0;
    out[k++] = b;
    while (b > 1) {
        const int l = wlog(b);
        if (l < 0 || t.next[l] <= 0 || k >= max_out) return 0;
        b = t.next[l];
        out[k++] = b;
    }
    return k;
}

static void store_tuned(sev_ctx *h, const TunedBands &t) {
    for (TunedBands &x : h->tuned)
        if (x.bucket == t.bucket && x.prec == t.prec) {
            x = t;
            return;
        }
    h->tuned.push_back(t);
}

// Cache file lines: "<gpu name>|<prec>|<bucket>|<b0>|<next of widths 1, 2, 4, ..., 128>".
void tune_cache_load(sev_ctx *h) {
    const char *path = getenv("SEV_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, h->device) != cudaSuccess) {
        fclose(f);
        return;
    }
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char *bar = strchr(line, '|');
        if (!bar) continue;
        *bar = 0;
        if (strcmp(line, p.name) != 0) continue;
        TunedBands t;
        int nx[kTuneWidths];
        const int got = sscanf(bar + 1, "%d|%d|%d|%d %d %d %d %d %d %d %d", &t.prec, &t.bucket, &t.b0, &nx[0], &nx[1],
                               &nx[2], &nx[3], &nx[4], &nx[5], &nx[6], &nx[7]);
        if (got != 3 + kTuneWidths) continue;
        for (int k = 0; k < kTuneWidths; ++k) t.next[k] = nx[k];
        store_tuned(h, t);
    }
    fclose(f);
}

static void tune_cache_append(sev_ctx *h, const TunedBands &t) {
    const char *path = getenv("SEV_TUNE_CACHE");
    if (!path || !*path) return;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, h->device) != cudaSuccess) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s|%d|%d|%d|", p.name, t.prec, t.bucket, t.b0);
    for (int k = 0; k < kTuneWidths; ++k) fprintf(f, k ? " %d" : "%d", t.next[k]);
    fprintf(f, "\n");
    fclose(f);
}

template <typename T>
static bool stage_ok(sev_ctx *h, int b, int w) {
    if (w == 1) return band_tri_supported(b, (int)sizeof(T)) != 0;
    return b % w == 0 && band_smem_bytes<T>(b, w) <= h->smem_optin;
}

// Device milliseconds of one call of f() on the handle's stream.
template <typename F>
static int time_ms(sev_ctx *h, F f, float *ms) {
    cudaEvent_t e0, e1;
    SEV_CUDA(cudaEventCreate(&e0));
    SEV_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, h->stream);
    int rc = f();
    cudaEventRecord(e1, h->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess && rc == SEV_OK) rc = SEV_ERR_CUDA;
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

template <typename T>
static int autotune_t(sev_ctx *h, int n, int prec, int b0_req, TunedBands *out, double *best_ms) {
    const int widths[] = {128, 64, 32, 16, 8, 4, 2};
    int cand_b0[3], ncand = 0;
    if (b0_req > 0) {
        if (wlog(b0_req) < 0) return -4;
        cand_b0[ncand++] = b0_req;
    } else {
        for (int w : {32, 64, 128})
            if (w < n - 1) cand_b0[ncand++] = w;
    }
    if (ncand == 0) return SEV_ERR_UNSUPPORTED;
    int bmax = 0;
    for (int q = 0; q < ncand; ++q) bmax = cand_b0[q] > bmax ? cand_b0[q] : bmax;
    const int ldab = 2 * bmax;
    // buffers: the dense matrix, the band, and the stage workspace
    size_t stage = band_tri_workspace(n);
    for (int b : widths)
        for (int w : widths)
            if (w < b && b <= bmax) {
                const size_t s = band_workspace(n, b, w);
                if (s > stage) stage = s;
            }
    for (int q = 0; q < ncand; ++q) {
        const size_t f = full_to_band_workspace<T>(h, n, cand_b0[q]);
        if (f > stage) stage = f;
    }
    Carver cv(nullptr);
    cv.take<T>((size_t)n * n);
    cv.take<T>((size_t)ldab * n);
    const size_t own = cv.bytes();
    char *buf = nullptr;
    if (cudaMalloc(&buf, own) != cudaSuccess) {
        cudaGetLastError();
        return SEV_ERR_WORKSPACE;
    }
    Carver c(buf);
    T *A = c.take<T>((size_t)n * n);
    T *AB = c.take<T>((size_t)ldab * n);
    void *ws = nullptr;
    int rc = get_workspace(h, stage, &ws);
    const int grid = h->sm_count * 8;
    // cost[log2 b][log2 w] in ms; every stage first runs once untimed at a
    // small order so the timed run pays no module loading
    double cost[kTuneWidths][kTuneWidths];
    for (auto &r : cost)
        for (double &x : r) x = -1.0;
    const int nwarm = n < 1024 ? n : 1024;
    const int targets[] = {64, 32, 16, 8, 4, 2, 1};
    for (int b : widths) {
        if (rc || b > bmax || b >= n - 1) continue;
        for (int w : targets) {
            if (rc) break;
            if (w >= b || !stage_ok<T>(h, b, w)) continue;
            tune_fill_band_kernel<T><<<grid, 256, 0, h->stream>>>(nwarm, b, AB, ldab, 0x7A11ull);
            rc = w == 1 ? launch_band_tri<T>(h, nwarm, AB, ldab, b, ws, stage)
                        : launch_band_to_band<T>(h, nwarm, AB, ldab, b, w, ws, stage);
            if (rc == SEV_ERR_UNSUPPORTED) {  // no kernel for this edge here: not a candidate
                rc = SEV_OK;
                continue;
            }
            if (rc) break;
            tune_fill_band_kernel<T><<<grid, 256, 0, h->stream>>>(n, b, AB, ldab, 0x7A12ull + b * 131 + w);
            float ms = 0.f;
            rc = time_ms(h, [&] { return w == 1 ? launch_band_tri<T>(h, n, AB, ldab, b, ws, stage)
                                                 : launch_band_to_band<T>(h, n, AB, ldab, b, w, ws, stage); },
                         &ms);
            if (rc == SEV_ERR_UNSUPPORTED) {
                rc = SEV_OK;
                continue;
            }
            cost[wlog(b)][wlog(w)] = ms;
        }
    }
    if (!rc) rc = cudaStreamSynchronize(h->stream) == cudaSuccess ? SEV_OK : SEV_ERR_CUDA;
    // cheapest path to 1 from every width (widths ascending)
    double best[kTuneWidths];
    int next[kTuneWidths];
    for (int k = 0; k < kTuneWidths; ++k) {
        best[k] = k == 0 ? 0.0 : -1.0;
        next[k] = 0;
    }
    for (int k = 1; k < kTuneWidths && !rc; ++k)
        for (int j = 0; j < k; ++j)
            if (cost[k][j] >= 0.0 && best[j] >= 0.0 && (best[k] < 0.0 || cost[k][j] + best[j] < best[k])) {
                best[k] = cost[k][j] + best[j];
                next[k] = 1 << j;
            }
    // full-to-band for every candidate b0
    int b0_best = 0;
    double tot_best = -1.0;
    for (int q = 0; q < ncand && !rc; ++q) {
        const int b0 = cand_b0[q], l = wlog(b0);
        if (best[l] < 0.0) continue;
        const int nw = 2 * b0 + 2 < n ? 2 * b0 + 2 : n;  // warm-up order: a couple of panels
        tune_fill_sym_kernel<T><<<grid, 256, 0, h->stream>>>(nw, A, nw, 0xF00Dull);
        rc = launch_full_to_band<T>(h, nw, A, nw, b0, AB, ldab, ws, stage);
        if (rc == SEV_ERR_UNSUPPORTED) {  // this width has no full-to-band kernel here
            rc = SEV_OK;
            continue;
        }
        if (rc) break;
        tune_fill_sym_kernel<T><<<grid, 256, 0, h->stream>>>(n, A, n, 0xF00Eull + b0);
        float ms = 0.f;
        rc = time_ms(h, [&] { return launch_full_to_band<T>(h, n, A, n, b0, AB, ldab, ws, stage); }, &ms);
        if (rc == SEV_ERR_UNSUPPORTED) {
            rc = SEV_OK;
            continue;
        }
        const double tot = ms + best[l];
        if (!rc && (tot_best < 0.0 || tot < tot_best)) {
            tot_best = tot;
            b0_best = b0;
        }
    }
    cudaStreamSynchronize(h->stream);
    cudaFree(buf);
    if (rc) return rc;
    if (b0_best == 0) return SEV_ERR_UNSUPPORTED;
    out->bucket = tune_bucket(n);
    out->prec = prec;
    out->b0 = b0_best;
    for (int k = 0; k < kTuneWidths; ++k) out->next[k] = next[k];
    if (best_ms) *best_ms = tot_best;
    return SEV_OK;
}

}  // namespace sev

extern "C" int sev_autotune(sev_handle h, int n, int prec, int b0, int *bands, int max_bands, int *nbands,
                            double *best_ms) {
    using namespace sev;
    if (!h) return -1;
    if (n < 0) return -2;
    if (prec != SEV_FP64 && prec != SEV_MIXED) return -3;
    if (b0 < 0) return -4;
    if (!bands) return -5;
    if (max_bands < 1) return -6;
    if (!nbands) return -7;
    *nbands = 0;
    if (n < 4) return SEV_OK;  // nothing to reduce
    if (cudaSetDevice(h->device) != cudaSuccess) return SEV_ERR_CUDA;
    TunedBands t;
    const int rc = prec == SEV_FP64 ? autotune_t<double>(h, n, prec, b0, &t, best_ms)
                                    : autotune_t<float>(h, n, prec, b0, &t, best_ms);
    if (rc) return rc;
    // with one b0 given, the bucket's choice of b0 stays what it was (none:
    // b0 = 0 calls keep the library's default), only the stage table changes
    const TunedBands *old = tuned_for(h, n, prec);
    if (b0 > 0) t.b0 = old ? old->b0 : 0;
    store_tuned(h, t);
    tune_cache_append(h, t);
    int sched[16];
    const int ns = tuned_schedule(t, b0 > 0 ? b0 : t.b0, sched, 16);
    if (ns == 0) return SEV_ERR_UNSUPPORTED;
    if (ns > max_bands) return -6;
    for (int k = 0; k < ns; ++k) bands[k] = sched[k];
    *nbands = ns;
    return SEV_OK;
}
