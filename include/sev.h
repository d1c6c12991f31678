/*
 * sev.h -- C ABI of the GB300 (sm_103a) symmetric eigenvalue library.
 *
 * The library computes the eigenvalues of a dense real symmetric matrix by
 * the successive band reduction of Solomonik, Ballard, Demmel and Hoefler,
 * "A communication-avoiding parallel algorithm for the symmetric eigenvalue
 * problem" (arXiv 1604.03703), on one GPU:
 *
 *   full-to-band    Algorithm 4.1 (tree QR of each panel, Algorithm 3.2;
 *                   compact-WY by Householder reconstruction, Cor. 3.7;
 *                   two-sided trailing update, Eq. 4.1)
 *   band-to-band    Algorithm 4.2 (bulge chasing, b -> h), repeated down
 *                   to the tridiagonal as in Algorithm 4.3
 *   tridiag_bisect  eigenvalues of the final tridiagonal by Sturm-count
 *                   bisection (the last step of Algorithm 4.3, where the
 *                   tridiagonal's eigenvalues are taken as the result)
 *
 * Conventions for every entry point:
 *  - Matrices are column-major.  Only the LOWER triangle of a symmetric input
 *    is read (the paper's algorithms keep A in full storage, Sec. 4; the
 *    upper triangle is never touched here).
 *  - Pointers are DEVICE pointers unless a name ends in _host.  The caller
 *    owns every buffer it passes; the library never frees them.
 *  - Inputs named A / AB are overwritten (LAPACK-style workspace semantics).
 *  - Calls are asynchronous on the handle's stream (sev_set_stream); a
 *    return of SEV_OK means the work was enqueued.  Errors detected on the
 *    device (non-finite input, a wait that timed out, a bisection that did
 *    not converge) are latched in the handle and returned by
 *    sev_get_error().
 *  - Precision: SEV_FP64 -- data double, all arithmetic FP64.
 *    SEV_MIXED -- data float (FP32); the trailing update runs as BF16x3
 *    split products on the tensor cores with FP32 accumulation; Householder
 *    norms, tau and beta are FP64-accurate (sums of squares accumulated
 *    error-free as pairs of floats, the scalars evaluated in pair-float
 *    arithmetic; they equal the FP64 evaluation rounded to float, which
 *    sev_diag_house_scalars lets a caller check); the Sturm recurrence of
 *    the bisection is FP64; eigenvalues are returned as double.
 *  - Return codes: SEV_OK = 0; a negative value -i means argument i (1-based,
 *    the handle counts as argument 1) is invalid; positive values are the
 *    SEV_ERR_* codes below.
 *
 * Band storage ("packed lower band"): a symmetric matrix with half-bandwidth
 * b (a_ij = 0 for |i - j| > b) is held in an ldab x n column-major array AB
 * with AB[d + j*ldab] = A(j + d, j) for 0 <= d < ldab and j + d < n; the
 * remaining entries are zero.  Band-to-band needs ldab >= 2b because the
 * bulges of Algorithm 4.2 reach 2b-1 below the diagonal.
 */
#ifndef SEV_H
#define SEV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sev_ctx *sev_handle;

typedef enum {
    SEV_FP64 = 0,  /* double data, FP64 arithmetic throughout */
    SEV_MIXED = 1  /* float data, BF16x3 tensor-core update, FP64-accurate norms/tau/beta, FP64 Sturm */
} sev_prec;

enum {
    SEV_OK = 0,
    SEV_ERR_NONFINITE = 1,  /* input holds NaN or Inf */
    SEV_ERR_NOCONV = 2,     /* bisection hit its iteration cap */
    SEV_ERR_TIMEOUT = 3,    /* a device-side wait hit its iteration cap */
    SEV_ERR_CUDA = 4,       /* a CUDA runtime call failed */
    SEV_ERR_WORKSPACE = 5,  /* caller workspace too small / allocation failed */
    SEV_ERR_UNSUPPORTED = 6, /* parameter combination not supported */
    SEV_ERR_INTERNAL = 7     /* a kernel's self-check found an index outside its buffer */
};

/* Create a handle bound to CUDA device `device`; the stream defaults to the
 * legacy default stream.  Returns SEV_ERR_CUDA if the device is unusable. */
int sev_create(sev_handle *handle, int device);

/* Destroy the handle and the workspace it allocated itself.  Does not
 * synchronise; the caller must not destroy a handle with work in flight. */
int sev_destroy(sev_handle handle);

/* Set the CUDA stream (a cudaStream_t passed as void*) for later calls. */
int sev_set_stream(sev_handle handle, void *stream);

/* Bytes of device workspace that sev_eigvalsh(n, b0, prec) needs. */
int sev_workspace_query(sev_handle handle, int n, int b0, int prec, size_t *bytes);

/* Give the handle a caller-owned device workspace of `bytes` bytes (at least
 * 256-byte aligned).  Later calls use it instead of allocating; calls whose
 * workspace need exceeds it return SEV_ERR_WORKSPACE.  NULL/0 reverts to
 * library-owned workspace (allocated on demand with cudaMalloc). */
int sev_set_workspace(sev_handle handle, void *workspace, size_t bytes);

/*
 * Eigenvalues of the symmetric n x n matrix A (Algorithm 4.3):
 * full-to-band to half-bandwidth b0, band-to-band stages down to the
 * tridiagonal, bisection.  The stage widths are the ones sev_eigvalsh_bands
 * reports: those sev_autotune chose on this handle for the bucket of n and
 * prec, else the fixed rule of sev_band_schedule (e.g. 128 -> 32 -> 16 -> 1).
 *   A      device, n x n, leading dimension lda >= max(1, n); double for
 *          SEV_FP64, float for SEV_MIXED; lower triangle read, overwritten.
 *   b0     first half-bandwidth, 1 <= b0 (values >= n-1 skip full-to-band);
 *          0 picks the tuned b0 for (n, prec) if sev_autotune set one, else
 *          the library's default.
 *   eigs   device, n doubles, ascending on completion.
 * Bisection tolerance: relative 1e-14 (SEV_FP64) or 1e-9 (SEV_MIXED) of the
 * Gershgorin bound of the tridiagonal.
 * A NaN or Inf in A's lower triangle latches SEV_ERR_NONFINITE; the
 * reductions still run over it (their work does not depend on the values),
 * the bisection is skipped and eigs receives NaNs.
 */
int sev_eigvalsh(sev_handle handle, int n, void *A, int lda, int b0, int prec, double *eigs);

/* sev_eigvalsh with HOST buffers: copies A_host (n x n, lda, float or double
 * by prec, not modified) to device workspace, runs sev_eigvalsh, copies the
 * eigenvalues back to eigs_host and synchronises the stream.  Page-locked
 * host memory makes the copies asynchronous DMA. */
int sev_eigvalsh_host(sev_handle handle, int n, const void *A_host, int lda, int b0, int prec,
                      double *eigs_host);

/*
 * Full-to-band reduction (Algorithm 4.1, run right-looking): per panel of b
 * columns, tree QR of the trailing N x b panel (Algorithm 3.2), Householder
 * reconstruction of (U, T) (Cor. 3.7), W = A22 U, V from the V_1 formula,
 * A22 <- A22 + U V^T + V U^T (Eq. 4.1), band block <- S R.
 *   A     device, n x n (lda), lower triangle read; on return A's lower
 *         triangle holds the band matrix (exact zeros below the band).
 *         A NaN or Inf in it latches SEV_ERR_NONFINITE (the reduction still
 *         runs; its output is then meaningless).
 *   b     half-bandwidth >= 1 (b >= n-1 only copies the band).
 *   AB    device, packed lower band, ldab >= b+1; receives the band matrix.
 */
int sev_full_to_band(sev_handle handle, int n, void *A, int lda, int b, int prec, void *AB, int ldab);

/*
 * Band-to-band reduction b -> h (Algorithm 4.2) in place on packed band
 * storage.  Requires h >= 1, h < b, b % h == 0, ldab >= 2b.  Entries of AB
 * at distance > b from the diagonal must be zero on entry; on return the
 * band has half-bandwidth h and entries beyond it are zero.  Chases run as a
 * persistent wavefront in which chase (i, j) starts once chase (i-1, j+2)
 * and (i, j-1) are complete.
 */
int sev_band_to_band(sev_handle handle, int n, void *AB, int ldab, int b, int h, int prec);

/*
 * All eigenvalues of the symmetric tridiagonal T with diagonal d[0..n-1] and
 * off-diagonal e[0..n-2] (device, double), ascending, into eigs (device,
 * n doubles), by bisection on the Sturm count (sign changes of the leading
 * principal minors of T - xI, evaluated on T scaled by the power of two
 * that brings its Gershgorin bound into [0.5, 1)) from the widened
 * Gershgorin interval, until hi - lo <= max(rtol*max(|lo|,|hi|),
 * rtol*||T||_G) (rtol > 0).  T = 0 gives exact zeros.
 */
int sev_tridiag_bisect(sev_handle handle, int n, const double *d, const double *e, double rtol,
                       double *eigs);

/*
 * Allocation-free bisection (no counterpart in the paper; a service for
 * callers that cannot allocate device memory -- e.g. code that runs inside a
 * framework owning every device allocation, or a latency-critical path that
 * must not pay cudaMalloc's implicit device synchronisation).
 * Same result as sev_tridiag_bisect, bit for bit, with no handle and no
 * allocation: its scratch is a fixed device array inside the library of
 * (65536 + 8) doubles (~512 KiB), resident on every device that loads the
 * library until the process exits.
 *   n       0 <= n <= 65536; larger n returns -1
 *   d, e    device, n and n-1 doubles;  eigs: device, n doubles, ascending
 *   rtol    1e-16 <= rtol < 1 (the bisection then always converges well
 *           inside its iteration cap, so no device-side status is needed)
 *   stream  cudaStream_t (as void*) on which the kernels are enqueued
 * Every call made outside stream capture looks up the array's device
 * address on the current device (so the address stays right after a
 * cudaDeviceReset); a call inside a capture uses the address found by the
 * last call outside one, so make the first call on each device before any
 * stream capture.  Every call on a device shares the one array, which keeps
 * the last call's contents: calls whose kernels overlap on the GPU
 * (different streams without ordering between them) race and must be
 * serialised by the caller.
 */
int sev_tridiag_bisect_static(int n, const double *d, const double *e, double rtol, double *eigs, void *stream);

/*
 * Batched eigenvalues of `count` independent symmetric matrices (no
 * counterpart in the paper, which treats one matrix; for workloads of many
 * small uneven matrices such as a sequence of SCF eigenproblems).  Each
 * matrix follows the same path as sev_eigvalsh: full-to-band with band
 * width b (Algorithm 4.1; per panel a one-leaf tree QR, Algorithm 3.2, the
 * compact-WY T and the update of Eq. 4.1), b -> 1 (Algorithm 4.2), Sturm
 * bisection (rtol 1e-14 FP64, 1e-9 mixed).
 *
 * A plan fixes the batch: host arrays n[count], lda[count] (lda[i] >= n[i]),
 * A[count] (device pointers to the matrices; float for SEV_MIXED, double for
 * SEV_FP64; lower triangle read, both triangles overwritten) and
 * eigs[count] (device pointers, n[i] doubles each, ascending on
 * completion).  The host arrays are read during sev_batch_plan_create only;
 * the device buffers must stay valid while the plan is run.
 *   b      band width of the batched kernel: 4, 8, 16 or 32 (32: SEV_MIXED
 *          only); 0 takes the value sev_batch_autotune chose on this handle
 *          for prec, else 16 (SEV_MIXED) or 8 (SEV_FP64).
 * Matrices with n <= 1024 whose path fits one CTA's shared memory run in ONE
 * persistent launch (each CTA takes matrices largest first from a device
 * queue); the others run through sev_eigvalsh one after another on the
 * handle's stream.  Plan creation allocates the descriptor table and
 * reserves the handle's workspace and synchronises; sev_batch_run only
 * enqueues work (no allocation, no host synchronisation) and may be
 * captured in a CUDA graph when every matrix runs in the batched launch
 * (sev_batch_plan_info reports large_count == 0).  Errors as sev_eigvalsh.
 */
typedef struct sev_batch_s *sev_batch_plan;
int sev_batch_plan_create(sev_handle handle, int count, const int *n, const int *lda, void *const *A,
                          double *const *eigs, int b, int prec, sev_batch_plan *plan);
int sev_batch_run(sev_handle handle, sev_batch_plan plan);
int sev_batch_plan_destroy(sev_batch_plan plan);
/* Band width, number of matrices in the batched launch, number run one by one. */
int sev_batch_plan_info(sev_batch_plan plan, int *b, int *small_count, int *large_count);
/* create + run + synchronise + destroy. */
int sev_eigvalsh_batched(sev_handle handle, int count, const int *n, const int *lda, void *const *A, int b, int prec,
                         double *const *eigs);
/*
 * Autotuner of the batched band width: times the batched launch on
 * synthetic matrices with a strided sample (at most 4096) of the sizes n[]
 * for every supported b, stores the fastest in the handle (used when a plan
 * passes b = 0) and returns it in *b_best (0 if no size fits the batched
 * kernel).  Allocates and synchronises.
 */
int sev_batch_autotune(sev_handle handle, int count, const int *n, int prec, int *b_best);

/*
 * The band widths sev_eigvalsh goes through for an n x n matrix (host only,
 * no device work): bands[0] = b0 (0 picks the default for (n, prec), and
 * b0 is clamped to n - 1), then every band-to-band stage's target width, the
 * last being 1 (Algorithm 4.3 with the stage widths of this library: a band
 * of width <= 16 goes straight to 1, one of 128 or more first to 32, other
 * multiples of 16 to 16).  Returns the number of widths written (0 for
 * n <= 1) or -5 if max_bands is too small; other negative values name the
 * invalid argument (n = 1, b0 = 2, prec = 3, bands = 4).
 */
int sev_band_schedule(int n, int b0, int prec, int *bands, int max_bands);

/*
 * Autotuner of the band widths sev_eigvalsh goes through (Algorithm 4.3
 * reduces to a first half-bandwidth b0, then through narrower bands to the
 * tridiagonal; the paper fixes neither b0 nor the stage widths for a
 * machine, and Algorithm 4.2 holds for any h dividing b).  On this handle's
 * GPU, at the order n and precision prec, it times once each: the
 * full-to-band reduction for every candidate b0 (32, 64 and 128 when
 * b0 = 0; only b0 otherwise -- a power of two up to 128), and every band
 * stage b -> h (powers of two, h | b) the kernels support; the cheapest
 * stage path from each width down to 1 follows by dynamic programming over
 * the measured costs.  The result is kept in the handle for the bucket of
 * n (orders within a factor sqrt 2) and prec: later sev_eigvalsh calls in
 * that bucket run the tuned stage path from their b0, and calls with
 * b0 = 0 take the tuned b0 (tuned only when this call had b0 = 0).  With
 * the environment variable SEV_TUNE_CACHE naming a file, the result is also
 * appended there, keyed by the GPU's name, and read back by sev_create.
 *   bands      host, receives the widths from b0 (b0 as given, or the tuned
 *              one) down to 1; max_bands entries available
 *   nbands     host, receives the number of widths written (0 for n < 4)
 *   best_ms    host, may be NULL: the predicted milliseconds of the
 *              reductions (full-to-band plus band stages) along that path
 * Returns SEV_OK, -i for invalid argument i (-6: max_bands too small for
 * the path), or an SEV_ERR_* code.  Allocates an n x n test matrix and the
 * workspace, and synchronises the handle's stream.
 */
int sev_autotune(sev_handle handle, int n, int prec, int b0, int *bands, int max_bands, int *nbands,
                 double *best_ms);

/* The band widths sev_eigvalsh(handle, n, ., ., b0, prec, .) runs (host
 * only, no device work): as sev_band_schedule, but with this handle's
 * autotuned b0 and stage widths where sev_autotune set them.  Returns the
 * number of widths, -6 if max_bands is too small, or -i for invalid
 * argument i. */
int sev_eigvalsh_bands(sev_handle handle, int n, int b0, int prec, int *bands, int max_bands);

/* Copy the diagonal and first subdiagonal of a packed band (float or double
 * by prec) into FP64 device arrays d (n) and e (n-1). */
int sev_band_tridiag_extract(sev_handle handle, int n, const void *AB, int ldab, int prec, double *d,
                             double *e);

/*
 * Self-check of the mixed form's Householder scalars (no counterpart in the
 * paper).  For count inputs alpha[i] (the leading entry, float) and the sum
 * of squares of the rest as an unevaluated pair ssq_hi[i] + ssq_lo[i]
 * (device floats), writes (tau, beta, 1/(alpha - beta)) as evaluated by the
 * library's pair-float routine to out_pairfloat[3i..3i+2] and as evaluated
 * in FP64 and rounded to float to out_fp64[3i..3i+2] (device), on `stream`.
 */
int sev_diag_house_scalars(int count, const float *alpha, const float *ssq_hi, const float *ssq_lo,
                           float *out_pairfloat, float *out_fp64, void *stream);

/* Synchronise the handle's stream and return (and clear) the first error
 * latched by device code since the last call, or SEV_OK. */
int sev_get_error(sev_handle handle);

/*
 * Time limit of every device-side wait of this handle's kernels (a sweep
 * waiting on its predecessor's progress, a ring slot, an mbarrier, a grid
 * barrier), in SM clock cycles; 0 restores the default of 4e9 (~2 s at
 * 2 GHz).  A wait that runs out latches SEV_ERR_TIMEOUT and its kernel
 * returns without finishing (the context stays usable).  Synchronises the
 * handle's stream first.  A short limit is a watchdog for tests: work that
 * legitimately waits longer than it then fails.  Negative cycles return -2.
 */
int sev_set_wait_limit(sev_handle handle, long long cycles);

/* Human-readable text of a return code. */
const char *sev_status_string(int code);

/*
 * Per-kernel timing for roofline reports.  Every launch of a library kernel
 * whose id k has bit k set in `mask` is bracketed by CUDA events on the
 * handle's stream; totals are read back per kernel id (see sev_kernel_name).
 * mask = 0 disables timing (the default); ~0ULL times every kernel.
 */
int sev_set_kernel_timing(sev_handle handle, unsigned long long mask);
/* Number of kernel ids. */
int sev_kernel_count(void);
/* Name of kernel id k (0 <= k < sev_kernel_count()). */
const char *sev_kernel_name(int k);
/* Synchronises; total milliseconds and launch count of kernel id k since
 * timing was enabled or last reset; reset != 0 clears the totals after. */
int sev_kernel_time(sev_handle handle, int k, double *total_ms, long *launches, int reset);

#ifdef __cplusplus
}
#endif

#endif /* SEV_H */
