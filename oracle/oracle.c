/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the symmetric eigenvalue path
 * of Solomonik, Ballard, Demmel, Hoefler, "A communication-avoiding parallel
 * algorithm for the symmetric eigenvalue problem" (arXiv 1604.03703).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no code, header, table or
 * helper with the CUDA library (paper_1604_03703_gb300/csrc).
 *
 * Conventions (all functions): column-major, 0-based indices, FP64, full
 * symmetric storage unless stated.  No blocking, fusion or reordering beyond
 * what the cited definition or algorithm states.  Compile with
 * -ffp-contract=off so that no multiply-add is fused behind our back.
 *
 * Contents
 *   orc_house            Householder reflector, "always reflect" sign rule
 *                        (Sec. 3.2, Lemma 3.4: Householder form Q = I - U T U^T)
 *   orc_tridiagonalize   unblocked Householder tridiagonalisation: Algorithm
 *                        4.1 with b = 1, the direct reduction of Sec. 4
 *   orc_sturm_count      Sturm count of a symmetric tridiagonal by LDL^T
 *                        pivots (cross-check of the minors count)
 *   orc_sturm_minors     Sturm count by the leading principal minors on the
 *                        exactly rescaled matrix (the count the bisection uses)
 *   orc_bisect           bisection on the minors count, eigenvalues ascending
 *                        (the final eigenvalue step of Algorithm 4.3)
 *   orc_eigvalsh         orc_tridiagonalize + orc_bisect (Algorithm 4.3's result)
 *   orc_jacobi           cyclic Jacobi (independent cross-check, n <= ~32)
 *   orc_inertia          LDL^T inertia of A - xI in long double (Sylvester)
 *   orc_band_inertia     the same for a packed band matrix, O(n b^2)
 *   orc_panel_qr         Householder QR of a panel + forward compact-WY T
 *   orc_full_to_band     Algorithm 4.1, right-looking, with the Eq. 4.1 update
 *   orc_band_to_band     Algorithm 4.2 on dense storage, with the readings
 *                        (A5-A8) of the index sets stated at the function
 */
#include <float.h>
#include <stdint.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

static double sgn1(double a) { return a < 0.0 ? -1.0 : 1.0; } /* sgn(0) = +1 */

/*
 * Householder reflector H = I - tau v v^T with v[0] = 1 such that
 * H x = beta e_1  (Sec. 3.2 / Lemma 3.4, Householder representation).
 * Sign rule ("always reflect"): beta = -sgn(alpha) ||x||, sgn(0) = +1,
 * tau = (beta - alpha)/beta in [1, 2]; a zero vector gives tau = beta = 0.
 * On return x[1..m-1] holds v[1..m-1] (x[0] is left unchanged).
 * The norm is computed with max-scaling so it neither overflows nor
 * underflows.
 */
double orc_house(int m, double *x, int incx, double *beta_out)
{
    double alpha = x[0];
    double scale = fabs(alpha);
    for (int i = 1; i < m; ++i) {
        double a = fabs(x[(size_t)i * incx]);
        if (a > scale) scale = a;
    }
    if (scale == 0.0) {
        *beta_out = 0.0;
        return 0.0;
    }
    double ssq = 0.0;
    for (int i = 0; i < m; ++i) {
        double t = x[(size_t)i * incx] / scale;
        ssq += t * t;
    }
    double nrm = scale * sqrt(ssq);
    double beta = -sgn1(alpha) * nrm;
    double tau = (beta - alpha) / beta;
    double inv = 1.0 / (alpha - beta);
    for (int i = 1; i < m; ++i) x[(size_t)i * incx] *= inv;
    *beta_out = beta;
    return tau;
}

/*
 * Unblocked Householder tridiagonalisation of the symmetric A (lower
 * triangle read and updated; the strict upper triangle is never touched).
 * This is the direct reduction that Sec. 4 describes as the b = 1 case of
 * the full-to-band reduction: for column j, a reflector annihilates
 * A[j+2:n, j]; the trailing matrix gets the two-sided update
 * A22 <- H A22 H = A22 - v w^T - w v^T with p = tau A22 v and
 * w = p - (tau/2)(p^T v) v (Eq. 4.1 with one Householder vector).
 * Output: d[0..n-1] diagonal, e[0..n-2] subdiagonal.  A is overwritten.
 * nsteps < 0 performs all n-2 steps; otherwise only the first nsteps
 * (d and e are then only partially meaningful; used to time a sample).
 */
void orc_tridiagonalize(int n, double *A, int lda, double *d, double *e, int nsteps)
{
    int last = n - 2; /* steps j = 0 .. n-3 */
    if (nsteps >= 0 && nsteps < last) last = nsteps;
    double *v = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *p = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#ifdef _OPENMP
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#endif
    for (int j = 0; j < last; ++j) {
        int m = n - j - 1; /* length of x = A[j+1:n, j] */
        double *x = &A[IDX(j + 1, j, lda)];
        double beta;
        double tau = orc_house(m, x, 1, &beta);
        v[0] = 1.0;
        for (int i = 1; i < m; ++i) v[i] = x[i];
        /* the column now holds (beta, 0, ..., 0) */
        x[0] = beta;
        for (int i = 1; i < m; ++i) x[i] = 0.0;
        e[j] = beta;
        if (tau == 0.0) continue;
        /* p = tau * A22 v, A22 = A[j+1:n, j+1:n] read from its lower triangle */
        double *A22 = &A[IDX(j + 1, j + 1, lda)];
        for (int i = 0; i < m; ++i) p[i] = 0.0;
#ifndef _OPENMP
        for (int c = 0; c < m; ++c) {
            double vc = v[c];
            double acc = A22[IDX(c, c, lda)] * vc;
            double pc = 0.0;
            for (int r = c + 1; r < m; ++r) {
                double a = A22[IDX(r, c, lda)];
                p[r] += a * vc;
                pc += a * v[r];
            }
            p[c] += acc + pc;
        }
#else
        /* The same sums in the same order per output, with independent
         * outputs on separate cores: p[r] first gathers A22[r, c] v_c for
         * c = 0 .. r-1 in increasing c, then adds acc_r + pc_r. */
        {
#pragma omp parallel for schedule(dynamic, 32)
            for (int c = 0; c < m; ++c) {
                double pc = 0.0;
                for (int r = c + 1; r < m; ++r) pc += A22[IDX(r, c, lda)] * v[r];
                tmp[c] = A22[IDX(c, c, lda)] * v[c] + pc;
            }
#pragma omp parallel for schedule(dynamic, 1)
            for (int r0 = 0; r0 < m; r0 += 64) {
                int r1 = r0 + 64 < m ? r0 + 64 : m;
                for (int c = 0; c < r1 - 1; ++c) {
                    double vc = v[c];
                    int rs = c + 1 > r0 ? c + 1 : r0;
                    for (int r = rs; r < r1; ++r) p[r] += A22[IDX(r, c, lda)] * vc;
                }
                for (int r = r0; r < r1; ++r) p[r] += tmp[r];
            }
        }
#endif
        for (int i = 0; i < m; ++i) p[i] *= tau;
        double ptv = 0.0;
        for (int i = 0; i < m; ++i) ptv += p[i] * v[i];
        double half = 0.5 * tau * ptv;
        for (int i = 0; i < m; ++i) p[i] -= half * v[i]; /* p now holds w */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
        for (int c = 0; c < m; ++c) {
            double vc = v[c], wc = p[c];
            for (int r = c; r < m; ++r)
                A22[IDX(r, c, lda)] -= v[r] * wc + p[r] * vc;
        }
    }
    for (int i = 0; i < n; ++i) d[i] = A[IDX(i, i, lda)];
    if (n >= 2 && (nsteps < 0 || nsteps >= n - 2)) e[n - 2] = A[IDX(n - 1, n - 2, lda)];
    free(v);
    free(p);
#ifdef _OPENMP
    free(tmp);
#endif
}

/*
 * pivmin for the Sturm recurrence: the smallest pivot magnitude allowed,
 * DBL_MIN * max(1, max_i e_i^2) (the guard used by LAPACK's bisection).
 */
double orc_pivmin(int n, const double *e)
{
    double m = 1.0;
    for (int i = 0; i + 1 < n; ++i) {
        double t = e[i] * e[i];
        if (t > m) m = t;
    }
    return DBL_MIN * m;
}

/*
 * Sturm count: number of eigenvalues of the symmetric tridiagonal T(d, e)
 * strictly less than x, as the number of negative pivots of the LDL^T
 * factorisation of T - xI:  q_0 = d_0 - x,  q_i = (d_i - x) - e2_{i-1}/q_{i-1},
 * with |q_i| < pivmin replaced by -pivmin.  e2[i] = e[i]*e[i] is passed in
 * precomputed so that every caller rounds it once, the same way.
 */
int orc_sturm_count(int n, const double *d, const double *e2, double x, double pivmin)
{
    int c = 0;
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++c;
    for (int i = 1; i < n; ++i) {
        q = (d[i] - x) - e2[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0.0) ++c;
    }
    return c;
}

/*
 * Gershgorin interval of T(d, e), widened by 2 n eps ||T|| + 4 pivmin so the
 * floating-point Sturm count is 0 at the left end and n at the right end.
 * Returns tnorm = max(|gl|, |gu|) of the unwidened interval.
 */
double orc_gershgorin(int n, const double *d, const double *e, double pivmin,
                      double *gl_out, double *gu_out)
{
    double gl = d[0], gu = d[0];
    for (int i = 0; i < n; ++i) {
        double r = 0.0;
        if (i > 0) r += fabs(e[i - 1]);
        if (i + 1 < n) r += fabs(e[i]);
        if (d[i] - r < gl) gl = d[i] - r;
        if (d[i] + r > gu) gu = d[i] + r;
    }
    double tnorm = fabs(gl) > fabs(gu) ? fabs(gl) : fabs(gu);
    double pad = 2.0 * (double)n * DBL_EPSILON * tnorm + 4.0 * pivmin;
    *gl_out = gl - pad;
    *gu_out = gu + pad;
    return tnorm;
}

/*
 * Exact power-of-two scaling of T(d, e) for the bisection: s is chosen so
 * that the Gershgorin bound tnorm = max(|gl|, |gu|) of T scaled by 2^-s lies
 * in [0.5, 1) (s = 0 for the zero matrix).  Returns s; sc = 2^-s.  Scaling by
 * a power of two is exact (barring underflow) and scales every eigenvalue by
 * the same factor, so the bisection runs on the scaled matrix and its
 * results are scaled back exactly.
 */
static int bis_scale(int n, const double *d, const double *e, double *gl_out, double *gu_out, double *tnorm_out)
{
    double gl = d[0], gu = d[0];
    for (int i = 0; i < n; ++i) {
        double r = 0.0;
        if (i > 0) r += fabs(e[i - 1]);
        if (i + 1 < n) r += fabs(e[i]);
        if (d[i] - r < gl) gl = d[i] - r;
        if (d[i] + r > gu) gu = d[i] + r;
    }
    double tnorm = fabs(gl) > fabs(gu) ? fabs(gl) : fabs(gu);
    int s = 0;
    if (tnorm > 0.0) (void)frexp(tnorm, &s); /* tnorm = m 2^s, m in [0.5, 1) */
    *gl_out = gl;
    *gu_out = gu;
    *tnorm_out = tnorm;
    return s;
}

static double pow2(int k) /* exact 2^k for -1022 <= k <= 1023 */
{
    uint64_t bits = (uint64_t)(1023 + k) << 52;
    double f;
    memcpy(&f, &bits, sizeof f);
    return f;
}

/*
 * Sturm count by the leading principal minors of T - xI (Sturm's theorem:
 * the number of eigenvalues below x is the number of sign changes in
 * p_0 = 1, p_1, ..., p_n):  p_1 = d_0 - x,
 *   p_{i+1} = (d_i - x) p_i - e_{i-1}^2 p_{i-1},
 * the division-free form of the LDL^T pivot count (q_i = p_i / p_{i-1}).
 * Works on the scaled matrix: d_i - x is formed as fma(d_i, sc, -x) (one
 * rounding of the exactly scaled entry minus x) and e2s holds the squared
 * scaled off-diagonal; each step is u = e2s_{i-1} p_{i-1} followed by
 * p_{i+1} = fma(d_i - x, p_i, -u).  A minor equal to zero takes the sign
 * opposite to its predecessor (it counts as a change, as a zero pivot does
 * under the pivmin rule).  Whenever |p_i| leaves [2^-256, 2^256] the pair
 * (p_{i-1}, p_i) is rescaled by the power of two 2^k, k = clamp(-exponent,
 * -512, 512), bringing p_i to [1, 2): signs are unchanged and nothing
 * overflows for a scaled matrix (|d_i - x| <= 2, e2s <= 1).
 */
int orc_sturm_minors(int n, const double *d, const double *e2s, double sc, double x)
{
    double a = 1.0, b = fma(d[0], sc, -x);
    int neg = b <= 0.0; /* p_0 = 1 > 0: a zero p_1 counts as negative */
    int c = neg;
    for (int i = 1; i < n; ++i) {
        double t = fma(d[i], sc, -x);
        double u = e2s[i - 1] * a;
        double p = fma(t, b, -u);
        int pn = (p < 0.0) || (p == 0.0 && !neg);
        c += pn != neg;
        neg = pn;
        a = b;
        b = p;
        uint64_t bits;
        memcpy(&bits, &b, sizeof bits);
        int ex = (int)((bits >> 52) & 0x7FF);
        if (ex > 1023 + 256 || (ex < 1023 - 256 && b != 0.0)) {
            int k = 1023 - ex;
            if (k > 512) k = 512;
            if (k < -512) k = -512;
            double f = pow2(k);
            a *= f;
            b *= f;
        }
    }
    return c;
}

/* The minors count of T(d, e) at x for unscaled inputs (scales first). */
int orc_sturm_count_minors(int n, const double *d, const double *e, double x)
{
    double gl, gu, tn;
    int s = bis_scale(n, d, e, &gl, &gu, &tn);
    double sc = pow2(-s);
    double *e2s = (double *)malloc(sizeof(double) * (size_t)(n > 1 ? n : 1));
    for (int i = 0; i + 1 < n; ++i) {
        double es = e[i] * sc;
        e2s[i] = es * es;
    }
    int c = orc_sturm_minors(n, d, e2s, sc, x * sc);
    free(e2s);
    return c;
}

/*
 * Bisection for every eigenvalue of T(d, e), ascending (index k = 0..n-1 is
 * the (k+1)-th smallest), on the matrix scaled by 2^-s (bis_scale):
 * [lo, hi] = the scaled Gershgorin interval widened by 2 n eps tnorm + 2^-1000;
 * mid = 0.5*(lo + hi); minors count(mid) >= k+1 -> hi = mid, else lo = mid;
 * stop when hi - lo <= max(rtol*max(|lo|,|hi|), rtol*tnorm), when mid no
 * longer splits the interval, or after maxit steps; eig = 2^s * 0.5*(lo+hi).
 * T = 0 (a zero Gershgorin bound) gives exact zeros.  Returns the number
 * of eigenvalues that hit maxit before converging.
 */
int orc_bisect_range(int n, const double *d, const double *e, double rtol, int maxit, int k0, int k1,
                     double *eigs);

int orc_bisect(int n, const double *d, const double *e, double rtol, int maxit, double *eigs)
{
    return orc_bisect_range(n, d, e, rtol, maxit, 0, n, eigs);
}

/* Bisection for eigenvalue indices k0 <= k < k1 only (eigs[k - k0]); the
 * same per-index procedure as orc_bisect (used to time a bounded sample). */
int orc_bisect_range(int n, const double *d, const double *e, double rtol, int maxit, int k0, int k1,
                     double *eigs)
{
    if (n <= 0) return 0;
    if (n == 1) {
        if (k0 == 0 && k1 > 0) eigs[0] = d[0];
        return 0;
    }
    double gl, gu, tnorm;
    int s = bis_scale(n, d, e, &gl, &gu, &tnorm);
    if (tnorm == 0.0) { /* a zero Gershgorin bound means T = 0 */
        for (int k = k0; k < k1; ++k) eigs[k - k0] = 0.0;
        return 0;
    }
    double sc = pow2(-s), up = pow2(s);
    double *e2s = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i + 1 < n; ++i) {
        double es = e[i] * sc;
        e2s[i] = es * es;
    }
    e2s[n - 1] = 0.0;
    gl *= sc;
    gu *= sc;
    tnorm *= sc;
    double pad = 2.0 * (double)n * DBL_EPSILON * tnorm + 0x1p-1000;
    gl -= pad;
    gu += pad;
    double atol = rtol * tnorm;
    int noconv = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : noconv)
#endif
    for (int k = k0; k < k1; ++k) {
        double lo = gl, hi = gu;
        int it = 0;
        for (;;) {
            double w = hi - lo;
            double mag = fabs(lo) > fabs(hi) ? fabs(lo) : fabs(hi);
            double tol = rtol * mag;
            if (atol > tol) tol = atol;
            if (w <= tol) break;
            if (it >= maxit) {
                ++noconv;
                break;
            }
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (orc_sturm_minors(n, d, e2s, sc, mid) >= k + 1)
                hi = mid;
            else
                lo = mid;
            ++it;
        }
        eigs[k - k0] = (0.5 * (lo + hi)) * up;
    }
    free(e2s);
    return noconv;
}

/*
 * Textbook Sturm bisection on the LDL^T pivot count (the final eigenvalue
 * step of Algorithm 4.3, by the method the eigenvalue step is defined with:
 * bisection on Sturm counts), written without any of the rescaling,
 * division-free or exponent tricks of orc_bisect, as an independent second
 * definition of the same result:
 *   pivmin = orc_pivmin(e);  [lo, hi] = orc_gershgorin(d, e) (unscaled,
 *   widened by 2 n eps ||T|| + 4 pivmin);  count(x) = orc_sturm_count (q_0 =
 *   d_0 - x, q_i = (d_i - x) - e_{i-1}^2 / q_{i-1}, |q_i| < pivmin -> -pivmin,
 *   negative q counted);  mid = (lo + hi)/2;  count(mid) >= k+1 -> hi = mid
 *   else lo = mid;  stop when hi - lo <= max(rtol max(|lo|,|hi|), rtol ||T||_G)
 *   or after maxit steps (or once mid no longer splits the interval);
 *   eigenvalue k = (lo + hi)/2.
 * For each of the nidx indices idx[m] (0-based, the (idx[m]+1)-th smallest)
 * the result goes to eigs[m].  Returns the number that hit maxit.
 */
int orc_bisect_ldlt(int n, const double *d, const double *e, double rtol, int maxit, int nidx, const int *idx,
                    double *eigs)
{
    if (n <= 0) return 0;
    if (n == 1) {
        for (int m = 0; m < nidx; ++m) eigs[m] = d[0];
        return 0;
    }
    double *e2 = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i + 1 < n; ++i) e2[i] = e[i] * e[i];
    e2[n - 1] = 0.0;
    double pm = orc_pivmin(n, e);
    double gl, gu;
    double tnorm = orc_gershgorin(n, d, e, pm, &gl, &gu);
    double atol = rtol * tnorm;
    int noconv = 0;
    for (int m = 0; m < nidx; ++m) {
        int k = idx[m];
        double lo = gl, hi = gu;
        for (int it = 0;; ++it) {
            double mag = fabs(lo) > fabs(hi) ? fabs(lo) : fabs(hi);
            double tol = rtol * mag > atol ? rtol * mag : atol;
            if (hi - lo <= tol) break;
            if (it >= maxit) {
                ++noconv;
                break;
            }
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (orc_sturm_count(n, d, e2, mid, pm) >= k + 1)
                hi = mid;
            else
                lo = mid;
        }
        eigs[m] = 0.5 * (lo + hi);
    }
    free(e2);
    return noconv;
}

/* Eigenvalues of the symmetric A (lower triangle), ascending: tridiagonalise
 * then bisect (the composite result of Algorithm 4.3).  A is overwritten. */
int orc_eigvalsh(int n, double *A, int lda, double rtol, double *eigs)
{
    if (n <= 0) return 0;
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *e = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i) e[i] = 0.0;
    orc_tridiagonalize(n, A, lda, d, e, -1);
    int r = orc_bisect(n, d, e, rtol, 200, eigs);
    free(d);
    free(e);
    return r;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/*
 * Cyclic Jacobi eigenvalue iteration (classical rotation formulas, row-cyclic
 * ordering) on a full symmetric copy of A.  Independent of every Householder
 * routine above; used only as a cross-check for small n.  Eigenvalues are
 * returned ascending.  Returns the number of sweeps taken.
 */
int orc_jacobi(int n, const double *A, int lda, double *eigs)
{
    double *M = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            M[IDX(i, j, n)] = (i >= j) ? A[IDX(i, j, lda)] : A[IDX(j, i, lda)];
    int sweep = 0;
    for (; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double t = M[IDX(i, j, n)] * M[IDX(i, j, n)];
                tot += t;
                if (i != j) off += t;
            }
        if (off <= 1e-34 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = M[IDX(p, q, n)];
                if (apq == 0.0) continue;
                double app = M[IDX(p, p, n)], aqq = M[IDX(q, q, n)];
                double theta = (aqq - app) / (2.0 * apq);
                double t = sgn1(theta) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) { /* columns p, q: M <- M J */
                    double mkp = M[IDX(k, p, n)], mkq = M[IDX(k, q, n)];
                    M[IDX(k, p, n)] = c * mkp - s * mkq;
                    M[IDX(k, q, n)] = s * mkp + c * mkq;
                }
                for (int k = 0; k < n; ++k) { /* rows p, q: M <- J^T M */
                    double mpk = M[IDX(p, k, n)], mqk = M[IDX(q, k, n)];
                    M[IDX(p, k, n)] = c * mpk - s * mqk;
                    M[IDX(q, k, n)] = s * mpk + c * mqk;
                }
            }
    }
    for (int i = 0; i < n; ++i) eigs[i] = M[IDX(i, i, n)];
    qsort(eigs, (size_t)n, sizeof(double), cmp_double);
    free(M);
    return sweep;
}

/*
 * Inertia count: number of negative pivots of the unpivoted LDL^T
 * factorisation of A - xI, computed in long double on a dense copy of the
 * lower triangle.  By Sylvester's law of inertia this is the number of
 * eigenvalues of A below x; no Householder code is involved.
 */
int orc_inertia(int n, const double *A, int lda, double x)
{
    long double *L = (long double *)malloc(sizeof(long double) * (size_t)n * (size_t)n);
    for (int j = 0; j < n; ++j)
        for (int i = j; i < n; ++i)
            L[IDX(i, j, n)] = (long double)A[IDX(i, j, lda)] - (i == j ? (long double)x : 0.0L);
    int neg = 0;
    for (int k = 0; k < n; ++k) {
        long double piv = L[IDX(k, k, n)];
        if (piv == 0.0L) piv = -1e-300L;
        if (piv < 0.0L) ++neg;
        for (int i = k + 1; i < n; ++i) {
            long double lik = L[IDX(i, k, n)] / piv;
            for (int j = k + 1; j <= i; ++j) L[IDX(i, j, n)] -= lik * L[IDX(j, k, n)];
        }
        for (int i = k + 1; i < n; ++i) L[IDX(i, k, n)] /= piv;
    }
    free(L);
    return neg;
}

/*
 * Number of eigenvalues of a banded symmetric B strictly below x: the
 * negative pivots of the unpivoted LDL^T factorisation of B - xI
 * (Sylvester's law of inertia), in long double.  B is given in packed lower
 * band storage AB[d + j*ldab] = B(j+d, j), 0 <= d <= b.  Without pivoting
 * the factor L keeps the half-bandwidth b, so the work is O(n b^2): this is
 * what checks eigenvalue counts of band matrices too large for a full
 * eigensolve.  A pivot of magnitude below DBL_MIN is replaced by -DBL_MIN
 * (the Sturm-count convention).
 */
int orc_band_inertia(int n, const double *AB, int ldab, int b, double x)
{
    const size_t ldl = (size_t)b + 1;
    long double *L = (long double *)calloc(ldl * (size_t)n, sizeof(long double));
    long double *D = (long double *)malloc(sizeof(long double) * (size_t)n);
    int neg = 0;
    for (int j = 0; j < n; ++j) {
        int k0 = j - b > 0 ? j - b : 0;
        long double s = (long double)AB[(size_t)j * ldab] - (long double)x;
        for (int k = k0; k < j; ++k) {
            long double l = L[(size_t)(j - k) + (size_t)k * ldl];
            s -= l * l * D[k];
        }
        if (fabsl(s) < (long double)DBL_MIN) s = -(long double)DBL_MIN;
        D[j] = s;
        if (s < 0.0L) ++neg;
        for (int i = j + 1; i <= j + b && i < n; ++i) {
            long double t = (long double)AB[(size_t)(i - j) + (size_t)j * ldab];
            int ki = i - b > 0 ? i - b : 0;
            for (int k = ki; k < j; ++k)
                t -= L[(size_t)(i - k) + (size_t)k * ldl] * L[(size_t)(j - k) + (size_t)k * ldl] * D[k];
            L[(size_t)(i - j) + (size_t)j * ldl] = t / s;
        }
    }
    free(L);
    free(D);
    return neg;
}

/*
 * Householder QR of the m x nc panel P (leading dimension ldp), computing
 * r = min(nc, m-1) reflectors (a column with a single remaining entry gets
 * none), in the "always reflect" convention of orc_house (Lemma 3.4).
 * On return: P holds R = Q^T P in its upper trapezoid and exact zeros below;
 * U (m x r, ldu) the unit lower-trapezoidal Householder vectors; T (r x r,
 * ldt) the upper-triangular compact-WY factor with Q = I - U T U^T, built by
 * the forward recurrence T[0:k,k] = -tau_k T[0:k,0:k] U[:,0:k]^T U[:,k]
 * (Cor. 3.7's Householder representation).  Returns r.
 */
/*
 * Sign margin of the Householder reflectors formed since the last reset:
 * the smallest |alpha| / ||x|| (alpha the leading entry before reflection).
 * The "always reflect" rule takes beta's sign from alpha, so a reduction
 * whose margin is far above the working precision's rounding error makes
 * the same sign choices in any precision -- the condition under which the
 * band produced by full_to_band is unique entry by entry.  Reporting only;
 * it changes no arithmetic.
 */
static double g_sign_margin = 1.0;
void orc_sign_margin_reset(void) { g_sign_margin = 1.0; }
double orc_sign_margin_get(void) { return g_sign_margin; }

int orc_panel_qr(int m, int nc, double *P, int ldp, double *U, int ldu, double *T, int ldt)
{
    int r = nc < m - 1 ? nc : m - 1;
    if (r < 0) r = 0;
    double *tau = (double *)malloc(sizeof(double) * (size_t)(r > 0 ? r : 1));
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(r > 0 ? r : 1));
    for (int k = 0; k < r; ++k) {
        double beta;
        double *x = &P[IDX(k, k, ldp)];
        double alpha = x[0];
        double t = orc_house(m - k, x, 1, &beta);
        if (beta != 0.0 && fabs(alpha) / fabs(beta) < g_sign_margin) g_sign_margin = fabs(alpha) / fabs(beta);
        tau[k] = t;
        /* store v in U (unit lower trapezoidal) */
        for (int i = 0; i < m; ++i) U[IDX(i, k, ldu)] = (i < k) ? 0.0 : (i == k ? 1.0 : x[i - k]);
        /* apply H_k = I - tau v v^T to P[k:m, k+1:nc] */
        for (int j = k + 1; j < nc; ++j) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += U[IDX(i, k, ldu)] * P[IDX(i, j, ldp)];
            s *= t;
            for (int i = k; i < m; ++i) P[IDX(i, j, ldp)] -= s * U[IDX(i, k, ldu)];
        }
        P[IDX(k, k, ldp)] = beta;
        for (int i = k + 1; i < m; ++i) P[IDX(i, k, ldp)] = 0.0;
    }
    /* rows below the diagonal of columns >= r (only when m - 1 < nc): none
     * remain below row m-1, so R is complete.  Forward T recurrence. */
    for (int k = 0; k < r; ++k) {
        for (int i = 0; i < r; ++i) T[IDX(i, k, ldt)] = 0.0;
        T[IDX(k, k, ldt)] = tau[k];
        for (int i = 0; i < k; ++i) {
            double s = 0.0;
            for (int q = 0; q < m; ++q) s += U[IDX(q, i, ldu)] * U[IDX(q, k, ldu)];
            tmp[i] = s;
        }
        for (int i = 0; i < k; ++i) {
            double s = 0.0;
            for (int q = i; q < k; ++q) s += T[IDX(i, q, ldt)] * tmp[q];
            T[IDX(i, k, ldt)] = -tau[k] * s;
        }
    }
    free(tau);
    free(tmp);
    return r;
}

/*
 * Two-sided update of the symmetric N x N block X (full storage, ldx) by
 * Q = I - U T U^T with U N x r, T r x r, in the rank-2r form of Eq. 4.1:
 *   W = X U (the symmetric product),  WT = W T,
 *   V = (1/2) U (T^T (U^T (W T))) - W T        (Algorithm 4.1, V_1 line)
 *   X <- X + U V^T + V U^T.
 * The products are formed right to left in the order the algorithm writes.
 */
static void orc_two_sided_update(int N, int r, double *X, int ldx, const double *U, int ldu,
                                 const double *T, int ldt)
{
    if (r <= 0 || N <= 0) return;
    double *W = (double *)calloc((size_t)N * r, sizeof(double));
    double *WT = (double *)calloc((size_t)N * r, sizeof(double));
    double *S = (double *)calloc((size_t)r * r, sizeof(double));
    double *Z = (double *)calloc((size_t)r * r, sizeof(double));
    double *V = (double *)calloc((size_t)N * r, sizeof(double));
    /* W = X U */
    for (int c = 0; c < r; ++c)
        for (int k = 0; k < N; ++k) {
            double u = U[IDX(k, c, ldu)];
            if (u == 0.0) continue;
            for (int i = 0; i < N; ++i) W[IDX(i, c, N)] += X[IDX(i, k, ldx)] * u;
        }
    /* WT = W T */
    for (int c = 0; c < r; ++c)
        for (int k = 0; k <= c; ++k) {
            double t = T[IDX(k, c, ldt)];
            for (int i = 0; i < N; ++i) WT[IDX(i, c, N)] += W[IDX(i, k, N)] * t;
        }
    /* S = U^T (W T) */
    for (int c = 0; c < r; ++c)
        for (int a = 0; a < r; ++a) {
            double s = 0.0;
            for (int i = 0; i < N; ++i) s += U[IDX(i, a, ldu)] * WT[IDX(i, c, N)];
            S[IDX(a, c, r)] = s;
        }
    /* Z = T^T S */
    for (int c = 0; c < r; ++c)
        for (int a = 0; a < r; ++a) {
            double s = 0.0;
            for (int k = 0; k <= a; ++k) s += T[IDX(k, a, ldt)] * S[IDX(k, c, r)];
            Z[IDX(a, c, r)] = s;
        }
    /* V = 0.5 U Z - W T */
    for (int c = 0; c < r; ++c) {
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
            for (int a = 0; a < r; ++a) s += U[IDX(i, a, ldu)] * Z[IDX(a, c, r)];
            V[IDX(i, c, N)] = 0.5 * s - WT[IDX(i, c, N)];
        }
    }
    /* X <- X + U V^T + V U^T */
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
            for (int a = 0; a < r; ++a)
                s += U[IDX(i, a, ldu)] * V[IDX(j, a, N)] + V[IDX(i, a, N)] * U[IDX(j, a, ldu)];
            X[IDX(i, j, ldx)] += s;
        }
    free(W);
    free(WT);
    free(S);
    free(Z);
    free(V);
}

/*
 * Algorithm 4.1 (full-to-band), run right-looking on one processor: for
 * panel k (columns kb .. kb+b-1, rows r0 = (k+1)b .. n-1, N = n - r0 >= 2):
 *   [U, T, R] = QR(A21)                (Householder QR, orc_panel_qr)
 *   A22 <- A22 + U V^T + V U^T          (Eq. 4.1; same V as the V_1 line)
 *   A21 <- [R; 0],  A12 <- A21^T         (the band assembly of Algorithm 4.1)
 * Applying each panel's update to the whole trailing matrix at once is the
 * same similarity as the aggregated left-looking U^(0), V^(0) form (Eq. 4.2).
 * A is full symmetric storage (both triangles kept), n x n, lda; on return
 * it holds the band matrix with half-bandwidth b (exact zeros outside).
 */
void orc_full_to_band(int n, double *A, int lda, int b)
{
    if (b < 1) return;
    double *U = (double *)malloc(sizeof(double) * (size_t)n * (size_t)b + 8);
    double *T = (double *)malloc(sizeof(double) * (size_t)b * (size_t)b + 8);
    double *P = (double *)malloc(sizeof(double) * (size_t)n * (size_t)b + 8);
    for (int k = 0;; ++k) {
        int c0 = k * b, r0 = c0 + b;
        if (r0 >= n) break;
        int N = n - r0;
        if (N < 2) break;
        int nc = b;
        for (int j = 0; j < nc; ++j)
            for (int i = 0; i < N; ++i) P[IDX(i, j, N)] = A[IDX(r0 + i, c0 + j, lda)];
        int r = orc_panel_qr(N, nc, P, N, U, N, T, b);
        orc_two_sided_update(N, r, &A[IDX(r0, r0, lda)], lda, U, N, T, b);
        for (int j = 0; j < nc; ++j)
            for (int i = 0; i < N; ++i) {
                A[IDX(r0 + i, c0 + j, lda)] = P[IDX(i, j, N)];
                A[IDX(c0 + j, r0 + i, lda)] = P[IDX(i, j, N)];
            }
    }
    free(U);
    free(T);
    free(P);
}

/*
 * One chase (i, j) of Algorithm 4.2 (band-to-band, b -> h with h | b) on
 * dense full symmetric storage.  Offsets (1-based i, j as in the algorithm;
 * 0-based storage):
 *   o_blg = (i-1)h + (j-1)b,  o_qr.r = o_blg + h
 *   j = 1: o_qr.c = o_qr.r - h, o_v = 0, o_up.c = o_qr.r     (reading A5)
 *   j > 1: o_qr.c = o_qr.r - b, o_v = b - h, o_up.c = o_qr.c + h
 *   n_r = min(n - o_qr.r, b)
 *   n_c = min(n - o_up.c, 2b) for j = 1, min(n - o_up.c, 3b - h) for j > 1
 *         (reading A6; nc_paper != 0 uses the printed min(n - o_up.c, h + 3b)
 *         instead, which must give the same result because the extra rows
 *         are exactly zero)
 *   QR of the n_r x h block B[I_qr.rs, I_qr.cs] (reading A8)
 * Steps: [U,T,R] = QR(B[qr rows, qr cols]); write [R;0] and its transpose;
 * W = B[up cols, qr rows] U T; V = -W;
 * V[v rows] += (1/2) U (T^T (U^T W[v rows])); B[qr rows, up cols] += U V^T;
 * B[up cols, qr rows] += V U^T.
 * Returns 0 if the chase does not exist (n - o_qr.r < 2, reading A7).
 */
static int orc_chase(int n, double *B, int ldb, int b, int h, int i, int j, int nc_paper)
{
    int o_blg = (i - 1) * h + (j - 1) * b;
    int o_qr_r = o_blg + h;
    if (n - o_qr_r < 2) return 0;
    int o_qr_c, o_v, o_up_c, n_c;
    if (j == 1) {
        o_qr_c = o_qr_r - h;
        o_v = 0;
        o_up_c = o_qr_r;
    } else {
        o_qr_c = o_qr_r - b;
        o_v = b - h;
        o_up_c = o_qr_c + h;
    }
    int n_r = n - o_qr_r < b ? n - o_qr_r : b;
    int lim = nc_paper ? (h + 3 * b) : (j == 1 ? 2 * b : 3 * b - h);
    n_c = n - o_up_c < lim ? n - o_up_c : lim;
    int ncmax = 3 * b + h + 1;
    double *Q = (double *)malloc(sizeof(double) * (size_t)b * (size_t)h);
    double *U = (double *)malloc(sizeof(double) * (size_t)b * (size_t)h);
    double *T = (double *)malloc(sizeof(double) * (size_t)h * (size_t)h);
    double *W = (double *)malloc(sizeof(double) * (size_t)ncmax * (size_t)h);
    double *V = (double *)malloc(sizeof(double) * (size_t)ncmax * (size_t)h);
    double *S = (double *)malloc(sizeof(double) * (size_t)h * (size_t)h);
    double *Z = (double *)malloc(sizeof(double) * (size_t)h * (size_t)h);
    /* QR of the n_r x h block */
    for (int c = 0; c < h; ++c)
        for (int r = 0; r < n_r; ++r) Q[IDX(r, c, n_r)] = B[IDX(o_qr_r + r, o_qr_c + c, ldb)];
    int nr = orc_panel_qr(n_r, h, Q, n_r, U, n_r, T, h);
    for (int c = 0; c < h; ++c)
        for (int r = 0; r < n_r; ++r) {
            B[IDX(o_qr_r + r, o_qr_c + c, ldb)] = Q[IDX(r, c, n_r)];
            B[IDX(o_qr_c + c, o_qr_r + r, ldb)] = Q[IDX(r, c, n_r)];
        }
    if (nr > 0) {
        /* W = B[up cols, qr rows] U T */
        for (int c = 0; c < nr; ++c)
            for (int r = 0; r < n_c; ++r) {
                double s = 0.0;
                for (int q = 0; q < n_r; ++q) s += B[IDX(o_up_c + r, o_qr_r + q, ldb)] * U[IDX(q, c, n_r)];
                V[IDX(r, c, n_c)] = s; /* V used as scratch for B U */
            }
        for (int c = 0; c < nr; ++c)
            for (int r = 0; r < n_c; ++r) {
                double s = 0.0;
                for (int q = 0; q <= c; ++q) s += V[IDX(r, q, n_c)] * T[IDX(q, c, h)];
                W[IDX(r, c, n_c)] = s;
            }
        /* V = -W */
        for (int c = 0; c < nr; ++c)
            for (int r = 0; r < n_c; ++r) V[IDX(r, c, n_c)] = -W[IDX(r, c, n_c)];
        /* S = U^T W[v rows], Z = T^T S, V[v rows] += 0.5 U Z */
        for (int c = 0; c < nr; ++c)
            for (int a = 0; a < nr; ++a) {
                double s = 0.0;
                for (int q = 0; q < n_r; ++q) s += U[IDX(q, a, n_r)] * W[IDX(o_v + q, c, n_c)];
                S[IDX(a, c, h)] = s;
            }
        for (int c = 0; c < nr; ++c)
            for (int a = 0; a < nr; ++a) {
                double s = 0.0;
                for (int q = 0; q <= a; ++q) s += T[IDX(q, a, h)] * S[IDX(q, c, h)];
                Z[IDX(a, c, h)] = s;
            }
        for (int c = 0; c < nr; ++c)
            for (int q = 0; q < n_r; ++q) {
                double s = 0.0;
                for (int a = 0; a < nr; ++a) s += U[IDX(q, a, n_r)] * Z[IDX(a, c, h)];
                V[IDX(o_v + q, c, n_c)] += 0.5 * s;
            }
        /* B[qr rows, up cols] += U V^T ; B[up cols, qr rows] += V U^T */
        for (int cc = 0; cc < n_c; ++cc)
            for (int q = 0; q < n_r; ++q) {
                double s = 0.0;
                for (int a = 0; a < nr; ++a) s += U[IDX(q, a, n_r)] * V[IDX(cc, a, n_c)];
                B[IDX(o_qr_r + q, o_up_c + cc, ldb)] += s;
            }
        for (int q = 0; q < n_r; ++q)
            for (int rr = 0; rr < n_c; ++rr) {
                double s = 0.0;
                for (int a = 0; a < nr; ++a) s += V[IDX(rr, a, n_c)] * U[IDX(q, a, n_r)];
                B[IDX(o_up_c + rr, o_qr_r + q, ldb)] += s;
            }
    }
    free(Q);
    free(U);
    free(T);
    free(W);
    free(V);
    free(S);
    free(Z);
    return 1;
}

/*
 * Algorithm 4.2 in the sequential order it writes: sweeps i = 1, 2, ...
 * while n - ih >= 2, and within a sweep chases j = 1, 2, ... while the chase
 * exists (reading A7).  max_chases >= 0 stops after that many chases (to
 * inspect intermediate fill); max_chases < 0 runs the whole reduction.
 */
void orc_band_to_band(int n, double *B, int ldb, int b, int h, int nc_paper, long max_chases)
{
    if (h < 1 || b <= h || b % h != 0) return;
    long done = 0;
    for (int i = 1; n - i * h >= 2; ++i) {
        for (int j = 1;; ++j) {
            if (max_chases >= 0 && done >= max_chases) return;
            if (!orc_chase(n, B, ldb, b, h, i, j, nc_paper)) break;
            ++done;
        }
    }
}

typedef struct {
    long key;
    int i, j;
} orc_chase_id;

static int cmp_chase(const void *a, const void *b)
{
    const orc_chase_id *x = (const orc_chase_id *)a, *y = (const orc_chase_id *)b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->i > y->i) - (x->i < y->i);
}

/*
 * The same chases as orc_band_to_band, executed in wavefront order: chase
 * (i, j) gets the time step t = wave * i + j, and chases of one time step
 * run in increasing i (tie_desc = 0) or decreasing i (tie_desc != 0).
 * A pipelined schedule is legal exactly when every such order reproduces
 * the sequential result bit for bit.  (The pipeline the paper pictures
 * for k = 2 corresponds to wave = 2.)
 */
void orc_band_to_band_wavefront(int n, double *B, int ldb, int b, int h, int wave, int tie_desc)
{
    if (h < 1 || b <= h || b % h != 0) return;
    long cnt = 0, cap = 1024;
    orc_chase_id *ids = (orc_chase_id *)malloc(sizeof(orc_chase_id) * (size_t)cap);
    for (int i = 1; n - i * h >= 2; ++i)
        for (int j = 1; n - ((i - 1) * h + (j - 1) * b + h) >= 2; ++j) {
            if (cnt == cap) {
                cap *= 2;
                ids = (orc_chase_id *)realloc(ids, sizeof(orc_chase_id) * (size_t)cap);
            }
            ids[cnt].key = (long)wave * i + j;
            ids[cnt].i = tie_desc ? -i : i;
            ids[cnt].j = j;
            ++cnt;
        }
    qsort(ids, (size_t)cnt, sizeof(orc_chase_id), cmp_chase);
    for (long k = 0; k < cnt; ++k) {
        int i = ids[k].i < 0 ? -ids[k].i : ids[k].i;
        orc_chase(n, B, ldb, b, h, i, ids[k].j, 0);
    }
    free(ids);
}
