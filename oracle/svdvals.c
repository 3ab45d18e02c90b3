/*
 * oracle/svdvals.c -- FP64 CPU oracle for singular values.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference against
 * which the GPU library is checked.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the library never does, and
 * this file shares no code, header, table or helper with the GPU sources.
 *
 * What is computed (paper Section 5.1.1, "Algorithm"): the singular values
 * sigma_1 >= ... >= sigma_p >= 0, p = min(m, n), of a dense real m x n matrix.
 * The paper reaches them by orthogonal transformations (dense -> band ->
 * bidiagonal -> diagonal) which leave the singular values intact.  The
 * oracle reaches the same values through a *different* exact algorithm:
 *
 *   1. one-stage Householder bidiagonalisation (Golub & Kahan 1965;
 *      Golub & Van Loan, "Matrix Computations", 4th ed., Alg. 5.4.2);
 *   2. implicit-shift Golub-Kahan QR iteration on the bidiagonal, with a
 *      Wilkinson shift taken from the trailing 2x2 of B^T B, splitting on
 *      negligible superdiagonals and the zero-diagonal chase
 *      (Golub & Reinsch 1970; Golub & Van Loan Alg. 8.6.1 / 8.6.2).
 *
 * A second, independent oracle -- one-sided Jacobi (Hestenes 1958) -- is
 * provided for small matrices so the first one can be cross-checked.
 *
 * Conventions: column-major storage with leading dimension lda >= rows.
 * Every function returns 0 on success, > 0 when the QR iteration hit its
 * iteration cap (the count of unconverged values), < 0 on a bad argument.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* Euclidean norm of x[0], x[inc], ..., x[(n-1)*inc].
 * Plain sum of squares; if that sum overflowed or fell into the range where
 * underflow may have destroyed it, recompute with every entry divided by the
 * largest magnitude (a two-pass scaled norm). */
static double norm2(const double *x, long n, long inc)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) {
        double v = x[i * inc];
        s += v * v;
    }
    if (s < DBL_MAX && s > DBL_MIN / DBL_EPSILON)
        return sqrt(s);
    double mx = 0.0;
    for (long i = 0; i < n; ++i) {
        double a = fabs(x[i * inc]);
        if (a > mx) mx = a;
    }
    if (mx == 0.0 || !isfinite(mx))
        return mx;
    double t = 0.0;
    for (long i = 0; i < n; ++i) {
        double v = x[i * inc] / mx;
        t += v * v;
    }
    return mx * sqrt(t);
}

/* Householder reflector H = I - tau v v^T with v = [1; x/(alpha-beta)] that
 * maps [alpha; x] to [beta; 0], beta = -sign(alpha) * ||[alpha; x]||,
 * sign(0) = +1 (Golub & Van Loan Alg. 5.1.1 in the LAPACK normalisation).
 * The tail x (n entries, stride inc) is overwritten by v(2:end).
 * Returns tau; *beta receives the new leading entry.  A zero tail gives
 * tau = 0 (H = I) and beta = alpha. */
static double householder(double alpha, double *x, long n, long inc, double *beta)
{
    double xn = norm2(x, n, inc);
    if (xn == 0.0) {
        *beta = alpha;
        return 0.0;
    }
    double r = hypot(alpha, xn);
    double b = (alpha >= 0.0) ? -r : r;
    double scale = 1.0 / (alpha - b);
    for (long i = 0; i < n; ++i)
        x[i * inc] *= scale;
    *beta = b;
    return (b - alpha) / b;
}

static int thread_count(int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    return nthreads;
#else
    (void)nthreads;
    return 1;
#endif
}

/*
 * Householder bidiagonalisation, m >= n (Golub & Van Loan Alg. 5.4.2).
 * For j = 0..n-1:
 *   - a left reflector annihilates A(j+1:m, j); d[j] is the new A(j, j);
 *   - for j < n-2 a right reflector annihilates A(j, j+2:n); e[j] is the new
 *     A(j, j+1).  For j = n-2, e[j] = A(j, j+1) needs no reflector.
 * A is overwritten (reflector tails are left in the annihilated entries).
 * Reflector application is parallelised over columns with OpenMP.
 */
int oracle_bidiag(int m, int n, double *A, long lda, double *d, double *e, int nthreads)
{
    if (m < n || n < 0 || lda < (m > 1 ? m : 1)) return -1;
    if (n == 0) return 0;
    int nt = thread_count(nthreads);
    double *w = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (!w) return -2;

    for (int j = 0; j < n; ++j) {
        /* ---- left reflector on column j, rows j..m-1 ---- */
        double beta;
        double tau = householder(A[IDX(j, j, lda)], &A[IDX(j + 1, j, lda)], m - j - 1, 1, &beta);
        A[IDX(j, j, lda)] = beta;
        d[j] = beta;
        if (tau != 0.0) {
            const double *v = &A[IDX(j + 1, j, lda)]; /* v(0) = 1 implicit */
#pragma omp parallel for num_threads(nt) schedule(static)
            for (int c = j + 1; c < n; ++c) {
                double *col = &A[IDX(j, c, lda)];
                double s = col[0];
                for (int i = 1; i < m - j; ++i) s += v[i - 1] * col[i];
                s *= tau;
                col[0] -= s;
                for (int i = 1; i < m - j; ++i) col[i] -= s * v[i - 1];
            }
        }
        if (j >= n - 1) break;
        if (j == n - 2) {
            e[j] = A[IDX(j, j + 1, lda)];
            continue;
        }
        /* ---- right reflector on row j, columns j+1..n-1 ---- */
        tau = householder(A[IDX(j, j + 1, lda)], &A[IDX(j, j + 2, lda)], n - j - 2, lda, &beta);
        A[IDX(j, j + 1, lda)] = beta;
        e[j] = beta;
        if (tau != 0.0) {
            /* rows j+1..m-1 : w = A(:, j+1:n) v ; A(:, j+1:n) -= tau w v^T */
            int r0 = j + 1, nr = m - r0;
            const double *vrow = &A[IDX(j, 0, lda)]; /* v(c) = A(j, c) for c >= j+2 */
#pragma omp parallel num_threads(nt)
            {
#pragma omp for schedule(static)
                for (int i = 0; i < nr; ++i) w[i] = A[IDX(r0 + i, j + 1, lda)];
#pragma omp for schedule(static)
                for (int i = 0; i < nr; ++i) {
                    double s = w[i];
                    for (int c = j + 2; c < n; ++c) s += A[IDX(r0 + i, c, lda)] * vrow[IDX(0, c, lda)];
                    w[i] = tau * s;
                }
#pragma omp for schedule(static)
                for (int c = j + 1; c < n; ++c) {
                    double vc = (c == j + 1) ? 1.0 : vrow[IDX(0, c, lda)];
                    double *col = &A[IDX(r0, c, lda)];
                    for (int i = 0; i < nr; ++i) col[i] -= w[i] * vc;
                }
            }
        }
    }
    free(w);
    return 0;
}

/* Plane rotation [c s; -s c] with c*f + s*g = r and -s*f + c*g = 0. */
static void rotation(double f, double g, double *c, double *s, double *r)
{
    if (g == 0.0) {
        *c = 1.0;
        *s = 0.0;
        *r = f;
        return;
    }
    double h = hypot(f, g);
    *c = f / h;
    *s = g / h;
    *r = h;
}

static int cmp_desc(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) - (x > y);
}

/* One implicit-shift Golub-Kahan SVD step on the unreduced block lo..hi of
 * the upper bidiagonal (d, e) (Golub & Van Loan Alg. 8.6.1).  The shift mu is
 * the eigenvalue of the trailing 2x2 of B^T B closer to its (2,2) entry. */
static void gk_step(double *d, double *e, int lo, int hi)
{
    double t22 = d[hi] * d[hi] + e[hi - 1] * e[hi - 1];
    double t11 = d[hi - 1] * d[hi - 1] + (hi - 1 > lo ? e[hi - 2] * e[hi - 2] : 0.0);
    double t12 = d[hi - 1] * e[hi - 1];
    double delta = 0.5 * (t11 - t22);
    double den = delta + (delta >= 0.0 ? 1.0 : -1.0) * hypot(delta, t12);
    double mu = (den == 0.0) ? t22 : t22 - t12 * t12 / den;

    double y = d[lo] * d[lo] - mu;
    double z = d[lo] * e[lo];
    for (int k = lo; k < hi; ++k) {
        double c, s, r;
        /* right rotation on columns k, k+1 */
        rotation(y, z, &c, &s, &r);
        if (k > lo) e[k - 1] = r;
        double dk = d[k], ek = e[k];
        d[k] = c * dk + s * ek;
        e[k] = -s * dk + c * ek;
        double bulge = s * d[k + 1]; /* fill at (k+1, k) */
        d[k + 1] = c * d[k + 1];
        /* left rotation on rows k, k+1 removes the fill */
        rotation(d[k], bulge, &c, &s, &r);
        d[k] = r;
        ek = e[k];
        e[k] = c * ek + s * d[k + 1];
        d[k + 1] = -s * ek + c * d[k + 1];
        if (k < hi - 1) {
            z = s * e[k + 1]; /* fill at (k, k+2) */
            e[k + 1] = c * e[k + 1];
            y = e[k];
        }
    }
}

/* Row k of the block has d[k] == 0: zero its superdiagonal e[k] with left
 * rotations against rows k+1..hi (Golub & Van Loan Sec. 8.6.2). */
static void chase_zero_row(double *d, double *e, int k, int hi)
{
    double x = e[k];
    e[k] = 0.0;
    for (int j = k + 1; j <= hi && x != 0.0; ++j) {
        double c, s, r;
        rotation(d[j], x, &c, &s, &r);
        d[j] = r;
        if (j < hi) {
            x = -s * e[j];
            e[j] = c * e[j];
        }
    }
}

/* The last diagonal d[hi] == 0: zero the column above it (e[hi-1]) with right
 * rotations against columns hi-1, ..., lo (Golub & Van Loan Sec. 8.6.2). */
static void chase_zero_last(double *d, double *e, int lo, int hi)
{
    double x = e[hi - 1];
    e[hi - 1] = 0.0;
    for (int j = hi - 1; j >= lo && x != 0.0; --j) {
        double c, s, r;
        rotation(d[j], x, &c, &s, &r);
        d[j] = r;
        if (j > lo) {
            x = -s * e[j - 1];
            e[j - 1] = c * e[j - 1];
        }
    }
}

/*
 * Singular values of the n x n upper bidiagonal matrix with diagonal d[0..n-1]
 * and superdiagonal e[0..n-2], by implicit-shift Golub-Kahan QR
 * (Golub & Reinsch 1970; Golub & Van Loan Alg. 8.6.2).  S receives the n
 * values sorted descending.  The iteration cap is 30 n + 100 SVD steps.
 */
int oracle_bdsvd(int n, const double *d_in, const double *e_in, double *S)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *e = (double *)malloc(sizeof(double) * (size_t)(n > 1 ? n : 1));
    if (!d || !e) {
        free(d);
        free(e);
        return -2;
    }
    /* scale by a power of two (exact) so squares in the shift cannot overflow */
    double anorm = 0.0;
    for (int i = 0; i < n; ++i) anorm = fmax(anorm, fabs(d_in[i]));
    for (int i = 0; i + 1 < n; ++i) anorm = fmax(anorm, fabs(e_in[i]));
    int ex = 0;
    if (anorm > 0.0) frexp(anorm, &ex);
    for (int i = 0; i < n; ++i) d[i] = ldexp(d_in[i], -ex);
    for (int i = 0; i + 1 < n; ++i) e[i] = ldexp(e_in[i], -ex);
    double bnorm = ldexp(anorm, -ex);

    const double eps = DBL_EPSILON;
    long maxit = 30L * n + 100, it = 0;
    int hi = n - 1, status = 0;
    while (hi > 0) {
        /* splitting: negligible superdiagonals become exact zeros */
        for (int i = 0; i < hi; ++i)
            if (fabs(e[i]) <= eps * (fabs(d[i]) + fabs(d[i + 1]))) e[i] = 0.0;
        if (e[hi - 1] == 0.0) {
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && e[lo - 1] != 0.0) --lo;
        /* zero (negligible) diagonal inside the unreduced block */
        int zk = -1;
        for (int k = lo; k <= hi; ++k)
            if (fabs(d[k]) <= eps * bnorm) {
                d[k] = 0.0;
                zk = k;
                break;
            }
        if (zk >= 0) {
            if (zk < hi)
                chase_zero_row(d, e, zk, hi);
            else
                chase_zero_last(d, e, lo, hi);
            continue;
        }
        if (++it > maxit) {
            status = hi; /* values lo..hi did not converge */
            break;
        }
        gk_step(d, e, lo, hi);
    }
    for (int i = 0; i < n; ++i) S[i] = ldexp(fabs(d[i]), ex);
    qsort(S, (size_t)n, sizeof(double), cmp_desc);
    free(d);
    free(e);
    return status;
}

/* Copy the m x n input into a packed column-major work matrix, transposed
 * when m < n (A and A^T have the same singular values). */
static double *packed_copy(int m, int n, const double *A, long lda, int *mm, int *nn)
{
    int tr = m < n;
    *mm = tr ? n : m;
    *nn = tr ? m : n;
    double *W = (double *)malloc(sizeof(double) * (size_t)(*mm) * (size_t)(*nn));
    if (!W) return NULL;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) {
            double v = A[IDX(i, j, lda)];
            if (tr)
                W[IDX(j, i, *mm)] = v;
            else
                W[IDX(i, j, *mm)] = v;
        }
    return W;
}

/* Singular values of a dense m x n matrix (column-major, lda >= m): S gets
 * min(m, n) values sorted descending.  nthreads <= 0 uses all OpenMP threads. */
int oracle_svdvals(int m, int n, const double *A, long lda, double *S, int nthreads)
{
    if (m < 0 || n < 0 || lda < (m > 1 ? m : 1)) return -1;
    if (m == 0 || n == 0) return 0;
    int mm, nn;
    double *W = packed_copy(m, n, A, lda, &mm, &nn);
    double *d = (double *)malloc(sizeof(double) * (size_t)nn);
    double *e = (double *)malloc(sizeof(double) * (size_t)nn);
    int st = -2;
    if (W && d && e) {
        st = oracle_bidiag(mm, nn, W, mm, d, e, nthreads);
        if (st == 0) st = oracle_bdsvd(nn, d, e, S);
    }
    free(W);
    free(d);
    free(e);
    return st;
}

/*
 * Second oracle: one-sided Jacobi (Hestenes 1958).  Columns of a copy G of A
 * are rotated in pairs until mutually orthogonal; the singular values are
 * then the column norms.  For the pair (p, q) with Gram entries
 * a = |g_p|^2, b = |g_q|^2, g = g_p.g_q, the rotation
 * [g_p g_q] <- [g_p g_q] [c s; -s c] zeroes g when t = s/c is the smaller
 * root of t^2 + 2 z t - 1 = 0, z = (b - a) / (2 g).  Meant for small n.
 */
int oracle_jacobi_svdvals(int m, int n, const double *A, long lda, double *S)
{
    if (m < 0 || n < 0 || lda < (m > 1 ? m : 1)) return -1;
    if (m == 0 || n == 0) return 0;
    int mm, nn;
    double *G = packed_copy(m, n, A, lda, &mm, &nn);
    if (!G) return -2;
    const double tol = DBL_EPSILON * (double)mm;
    /* a column whose norm is at rounding level of ||A||_F cannot move any
       singular value by more than that level: such pairs are left alone */
    double fro = 0.0;
    for (int j = 0; j < nn; ++j) {
        double c = norm2(&G[IDX(0, j, mm)], mm, 1);
        fro = hypot(fro, c);
    }
    const double floor2 = (DBL_EPSILON * fro) * (DBL_EPSILON * fro);
    int status = 1;
    for (int sweep = 0; sweep < 80; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < nn - 1; ++p)
            for (int q = p + 1; q < nn; ++q) {
                double *gp = &G[IDX(0, p, mm)], *gq = &G[IDX(0, q, mm)];
                double a = 0.0, b = 0.0, g = 0.0;
                for (int i = 0; i < mm; ++i) {
                    a += gp[i] * gp[i];
                    b += gq[i] * gq[i];
                    g += gp[i] * gq[i];
                }
                if (g == 0.0 || fabs(g) <= tol * sqrt(a * b) || fmin(a, b) <= floor2) continue;
                rotated = 1;
                double z = (b - a) / (2.0 * g);
                double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < mm; ++i) {
                    double x = gp[i], y = gq[i];
                    gp[i] = c * x - s * y;
                    gq[i] = s * x + c * y;
                }
            }
        if (!rotated) {
            status = 0;
            break;
        }
    }
    for (int j = 0; j < nn; ++j) S[j] = norm2(&G[IDX(0, j, mm)], mm, 1);
    qsort(S, (size_t)nn, sizeof(double), cmp_desc);
    free(G);
    return status;
}
