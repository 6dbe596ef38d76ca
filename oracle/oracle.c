/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the real skew-symmetric
 * eigenproblem (Penke, Marek, Vorwerk, Draxl, Benner: "High Performance
 * Solution of Skew-symmetric Eigenvalue Problems with Applications in Solving
 * the Bethe-Salpeter Eigenvalue Problem", Parallel Computing).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only tests/, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py do.  It shares no code, header or constant with the CUDA
 * library.
 *
 * Route (Algorithm 1, unblocked, no reordering):
 *   1. Householder tridiagonalisation (Sec. 2.1 step 1; Sec. 2.3.1, Eqs. 2-6
 *      with the skew sign u1 = -u2): for c = 0..n-3 a reflector
 *      Q_c = I - tau_c v_c v_c^T annihilates A[c+2:n, c]; the trailing block is
 *      updated as A22 <- A22 + v p^T - p v^T with p = tau A22 v (the symmetric
 *      0.5*tau^2 (v^T A v) v correction is zero for skew A).
 *   2. Link (Lemma 1, Eq. 1): alpha_c = T[c, c+1]; the symmetric tridiagonal
 *      tridiag(alpha, 0, alpha) = -i D^H T D, D = diag(1, i, ..., i^(n-1)).
 *   3. Tridiagonal solve by bisection (Sturm counts) and inverse iteration
 *      (Sec. 3, the solver BSEPACK adapted from ScaLAPACK).
 *   4. Back transformation by D (Algorithm 1 step 3) on real and imaginary
 *      parts separately (Sec. 2.3), then by Q_trd = Q_0 Q_1 ... Q_{n-3}
 *      (Algorithm 1 step 4).
 *
 * Storage: column-major FP64, element (i, j) of a matrix with leading
 * dimension ld at [i + j*ld].  Only the strict lower triangle of A is read.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(M, i, j, ld) ((M)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])
#define ROWBLK 64   /* rows per thread task in the row sums of A22 v */

/* Threads (OpenMP, when built with it): the level-2 loops of the
 * tridiagonalisation, the bisection over eigenvalues, the D map and Q_trd over
 * columns run in parallel.  Every floating-point sum keeps the order of the
 * serial loop, so the results are the same for any thread count.  Inverse
 * iteration stays serial (the Gram-Schmidt chain of a cluster is sequential).
 * oracle_set_threads(t <= 0) leaves the OpenMP default; it returns the number
 * of threads a parallel loop will use (1 without OpenMP).                  */
int oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Householder reflector (Sec. 2.1: Q_i = I - tau_i v_i v_i^T, v stored in the
 * eliminated column).  Convention: beta = -sign(x0) ||x||, sign(0) = +1,
 * tau = (beta - x0)/beta, v = x/(x0 - beta), v0 = 1; tau = 0 (Q = I) when the
 * tail x[1:] is zero.  On exit x[1:] holds v[1:], *beta the new x0.       */
static void reflector(int m, double *x, double *tau, double *beta)
{
    double x0 = x[0], tail = 0.0;
    for (int i = 1; i < m; i++) tail += x[i] * x[i];
    if (tail == 0.0) {
        *tau = 0.0;
        *beta = x0;
        return;
    }
    double r = sqrt(x0 * x0 + tail);
    double b = (x0 >= 0.0) ? -r : r;
    *tau = (b - x0) / b;
    double s = 1.0 / (x0 - b);
    for (int i = 1; i < m; i++) x[i] *= s;
    *beta = b;
}

/* Tridiagonalise skew A (n x n, strict lower triangle read; A overwritten by
 * a full skew working copy is NOT required: the routine works on its own
 * lower-triangle copy).  Outputs:
 *   alpha[0..n-2]  super-diagonal of T = Q^T A Q (T[c, c+1] = alpha[c]),
 *   V (n x n, ld n): column c holds v_c in rows c+1..n-1 (v_c[c+1] = 1),
 *   tau[0..n-3].
 * Only the lower triangle of the trailing block is kept: for skew A22,
 * (A22 v)_i = sum_{j<i} L_ij v_j - sum_{j>i} L_ji v_j.                     */
int oracle_tridiagonalize(int n, const double *A, int lda, double *alpha,
                          double *V, double *tau)
{
    if (n <= 0) return 0;
    double *L = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *s = (double *)malloc(sizeof(double) * (size_t)n);
    if (!L || !p || !s) { free(L); free(p); free(s); return -1; }
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; j++) {
        for (int i = 0; i < n; i++) {
            AT(L, i, j, n) = (i > j) ? AT(A, i, j, lda) : 0.0;
            AT(V, i, j, n) = 0.0;
        }
    }
    for (int c = 0; c + 2 < n; c++) {
        int m = n - c - 1;               /* length of x = L[c+1:n, c] */
        double *x = &AT(L, c + 1, c, n);
        double t, beta;
        reflector(m, x, &t, &beta);
        tau[c] = t;
        /* v = (1, x[1:]) */
        AT(V, c + 1, c, n) = 1.0;
        for (int i = 1; i < m; i++) AT(V, c + 1 + i, c, n) = x[i];
        const double *v = &AT(V, c + 1, c, n);
        /* p = tau * A22 v, A22 = L[c+1:, c+1:] - L[c+1:, c+1:]^T:
         *   p_i = tau * (r_i - s_i),  r_i = sum_{j<i} L_ij v_j,
         *                             s_i = sum_{j>i} L_ji v_j,
         * each sum taken in ascending j.  s_i reads column i of L; r_i is
         * accumulated over a block of rows, column by column, so that every
         * read is a contiguous piece of a column.  The threads split columns
         * (s) and row blocks (r); each sum keeps its order, so the result does
         * not depend on the thread count. */
#pragma omp parallel for schedule(dynamic, 16)
        for (int j = 0; j < m; j++) {
            const double *Lj = &AT(L, c + 1, c + 1 + j, n);
            double sj = 0.0;
            for (int i = j + 1; i < m; i++) sj += Lj[i] * v[i];
            s[j] = sj;
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int i0 = 0; i0 < m; i0 += ROWBLK) {
            const int i1 = (i0 + ROWBLK < m) ? i0 + ROWBLK : m;
            for (int i = i0; i < i1; i++) p[i] = 0.0;
            for (int j = 0; j + 1 < i1; j++) {
                const double *Lj = &AT(L, c + 1, c + 1 + j, n);
                const double vj = v[j];
                for (int i = (j + 1 > i0) ? j + 1 : i0; i < i1; i++) p[i] += Lj[i] * vj;
            }
            for (int i = i0; i < i1; i++) p[i] = (p[i] - s[i]) * t;
        }
        /* A22 <- A22 + v p^T - p v^T (strict lower part) */
#pragma omp parallel for schedule(dynamic, 16)
        for (int j = 0; j < m; j++)
            for (int i = j + 1; i < m; i++)
                AT(L, c + 1 + i, c + 1 + j, n) += v[i] * p[j] - p[i] * v[j];
        /* column c becomes beta e1: T[c+1, c] = beta, T[c, c+1] = -beta */
        x[0] = beta;
        for (int i = 1; i < m; i++) x[i] = 0.0;
        alpha[c] = -beta;
    }
    if (n >= 2) alpha[n - 2] = -AT(L, n - 1, n - 2, n);
    free(L);
    free(p);
    free(s);
    return 0;
}

/* Apply Q_trd = Q_0 Q_1 ... Q_{n-3} to Z (n x k, ld ldz): Z <- Q_trd Z, i.e.
 * the reflectors in reverse order of generation (Algorithm 1 step 4).      */
void oracle_apply_q(int n, const double *V, const double *tau, int k, double *Z,
                    int ldz)
{
    for (int c = n - 3; c >= 0; c--) {
        double t = tau[c];
        if (t == 0.0) continue;
        const double *v = &AT(V, c + 1, c, n);
        int m = n - c - 1;
#pragma omp parallel for schedule(static)
        for (int j = 0; j < k; j++) {
            double *z = &AT(Z, c + 1, j, ldz);
            double w = 0.0;
            for (int i = 0; i < m; i++) w += v[i] * z[i];
            w *= t;
            for (int i = 0; i < m; i++) z[i] -= w * v[i];
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Symmetric tridiagonal S = tridiag(alpha, 0, alpha) (Lemma 1).           */

/* ||S||_1 (Gershgorin radius): max_i |alpha_{i-1}| + |alpha_i|.          */
static double gersh(int n, const double *alpha)
{
    double g = 0.0;
    for (int i = 0; i < n; i++) {
        double r = 0.0;
        if (i > 0) r += fabs(alpha[i - 1]);
        if (i < n - 1) r += fabs(alpha[i]);
        if (r > g) g = r;
    }
    return g;
}

/* Number of eigenvalues of S strictly less than x (Sturm sequence of the
 * LDL^T pivots of S - xI, with tiny pivots replaced by -pivmin).          */
static int sturm_count(int n, const double *a2, double pivmin, double x)
{
    int cnt = 0;
    double d = -x;
    if (fabs(d) < pivmin) d = -pivmin;
    if (d < 0.0) cnt++;
    for (int i = 1; i < n; i++) {
        d = -x - a2[i - 1] / d;
        if (fabs(d) < pivmin) d = -pivmin;
        if (d < 0.0) cnt++;
    }
    return cnt;
}

/* The nev largest eigenvalues of S, descending (lambda[0] largest), by
 * bisection on [-g, g].  Stop when hi - lo <= 2 eps max(|lo|,|hi|) +
 * DBL_MIN; return the midpoint.  nev may be up to n (used by tests).     */
int oracle_bisect(int n, const double *alpha, int nev, double *lambda)
{
    if (n <= 0 || nev <= 0) return 0;
    if (n == 1) { lambda[0] = 0.0; return 0; }
    double *a2 = (double *)malloc(sizeof(double) * (size_t)n);
    if (!a2) return -1;
    double amax = 0.0;
    for (int i = 0; i < n - 1; i++) {
        a2[i] = alpha[i] * alpha[i];
        if (a2[i] > amax) amax = a2[i];
    }
    double pivmin = DBL_MIN * (amax > 1.0 ? amax : 1.0);
    double g = gersh(n, alpha);
    if (g == 0.0) {                     /* S = 0: every eigenvalue is 0 */
        for (int k = 0; k < nev; k++) lambda[k] = 0.0;
        free(a2);
        return 0;
    }
    double glo = -g - 2.0 * DBL_EPSILON * g - pivmin;
    double ghi = g + 2.0 * DBL_EPSILON * g + pivmin;
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < nev; k++) {
        int j = n - 1 - k;              /* 0-based ascending index */
        double lo = glo, hi = ghi;      /* count(lo) <= j < count(hi) */
        for (int it = 0; it < 4000; it++) {
            double w = hi - lo;
            double tol = 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + DBL_MIN;
            if (w <= tol) break;
            double mid = lo + 0.5 * w;
            if (mid <= lo || mid >= hi) break;
            if (sturm_count(n, a2, pivmin, mid) <= j) lo = mid;
            else hi = mid;
        }
        lambda[k] = lo + 0.5 * (hi - lo);
    }
    free(a2);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Zero-diagonal form (the remark after Algorithm 1 in Sec. 2.2: a solver that
 * uses the zero diagonal of tridiag(alpha, 0, alpha) may pay off).  Ordering
 * the unknowns even indices first, odd second (a perfect shuffle), S becomes
 * [[0, B], [B^T, 0]] with B lower bidiagonal, ceil(n/2) x floor(n/2):
 *   B[i][i] = a_i = alpha_{2i},  B[i+1][i] = b_i = alpha_{2i+1}
 * (alpha_j = 0 for j > n-2).  The eigenvalues of S are +-sigma(B), and 0 when
 * n is odd, so its eigenvalues >= 0 are the square roots of the eigenvalues
 * of B B^T (order ceil(n/2)).  B B^T = L D L^T with D_i = a_i^2 and the unit
 * lower bidiagonal L of l_i = b_i / a_i; the stationary qd transform
 * L D L^T - t I = L+ D+ L+^T gives, with s_0 = -t,
 *   D+_i = a_i^2 + s_i,   s_{i+1} = b_i^2 s_i / D+_i - t,
 * and the number of negative D+_i is the number of eigenvalues of B B^T below
 * t (Sylvester's law of inertia).  Pivots of modulus below pivmin are replaced
 * by -pivmin, as in the Sturm count above.  The counts work with squares, so
 * singular values below about 1e-154 times the scale are resolved to absolute
 * accuracy only (the full-length count has the same kind of floor).       */
static int bidiag_count(int m, const double *a2, const double *b2, double pivmin, double t)
{
    int cnt = 0;
    double sv = -t;
    for (int i = 0; i < m; i++) {
        double d = a2[i] + sv;
        if (fabs(d) < pivmin) d = -pivmin;
        if (d < 0.0) cnt++;
        sv = b2[i] * sv / d - t;
    }
    return cnt;
}

/* The nev largest eigenvalues of S = tridiag(alpha, 0, alpha), descending,
 * as sqrt of the eigenvalues of B B^T found by bisection on x in [0, g] with
 * counts at t = x^2; same stopping rule as oracle_bisect.  nev <= n/2 (the
 * nonnegative half; for odd n the zero eigenvalue is the (n+1)/2-th).      */
int oracle_bidiag_bisect(int n, const double *alpha, int nev, double *lambda)
{
    if (n <= 0 || nev <= 0) return 0;
    if (n == 1) { lambda[0] = 0.0; return 0; }
    const int m = (n + 1) / 2;
    double *a2 = (double *)malloc(sizeof(double) * (size_t)m);
    double *b2 = (double *)malloc(sizeof(double) * (size_t)m);
    if (!a2 || !b2) { free(a2); free(b2); return -1; }
    double amax = 0.0;
    for (int i = 0; i < m; i++) {
        const double a = (2 * i <= n - 2) ? alpha[2 * i] : 0.0;
        const double b = (2 * i + 1 <= n - 2) ? alpha[2 * i + 1] : 0.0;
        a2[i] = a * a;
        b2[i] = b * b;
        if (a2[i] > amax) amax = a2[i];
        if (b2[i] > amax) amax = b2[i];
    }
    const double pivmin = DBL_MIN * (amax > 1.0 ? amax : 1.0);
    const double g = gersh(n, alpha);
    if (g == 0.0) {
        for (int k = 0; k < nev; k++) lambda[k] = 0.0;
        free(a2); free(b2);
        return 0;
    }
    const double ghi = g + 2.0 * DBL_EPSILON * g + pivmin;
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < nev; k++) {
        const int j = m - 1 - k;        /* 0-based ascending index in B B^T */
        double lo = 0.0, hi = ghi;      /* count(lo^2) <= j < count(hi^2) */
        for (int it = 0; it < 4000; it++) {
            double w = hi - lo;
            double tol = 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + DBL_MIN;
            if (w <= tol) break;
            double mid = lo + 0.5 * w;
            if (mid <= lo || mid >= hi) break;
            if (bidiag_count(m, a2, b2, pivmin, mid * mid) <= j) lo = mid;
            else hi = mid;
        }
        lambda[k] = lo + 0.5 * (hi - lo);
    }
    free(a2); free(b2);
    return 0;
}

/* counter-based start vector: splitmix64 of (seed, index) -> uniform(-1,1) */
static double start_entry(uint64_t seed, uint64_t i)
{
    uint64_t z = seed * 0x9E3779B97F4A7C15ULL + i + 0x632BE59BD9B4E019ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

/* Eigenvectors of S for given eigenvalues lambda[0..nev-1] (descending) by
 * inverse iteration (Sec. 3).  Each solve factors S - lambda I by Gaussian
 * elimination with partial pivoting (pivots of modulus < eps*||S|| raised to
 * that size), starts from a seeded uniform(-1,1) vector, iterates at most 5
 * times and, within a cluster (consecutive eigenvalues closer than
 * 1e-3*||S||_1), orthogonalises (modified Gram-Schmidt) against the earlier
 * vectors of the cluster after every solve.  Converged once the solve grows
 * the unit right-hand side to >= 1/(100 sqrt(n) eps ||S||); one more
 * iteration follows.  Each vector is normalised with its largest-modulus
 * entry (lowest index on ties) made positive.  Q is n x nev, ld ldq.
 * Returns 0, or 1000 + k (0-based k) for the first unconverged vector.     */
int oracle_inverse_iteration(int n, const double *alpha, int nev,
                             const double *lambda, double *Q, int ldq)
{
    if (n <= 0 || nev <= 0) return 0;
    double g = gersh(n, alpha);
    if (n == 1 || g == 0.0) {
        for (int k = 0; k < nev; k++)
            for (int i = 0; i < n; i++) AT(Q, i, k, ldq) = (i == k) ? 1.0 : 0.0;
        return 0;
    }
    size_t sz = (size_t)n;
    double *u0 = malloc(sizeof(double) * sz), *u1 = malloc(sizeof(double) * sz),
           *u2 = malloc(sizeof(double) * sz), *ml = malloc(sizeof(double) * sz),
           *y = malloc(sizeof(double) * sz);
    char *sw = malloc(sz);
    if (!u0 || !u1 || !u2 || !ml || !y || !sw) return -1;
    const double eps = DBL_EPSILON;
    const double ptol = eps * g;
    const double ortol = 1e-3 * g;
    const double grow = 1.0 / (100.0 * sqrt((double)n) * eps * g);
    int info = 0, cstart = 0;
    for (int k = 0; k < nev; k++) {
        if (k > 0 && lambda[k - 1] - lambda[k] > ortol) cstart = k;
        double lam = lambda[k];
        /* LU with partial pivoting of M = S - lam I.  Active row at step i
         * holds (a0 at col i, a1 at col i+1); original row i+1 holds
         * (alpha_i, -lam, alpha_{i+1}).  U row i = (u0, u1, u2).          */
        double a0 = -lam, a1 = alpha[0];
        for (int i = 0; i < n - 1; i++) {
            double l = alpha[i];
            double dn = -lam;
            double un = (i + 1 < n - 1) ? alpha[i + 1] : 0.0;
            if (fabs(a0) >= fabs(l)) {
                double piv = a0;
                if (fabs(piv) < ptol) piv = (piv < 0.0) ? -ptol : ptol;
                u0[i] = piv; u1[i] = a1; u2[i] = 0.0; sw[i] = 0;
                ml[i] = l / piv;
                a0 = dn - ml[i] * a1;
                a1 = un;
            } else {
                u0[i] = l; u1[i] = dn; u2[i] = un; sw[i] = 1;
                ml[i] = a0 / l;
                double na0 = a1 - ml[i] * dn;
                a1 = -ml[i] * un;
                a0 = na0;
            }
        }
        if (fabs(a0) < ptol) a0 = (a0 < 0.0) ? -ptol : ptol;
        u0[n - 1] = a0; u1[n - 1] = 0.0; u2[n - 1] = 0.0;

        double *q = &AT(Q, 0, k, ldq);
        for (int i = 0; i < n; i++) q[i] = start_entry((uint64_t)k + 1, (uint64_t)i);
        double nrm = 0.0;
        for (int i = 0; i < n; i++) nrm += q[i] * q[i];
        nrm = sqrt(nrm);
        for (int i = 0; i < n; i++) q[i] /= nrm;
        int conv = 0, done = 0;
        for (int it = 0; it < 5 && !done; it++) {
            /* forward: apply row interchanges and multipliers */
            for (int i = 0; i < n; i++) y[i] = q[i];
            for (int i = 0; i < n - 1; i++) {
                if (sw[i]) { double t = y[i]; y[i] = y[i + 1]; y[i + 1] = t; }
                y[i + 1] -= ml[i] * y[i];
            }
            /* back substitution with U */
            y[n - 1] /= u0[n - 1];
            if (n >= 2) y[n - 2] = (y[n - 2] - u1[n - 2] * y[n - 1]) / u0[n - 2];
            for (int i = n - 3; i >= 0; i--)
                y[i] = (y[i] - u1[i] * y[i + 1] - u2[i] * y[i + 2]) / u0[i];
            /* orthogonalise against earlier vectors of the cluster */
            for (int p = cstart; p < k; p++) {
                const double *qp = &AT(Q, 0, p, ldq);
                double d = 0.0;
                for (int i = 0; i < n; i++) d += qp[i] * y[i];
                for (int i = 0; i < n; i++) y[i] -= d * qp[i];
            }
            nrm = 0.0;
            for (int i = 0; i < n; i++) nrm += y[i] * y[i];
            nrm = sqrt(nrm);
            if (!(nrm > 0.0) || !isfinite(nrm)) break;
            for (int i = 0; i < n; i++) q[i] = y[i] / nrm;
            if (conv) done = 1;
            else if (nrm >= grow) conv = 1;
        }
        if (!conv && info == 0) info = 1000 + k;
        /* sign: largest-modulus entry positive (lowest index on ties) */
        int imax = 0;
        for (int i = 1; i < n; i++)
            if (fabs(q[i]) > fabs(q[imax])) imax = i;
        if (q[imax] < 0.0)
            for (int i = 0; i < n; i++) q[i] = -q[i];
    }
    free(u0); free(u1); free(u2); free(ml); free(y); free(sw);
    return info;
}

/* Eigenvectors from the zero-diagonal form: for lambda = sigma > 0 of S,
 * B v = sigma u and B^T u = sigma v, so q = [u; v] / sqrt(2) in the shuffled
 * order (u on the even rows, v on the odd rows) and S q = sigma q.  u comes
 * from inverse iteration on B B^T - sigma^2 I (order ceil(n/2), the symmetric
 * tridiagonal with diagonal a_i^2 + b_{i-1}^2 and off-diagonal a_i b_i) by
 * oracle_inverse_iteration's steps (LU with partial pivoting, seeded start,
 * at most 5 solves, Gram-Schmidt within clusters of the squared values),
 * then v = B^T u / sigma, and q is normalised with its largest-modulus entry
 * positive.  lambda[0..nev-1] > 0, descending.  Q is n x nev, ld ldq.
 * Returns 0 or 1000 + k for the first vector whose iteration did not
 * converge; -1 for lambda <= 0 or on allocation failure.                   */
int oracle_bidiag_vectors(int n, const double *alpha, int nev, const double *lambda,
                          double *Q, int ldq)
{
    if (n <= 0 || nev <= 0) return 0;
    const int m = (n + 1) / 2;
    for (int k = 0; k < nev; k++)
        if (!(lambda[k] > 0.0)) return -1;
    double *a = malloc(sizeof(double) * (size_t)m), *b = malloc(sizeof(double) * (size_t)m);
    double *dd = malloc(sizeof(double) * (size_t)m), *ee = malloc(sizeof(double) * (size_t)m);
    double *u0 = malloc(sizeof(double) * (size_t)m), *u1 = malloc(sizeof(double) * (size_t)m);
    double *u2 = malloc(sizeof(double) * (size_t)m), *ml = malloc(sizeof(double) * (size_t)m);
    double *y = malloc(sizeof(double) * (size_t)m), *U = malloc(sizeof(double) * (size_t)m * nev);
    char *sw = malloc((size_t)m);
    if (!a || !b || !dd || !ee || !u0 || !u1 || !u2 || !ml || !y || !U || !sw) {
        free(a); free(b); free(dd); free(ee); free(u0); free(u1); free(u2); free(ml); free(y); free(U); free(sw);
        return -1;
    }
    for (int i = 0; i < m; i++) {
        a[i] = (2 * i <= n - 2) ? alpha[2 * i] : 0.0;
        b[i] = (2 * i + 1 <= n - 2) ? alpha[2 * i + 1] : 0.0;
    }
    /* B B^T: diagonal a_i^2 + b_{i-1}^2, off-diagonal a_i b_i */
    double gs = 0.0;
    for (int i = 0; i < m; i++) {
        dd[i] = a[i] * a[i] + (i > 0 ? b[i - 1] * b[i - 1] : 0.0);
        ee[i] = (i + 1 < m) ? a[i] * b[i] : 0.0;
        double r = fabs(dd[i]) + fabs(ee[i]) + (i > 0 ? fabs(ee[i - 1]) : 0.0);
        if (r > gs) gs = r;
    }
    const double eps = DBL_EPSILON;
    const double ptol = eps * (gs > 0.0 ? gs : 1.0);
    const double ortol = 1e-3 * gs;
    const double grow = 1.0 / (100.0 * sqrt((double)m) * eps * (gs > 0.0 ? gs : 1.0));
    int info = 0, cstart = 0;
    for (int k = 0; k < nev; k++) {
        const double mu = lambda[k] * lambda[k];
        if (k > 0 && lambda[k - 1] * lambda[k - 1] - mu > ortol) cstart = k;
        /* LU with partial pivoting of B B^T - mu I (rows i: ee[i-1], dd[i]-mu, ee[i]) */
        double p0 = dd[0] - mu, p1 = (m > 1) ? ee[0] : 0.0;
        for (int i = 0; i < m - 1; i++) {
            double l = ee[i];
            double dn = dd[i + 1] - mu;
            double un = (i + 2 < m) ? ee[i + 1] : 0.0;
            if (fabs(p0) >= fabs(l)) {
                double piv = p0;
                if (fabs(piv) < ptol) piv = (piv < 0.0) ? -ptol : ptol;
                u0[i] = piv; u1[i] = p1; u2[i] = 0.0; sw[i] = 0;
                ml[i] = l / piv;
                p0 = dn - ml[i] * p1;
                p1 = un;
            } else {
                u0[i] = l; u1[i] = dn; u2[i] = un; sw[i] = 1;
                ml[i] = p0 / l;
                double np0 = p1 - ml[i] * dn;
                p1 = -ml[i] * un;
                p0 = np0;
            }
        }
        if (fabs(p0) < ptol) p0 = (p0 < 0.0) ? -ptol : ptol;
        u0[m - 1] = p0; u1[m - 1] = 0.0; u2[m - 1] = 0.0;
        double *u = &U[(size_t)k * m];
        for (int i = 0; i < m; i++) u[i] = start_entry((uint64_t)k + 1, (uint64_t)i);
        double nrm = 0.0;
        for (int i = 0; i < m; i++) nrm += u[i] * u[i];
        nrm = sqrt(nrm);
        for (int i = 0; i < m; i++) u[i] /= nrm;
        int conv = 0, done = 0;
        for (int it = 0; it < 5 && !done; it++) {
            for (int i = 0; i < m; i++) y[i] = u[i];
            for (int i = 0; i < m - 1; i++) {
                if (sw[i]) { double t = y[i]; y[i] = y[i + 1]; y[i + 1] = t; }
                y[i + 1] -= ml[i] * y[i];
            }
            y[m - 1] /= u0[m - 1];
            if (m >= 2) y[m - 2] = (y[m - 2] - u1[m - 2] * y[m - 1]) / u0[m - 2];
            for (int i = m - 3; i >= 0; i--)
                y[i] = (y[i] - u1[i] * y[i + 1] - u2[i] * y[i + 2]) / u0[i];
            for (int pc = cstart; pc < k; pc++) {
                const double *up = &U[(size_t)pc * m];
                double dt = 0.0;
                for (int i = 0; i < m; i++) dt += up[i] * y[i];
                for (int i = 0; i < m; i++) y[i] -= dt * up[i];
            }
            nrm = 0.0;
            for (int i = 0; i < m; i++) nrm += y[i] * y[i];
            nrm = sqrt(nrm);
            if (!(nrm > 0.0) || !isfinite(nrm)) break;
            for (int i = 0; i < m; i++) u[i] = y[i] / nrm;
            if (conv) done = 1;
            else if (nrm >= grow) conv = 1;
        }
        if (!conv && info == 0) info = 1000 + k;
        /* q: u on the even rows, v = B^T u / sigma on the odd rows */
        double *q = &AT(Q, 0, k, ldq);
        for (int i = 0; i < m; i++) q[2 * i] = u[i];
        for (int i = 0; 2 * i + 1 < n; i++)
            q[2 * i + 1] = (a[i] * u[i] + (i + 1 < m ? b[i] * u[i + 1] : 0.0)) / lambda[k];
        nrm = 0.0;
        for (int i = 0; i < n; i++) nrm += q[i] * q[i];
        nrm = sqrt(nrm);
        int imax = 0;
        for (int i = 1; i < n; i++)
            if (fabs(q[i]) > fabs(q[imax])) imax = i;
        const double sgn = (q[imax] < 0.0) ? -1.0 : 1.0;
        for (int i = 0; i < n; i++) q[i] *= sgn / nrm;
    }
    free(a); free(b); free(dd); free(ee); free(u0); free(u1); free(u2); free(ml); free(y); free(U); free(sw);
    return info;
}

/* Algorithm 1 step 3: z_k = D q_k, D = diag(i^r), r = 0..n-1, split into
 * real and imaginary parts (Sec. 2.3): r mod 4 = 0 -> re = q, 1 -> im = q,
 * 2 -> re = -q, 3 -> im = -q; the other part is 0.                        */
void oracle_dmap(int n, int k, const double *Q, int ldq, double *X, double *Y,
                 int ldz)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < k; j++)
        for (int r = 0; r < n; r++) {
            double q = AT(Q, r, j, ldq);
            double re = 0.0, im = 0.0;
            switch (r & 3) {
            case 0: re = q; break;
            case 1: im = q; break;
            case 2: re = -q; break;
            default: im = -q; break;
            }
            AT(X, r, j, ldz) = re;
            AT(Y, r, j, ldz) = im;
        }
}

/* Full solve: the nev largest lambda (descending) and Z = X + iY with
 * A Z[:,j] = i lambda[j] Z[:,j].  X, Y are n x nev, ld ldz (may be NULL for
 * eigenvalues only).  Returns 0, 1000+k (inverse iteration), <0 on error.  */
int oracle_skew_eig(int n, const double *A, int lda, int nev, double *lambda,
                    double *X, double *Y, int ldz)
{
    if (n < 0 || lda < (n > 1 ? n : 1) || nev < 0 || nev > n / 2) return -1;
    if (n == 0 || nev == 0) return 0;
    double *alpha = calloc((size_t)n, sizeof(double));
    double *tau = calloc((size_t)n, sizeof(double));
    double *V = malloc(sizeof(double) * (size_t)n * n);
    if (!alpha || !tau || !V) { free(alpha); free(tau); free(V); return -2; }
    int info = oracle_tridiagonalize(n, A, lda, alpha, V, tau);
    if (info == 0) info = oracle_bisect(n, alpha, nev, lambda);
    if (info == 0 && X && Y) {
        double *Qd = malloc(sizeof(double) * (size_t)n * nev);
        if (!Qd) info = -2;
        else {
            info = oracle_inverse_iteration(n, alpha, nev, lambda, Qd, n);
            oracle_dmap(n, nev, Qd, n, X, Y, ldz);
            oracle_apply_q(n, V, tau, nev, X, ldz);
            oracle_apply_q(n, V, tau, nev, Y, ldz);
            free(Qd);
        }
    }
    free(alpha); free(tau); free(V);
    return info;
}
