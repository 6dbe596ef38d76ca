// tridiag_dev.cuh -- device routines of the tridiagonal eigensolver (Sec. 3:
// bisection + inverse iteration on S = tridiag(alpha, 0, alpha)), shared by
// the single-matrix kernels and the batched ones.
#pragma once
#include <cfloat>
#include <cmath>

#include "common.cuh"

namespace sk {
namespace tri {

struct TriScalars {
    double g;       // ||S||_1
    double pivmin;  // DBL_MIN * max(1, max alpha^2)
};

__device__ __forceinline__ int sturm(int n, const double* __restrict__ a2, double pivmin, double x) {
    int cnt = 0;
    double d = -x;
    if (fabs(d) < pivmin) d = -pivmin;
    cnt += (d < 0.0);
    for (int i = 1; i < n; i++) {
        d = -x - a2[i - 1] / d;
        if (fabs(d) < pivmin) d = -pivmin;
        cnt += (d < 0.0);
    }
    return cnt;
}

// The wanted eigenvalue of ascending index j (Sturm bisection on [-g, g]).
__device__ __forceinline__ double bisect_one(int n, int j, const double* __restrict__ a2, double g, double pivmin) {
    if (n == 1 || g == 0.0) return 0.0;
    double lo = -g - 2.0 * DBL_EPSILON * g - pivmin;
    double hi = g + 2.0 * DBL_EPSILON * g + pivmin;
    for (int it = 0; it < 4000; it++) {
        double w = hi - lo;
        double tol = 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + DBL_MIN;
        if (w <= tol) break;
        double mid = lo + 0.5 * w;
        if (mid <= lo || mid >= hi) break;
        if (sturm(n, a2, pivmin, mid) <= j) lo = mid;
        else hi = mid;
    }
    return lo + 0.5 * (hi - lo);
}

__device__ __forceinline__ double splitmix_uniform(unsigned long long seed, unsigned long long i) {
    // splitmix64 (Steele, Lea, Flood 2014) of seed * golden + i -> uniform(-1, 1)
    unsigned long long z = seed * 0x9E3779B97F4A7C15ULL + i + 0x632BE59BD9B4E019ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

struct InvitBufs {
    double *u0, *u1, *u2, *ml;
    unsigned char* sw;
};

// Inverse iteration for the cluster led by eigenvalue k0 (nothing unless k0
// starts a cluster): vectors into Q[i * nev + k], LU rows in bf (same layout).
__device__ __forceinline__ void invit_cluster(int n, int nev, const double* __restrict__ alpha,
                                              const double* __restrict__ lambda, double g, double ctol_rel,
                                              int maxit, const InvitBufs& bf, double* __restrict__ Q,
                                              int* __restrict__ fail, int k0) {
    const double ctol = ctol_rel * g;
    if (k0 > 0 && !(lambda[k0 - 1] - lambda[k0] > ctol)) return;  // not a cluster leader
    int k1 = k0 + 1;
    while (k1 < nev && !(lambda[k1 - 1] - lambda[k1] > ctol)) k1++;
    const size_t ld = (size_t)nev;
    if (n == 1 || g == 0.0) {
        for (int k = k0; k < k1; k++)
            for (int i = 0; i < n; i++) Q[i * ld + k] = (i == k) ? 1.0 : 0.0;
        return;
    }
    const double eps = DBL_EPSILON;
    const double ptol = eps * g;
    const double grow = 1.0 / (100.0 * sqrt((double)n) * eps * g);
    for (int k = k0; k < k1; k++) {
        const double lam = lambda[k];
        // ---- LU with partial pivoting of S - lam I (U rows: u0, u1, u2)
        double a0 = -lam, a1 = alpha[0];
        for (int i = 0; i < n - 1; i++) {
            const double l = alpha[i], dn = -lam;
            const double un = (i + 1 < n - 1) ? alpha[i + 1] : 0.0;
            const size_t at = i * ld + k;
            if (fabs(a0) >= fabs(l)) {
                double piv = a0;
                if (fabs(piv) < ptol) piv = (piv < 0.0) ? -ptol : ptol;
                double m = l / piv;
                bf.u0[at] = piv; bf.u1[at] = a1; bf.u2[at] = 0.0; bf.sw[at] = 0; bf.ml[at] = m;
                a0 = dn - m * a1;
                a1 = un;
            } else {
                double m = a0 / l;
                bf.u0[at] = l; bf.u1[at] = dn; bf.u2[at] = un; bf.sw[at] = 1; bf.ml[at] = m;
                double na0 = a1 - m * dn;
                a1 = -m * un;
                a0 = na0;
            }
        }
        if (fabs(a0) < ptol) a0 = (a0 < 0.0) ? -ptol : ptol;
        {
            const size_t at = (size_t)(n - 1) * ld + k;
            bf.u0[at] = a0; bf.u1[at] = 0.0; bf.u2[at] = 0.0;
        }
        // ---- start vector
        double nrm = 0.0;
        for (int i = 0; i < n; i++) {
            double x = splitmix_uniform((unsigned long long)k + 1ULL, (unsigned long long)i);
            Q[i * ld + k] = x;
            nrm = fma(x, x, nrm);
        }
        nrm = 1.0 / sqrt(nrm);
        for (int i = 0; i < n; i++) Q[i * ld + k] *= nrm;
        bool conv = false, done = false;
        for (int it = 0; it < maxit && !done; it++) {
            // forward: interchanges and multipliers
            double prev = Q[k];
            for (int i = 0; i < n - 1; i++) {
                const size_t at = i * ld + k;
                double next = Q[at + ld];
                if (bf.sw[at]) { double tmp = prev; prev = next; next = tmp; }
                Q[at] = prev;
                prev = next - bf.ml[at] * prev;
            }
            Q[(size_t)(n - 1) * ld + k] = prev;
            // back substitution
            double y2 = 0.0, y1 = prev / bf.u0[(size_t)(n - 1) * ld + k];
            Q[(size_t)(n - 1) * ld + k] = y1;
            for (int i = n - 2; i >= 0; i--) {
                const size_t at = i * ld + k;
                double y = (Q[at] - bf.u1[at] * y1 - bf.u2[at] * y2) / bf.u0[at];
                Q[at] = y;
                y2 = y1;
                y1 = y;
            }
            // orthogonalise against the earlier vectors of the cluster
            for (int p = k0; p < k; p++) {
                double d = 0.0;
                for (int i = 0; i < n; i++) d = fma(Q[i * ld + p], Q[i * ld + k], d);
                for (int i = 0; i < n; i++) Q[i * ld + k] = fma(-d, Q[i * ld + p], Q[i * ld + k]);
            }
            nrm = 0.0;
            for (int i = 0; i < n; i++) { double y = Q[i * ld + k]; nrm = fma(y, y, nrm); }
            nrm = sqrt(nrm);
            if (!(nrm > 0.0) || !isfinite(nrm)) break;
            const double inv = 1.0 / nrm;
            for (int i = 0; i < n; i++) Q[i * ld + k] *= inv;
            if (conv) done = true;
            else if (nrm >= grow) conv = true;
        }
        if (!conv) atomicMin(fail, k);
        // sign: largest-modulus entry positive (lowest index on ties)
        int imax = 0;
        double vmax = fabs(Q[k]);
        for (int i = 1; i < n; i++) {
            double a = fabs(Q[i * ld + k]);
            if (a > vmax) { vmax = a; imax = i; }
        }
        if (Q[imax * ld + k] < 0.0)
            for (int i = 0; i < n; i++) Q[i * ld + k] = -Q[i * ld + k];
    }
}

}  // namespace tri
}  // namespace sk
