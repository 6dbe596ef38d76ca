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

// Zero-diagonal form (Sec. 2.2, remark after Algorithm 1): with the unknowns
// shuffled even first, S = [[0, B], [B^T, 0]], B lower bidiagonal with
// diagonal a_i = alpha_{2i} and subdiagonal b_i = alpha_{2i+1}; the
// eigenvalues >= 0 of S are the square roots of those of B B^T (order
// m = ceil(n/2)).  Number of eigenvalues of B B^T below t from the stationary
// qd transform of its L D L^T form (D_i = a_i^2, l_i = b_i / a_i):
// D+_i = a_i^2 + s_i, s_{i+1} = b_i^2 s_i / D+_i - t, s_0 = -t (one division per
// step over m steps, against n steps of the full Sturm count).
__device__ __forceinline__ int bd_count(int m, const double* __restrict__ a2e, const double* __restrict__ b2e,
                                        double pivmin, double t) {
    int cnt = 0;
    double sv = -t;
    for (int i = 0; i < m; i++) {
        double d = a2e[i] + sv;
        if (fabs(d) < pivmin) d = -pivmin;
        cnt += (d < 0.0);
        sv = b2e[i] * sv / d - t;
    }
    return cnt;
}

// The k-th largest eigenvalue (k < n/2) of S by bisection on x in [0, g] with
// counts of B B^T at t = x^2 (ascending index m - 1 - k there).
__device__ __forceinline__ double bisect_one_bd(int m, int k, const double* __restrict__ a2e,
                                                const double* __restrict__ b2e, double g, double pivmin) {
    if (m < 1 || g == 0.0) return 0.0;  // m = 1 (n = 2): the eigenvalue |alpha_0|
    const int j = m - 1 - k;
    double lo = 0.0, hi = g + 2.0 * DBL_EPSILON * g + pivmin;
    for (int it = 0; it < 4000; it++) {
        double w = hi - lo;
        double tol = 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + DBL_MIN;
        if (w <= tol) break;
        double mid = lo + 0.5 * w;
        if (mid <= lo || mid >= hi) break;
        if (bd_count(m, a2e, b2e, pivmin, mid * mid) <= j) lo = mid;
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

// ---- double-float (FP32 pair) arithmetic: Dekker, "A floating-point
// technique for extending the available precision" (1971); Knuth's two_sum.
// About 46 bits, at FP32-pipe latency.
struct Df {
    float h, l;
};
__device__ __forceinline__ Df df_of(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ Df df_fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
// (a + b) with an error below a few 2^-46 (|a| + |b|): as a perturbation of
// the shift and of the quotient separately, which a Sturm count tolerates
__device__ __forceinline__ Df df_add(Df a, Df b) {
    const float s = a.h + b.h;
    const float bb = s - a.h;
    const float e = (a.h - (s - bb)) + (b.h - bb);
    return df_fast_two_sum(s, e + (a.l + b.l));
}
// a / b: quotient of the leading parts, corrected by the exact remainder
__device__ __forceinline__ Df df_div(Df a, Df b) {
    const float q1 = __fdividef(a.h, b.h);
    const float p1 = q1 * b.h;
    const float p2 = fmaf(q1, b.h, -p1);
    const float r = (((a.h - p1) - p2) + a.l) - q1 * b.l;
    return df_fast_two_sum(q1, __fdividef(r, b.h));
}

__device__ __forceinline__ Df df_mul(Df a, Df b) {
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p) + (a.h * b.l + a.l * b.h);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ Df df_neg(Df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ double df_to_double(Df a) { return (double)a.h + (double)a.l; }

struct InvitBufs {
    double *u0, *u1, *u2, *ml;
    unsigned char* sw;
};

// ---- inverse iteration, one vector (column k of the interleaved buffers) ----
// LU with partial pivoting of S - lam I (U rows u0, u1, u2; multipliers ml;
// interchanges sw); pivots below ptol are raised to ptol.
__device__ __forceinline__ void invit_lu(int n, const double* __restrict__ alpha, double lam, double ptol,
                                         const InvitBufs& bf, size_t ld, int k) {
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
    const size_t at = (size_t)(n - 1) * ld + k;
    bf.u0[at] = a0; bf.u1[at] = 0.0; bf.u2[at] = 0.0;
}

// The sweeps below are sequential in i and each thread owns column k: loads
// run IB elements ahead of the dependent arithmetic (a store to element i
// never precedes the load of element i), so the chain waits on global memory
// once per IB elements instead of once per element.
constexpr int INV_IB = 8;

// Counter-based start vector (splitmix64 of (k + 1, i)), normalised.
__device__ __forceinline__ void invit_start(int n, double* __restrict__ Q, size_t ld, int k) {
    double nrm = 0.0;
    for (int i = 0; i < n; i++) {
        double x = splitmix_uniform((unsigned long long)k + 1ULL, (unsigned long long)i);
        Q[i * ld + k] = x;
        nrm = fma(x, x, nrm);
    }
    nrm = 1.0 / sqrt(nrm);
    for (int i = 0; i < n; i++) Q[i * ld + k] *= nrm;
}

// One solve with the stored LU, in place on column k.
__device__ __forceinline__ void invit_solve(int n, const InvitBufs& bf, double* __restrict__ Q, size_t ld, int k) {
    // forward: interchanges and multipliers
    double prev = Q[k];
    for (int i0 = 0; i0 < n - 1; i0 += INV_IB) {
        double nx[INV_IB], ml[INV_IB];
        unsigned char sw[INV_IB];
#pragma unroll
        for (int u = 0; u < INV_IB; u++)
            if (i0 + u < n - 1) {
                const size_t at = (size_t)(i0 + u) * ld + k;
                nx[u] = Q[at + ld];
                ml[u] = bf.ml[at];
                sw[u] = bf.sw[at];
            }
#pragma unroll
        for (int u = 0; u < INV_IB; u++)
            if (i0 + u < n - 1) {
                double next = nx[u];
                if (sw[u]) { double tmp = prev; prev = next; next = tmp; }
                Q[(size_t)(i0 + u) * ld + k] = prev;
                prev = next - ml[u] * prev;
            }
    }
    Q[(size_t)(n - 1) * ld + k] = prev;
    // back substitution
    double y2 = 0.0, y1 = prev / bf.u0[(size_t)(n - 1) * ld + k];
    Q[(size_t)(n - 1) * ld + k] = y1;
    for (int i0 = n - 2; i0 >= 0; i0 -= INV_IB) {
        double q[INV_IB], u0[INV_IB], u1[INV_IB], u2[INV_IB];
#pragma unroll
        for (int u = 0; u < INV_IB; u++)
            if (i0 - u >= 0) {
                const size_t at = (size_t)(i0 - u) * ld + k;
                q[u] = Q[at];
                u0[u] = bf.u0[at];
                u1[u] = bf.u1[at];
                u2[u] = bf.u2[at];
            }
#pragma unroll
        for (int u = 0; u < INV_IB; u++)
            if (i0 - u >= 0) {
                double y = (q[u] - u1[u] * y1 - u2[u] * y2) / u0[u];
                Q[(size_t)(i0 - u) * ld + k] = y;
                y2 = y1;
                y1 = y;
            }
    }
}

// Largest-modulus entry of column k made positive (lowest index on ties).
__device__ __forceinline__ void invit_sign(int n, double* __restrict__ Q, size_t ld, int k) {
    int imax = 0;
    double vmax = fabs(Q[k]);
    for (int i = 1; i < n; i++) {
        double a = fabs(Q[i * ld + k]);
        if (a > vmax) { vmax = a; imax = i; }
    }
    if (Q[imax * ld + k] < 0.0)
        for (int i = 0; i < n; i++) Q[i * ld + k] = -Q[i * ld + k];
}

// Cluster membership: eigenvalue k continues the cluster of k - 1 unless
// lambda[k-1] - lambda[k] > ctol.
__device__ __forceinline__ bool starts_cluster(const double* __restrict__ lambda, int k, double ctol) {
    return k == 0 || lambda[k - 1] - lambda[k] > ctol;
}

// Inverse iteration for the cluster led by eigenvalue k0 (nothing unless k0
// starts a cluster): vectors into Q[i * nev + k], LU rows in bf (same layout).
// One thread handles the whole cluster, orthogonalising each new vector
// against the cluster's earlier vectors after every solve.  singles_only:
// clusters of two or more are left to the lockstep cluster kernel.
__device__ __forceinline__ void invit_cluster(int n, int nev, const double* __restrict__ alpha,
                                              const double* __restrict__ lambda, double g, double ctol_rel,
                                              int maxit, const InvitBufs& bf, double* __restrict__ Q,
                                              int* __restrict__ fail, int k0, bool singles_only = false) {
    const double ctol = ctol_rel * g;
    if (!starts_cluster(lambda, k0, ctol)) return;  // not a cluster leader
    int k1 = k0 + 1;
    while (k1 < nev && !starts_cluster(lambda, k1, ctol)) k1++;
    if (singles_only && k1 - k0 > 1) return;
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
        invit_lu(n, alpha, lambda[k], ptol, bf, ld, k);
        invit_start(n, Q, ld, k);
        bool conv = false, done = false;
        for (int it = 0; it < maxit && !done; it++) {
            invit_solve(n, bf, Q, ld, k);
            // orthogonalise against the earlier vectors of the cluster
            for (int p = k0; p < k; p++) {
                double d = 0.0;
                for (int i = 0; i < n; i++) d = fma(Q[i * ld + p], Q[i * ld + k], d);
                for (int i = 0; i < n; i++) Q[i * ld + k] = fma(-d, Q[i * ld + p], Q[i * ld + k]);
            }
            double nrm = 0.0;
            for (int i = 0; i < n; i++) { double y = Q[i * ld + k]; nrm = fma(y, y, nrm); }
            nrm = sqrt(nrm);
            if (!(nrm > 0.0) || !isfinite(nrm)) break;
            const double inv = 1.0 / nrm;
            for (int i = 0; i < n; i++) Q[i * ld + k] *= inv;
            if (conv) done = true;
            else if (nrm >= grow) conv = true;
        }
        if (!conv) atomicMin(fail, k);
        invit_sign(n, Q, ld, k);
    }
}

// Inverse iteration in double-float (about 2^-44 relative; Dekker's pair
// arithmetic runs at FP32 latency, the FP64 division chain here is about ten
// times longer): for a caller that refines the vectors afterwards.  The steps
// are those of the FP64 routines with the pivot floor and growth threshold
// taken at 2^-44; the LU rows and the vectors are kept as FP32 pairs in the
// same buffers, and the vectors are converted to FP64 at the end.  alpha as a
// pair: alh + all_.
struct InvitDf {
    Df *U0, *U1, *U2, *ML, *Qd;
    unsigned char* sw;
};
__device__ __forceinline__ InvitDf invit_df_view(const InvitBufs& bf, double* Q) {
    return {reinterpret_cast<Df*>(bf.u0), reinterpret_cast<Df*>(bf.u1), reinterpret_cast<Df*>(bf.u2),
            reinterpret_cast<Df*>(bf.ml), reinterpret_cast<Df*>(Q), bf.sw};
}

__device__ __forceinline__ void invit_lu_df(int n, const float* __restrict__ alh, const float* __restrict__ all_,
                                            double lam, float ptol, const InvitDf& v, size_t ld, int k) {
    const Df zero = {0.f, 0.f};
    const Df mlam = df_neg(df_of(lam));
    Df a0 = mlam, a1 = {alh[0], all_[0]};
    for (int i = 0; i < n - 1; i++) {
        const Df l = {alh[i], all_[i]};
        const Df un = (i + 1 < n - 1) ? Df{alh[i + 1], all_[i + 1]} : zero;
        const size_t at = i * ld + k;
        if (fabsf(a0.h) >= fabsf(l.h)) {
            Df piv = a0;
            if (fabsf(piv.h) < ptol) piv = {(piv.h < 0.f) ? -ptol : ptol, 0.f};
            const Df m = df_div(l, piv);
            v.U0[at] = piv; v.U1[at] = a1; v.U2[at] = zero; v.sw[at] = 0; v.ML[at] = m;
            a0 = df_add(mlam, df_neg(df_mul(m, a1)));
            a1 = un;
        } else {
            const Df m = df_div(a0, l);
            v.U0[at] = l; v.U1[at] = mlam; v.U2[at] = un; v.sw[at] = 1; v.ML[at] = m;
            const Df na0 = df_add(a1, df_neg(df_mul(m, mlam)));
            a1 = df_neg(df_mul(m, un));
            a0 = na0;
        }
    }
    if (fabsf(a0.h) < ptol) a0 = {(a0.h < 0.f) ? -ptol : ptol, 0.f};
    const size_t at = (size_t)(n - 1) * ld + k;
    v.U0[at] = a0; v.U1[at] = zero; v.U2[at] = zero;
}

__device__ __forceinline__ void invit_scale_df(int n, Df* __restrict__ Qd, size_t ld, int k, Df s) {
    for (int i0 = 0; i0 < n; i0 += INV_IB) {
        Df x[INV_IB];
#pragma unroll
        for (int u = 0; u < INV_IB; u++)
            if (i0 + u < n) x[u] = Qd[(size_t)(i0 + u) * ld + k];
#pragma unroll
        for (int u = 0; u < INV_IB; u++)
            if (i0 + u < n) Qd[(size_t)(i0 + u) * ld + k] = df_mul(x[u], s);
    }
}

// the FP64 routine's start vector, norm in FP32
__device__ __forceinline__ void invit_start_df(int n, Df* __restrict__ Qd, size_t ld, int k) {
    float nrm = 0.f;
    for (int i = 0; i < n; i++) {
        const Df x = df_of(splitmix_uniform((unsigned long long)k + 1ULL, (unsigned long long)i));
        Qd[i * ld + k] = x;
        nrm = fmaf(x.h, x.h, nrm);
    }
    invit_scale_df(n, Qd, ld, k, {1.0f / sqrtf(nrm), 0.f});
}

__device__ __forceinline__ void invit_solve_df(int n, const InvitDf& v, size_t ld, int k) {
    const Df zero = {0.f, 0.f};
    Df* Qd = v.Qd;
    // forward: interchanges and multipliers
    Df prev = Qd[k];
    for (int i0 = 0; i0 < n - 1; i0 += INV_IB) {
        Df nx[INV_IB], ml[INV_IB];
        unsigned char sw[INV_IB];
#pragma unroll
        for (int u = 0; u < INV_IB; u++)
            if (i0 + u < n - 1) {
                const size_t at = (size_t)(i0 + u) * ld + k;
                nx[u] = Qd[at + ld];
                ml[u] = v.ML[at];
                sw[u] = v.sw[at];
            }
#pragma unroll
        for (int u = 0; u < INV_IB; u++)
            if (i0 + u < n - 1) {
                Df next = nx[u];
                if (sw[u]) { const Df tmp = prev; prev = next; next = tmp; }
                Qd[(size_t)(i0 + u) * ld + k] = prev;
                prev = df_add(next, df_neg(df_mul(ml[u], prev)));
            }
    }
    // back substitution
    Df y2 = zero, y1 = df_div(prev, v.U0[(size_t)(n - 1) * ld + k]);
    Qd[(size_t)(n - 1) * ld + k] = y1;
    for (int i0 = n - 2; i0 >= 0; i0 -= INV_IB) {
        Df q[INV_IB], u0[INV_IB], u1[INV_IB], u2[INV_IB];
#pragma unroll
        for (int u = 0; u < INV_IB; u++)
            if (i0 - u >= 0) {
                const size_t at = (size_t)(i0 - u) * ld + k;
                q[u] = Qd[at];
                u0[u] = v.U0[at];
                u1[u] = v.U1[at];
                u2[u] = v.U2[at];
            }
#pragma unroll
        for (int u = 0; u < INV_IB; u++)
            if (i0 - u >= 0) {
                const Df r = df_add(q[u], df_neg(df_add(df_mul(u1[u], y1), df_mul(u2[u], y2))));
                const Df y = df_div(r, u0[u]);
                Qd[(size_t)(i0 - u) * ld + k] = y;
                y2 = y1;
                y1 = y;
            }
    }
}

__device__ __forceinline__ void invit_sign_df(int n, Df* __restrict__ Qd, size_t ld, int k) {
    int imax = 0;
    float vmax = fabsf(Qd[k].h);
    for (int i = 1; i < n; i++) {
        const float a = fabsf(Qd[i * ld + k].h);
        if (a > vmax) { vmax = a; imax = i; }
    }
    if (Qd[imax * ld + k].h < 0.f)
        for (int i = 0; i < n; i++) Qd[i * ld + k] = df_neg(Qd[i * ld + k]);
}

__device__ __forceinline__ void invit_cluster_df(int n, int nev, const float* __restrict__ alh,
                                                 const float* __restrict__ all_, const double* __restrict__ lambda,
                                                 double g, double ctol_rel, int maxit, const InvitBufs& bf,
                                                 double* __restrict__ Q, int* __restrict__ fail, int k0,
                                                 bool singles_only = false) {
    const double ctol = ctol_rel * g;
    if (!starts_cluster(lambda, k0, ctol)) return;  // not a cluster leader
    int k1 = k0 + 1;
    while (k1 < nev && !starts_cluster(lambda, k1, ctol)) k1++;
    if (singles_only && k1 - k0 > 1) return;
    const size_t ld = (size_t)nev;
    if (n == 1 || g == 0.0) {
        for (int k = k0; k < k1; k++)
            for (int i = 0; i < n; i++) Q[i * ld + k] = (i == k) ? 1.0 : 0.0;
        return;
    }
    const double eps = 1.0 / 17592186044416.0;  // 2^-44
    const float ptol = (float)(eps * g);
    const float grow = (float)(1.0 / (100.0 * sqrt((double)n) * eps * g));
    const InvitDf v = invit_df_view(bf, Q);
    Df* Qd = v.Qd;
    const Df zero = {0.f, 0.f};
    for (int k = k0; k < k1; k++) {
        invit_lu_df(n, alh, all_, lambda[k], ptol, v, ld, k);
        invit_start_df(n, Qd, ld, k);
        bool conv = false, done = false;
        for (int it = 0; it < maxit && !done; it++) {
            invit_solve_df(n, v, ld, k);
            // orthogonalise against the earlier vectors of the cluster
            for (int p = k0; p < k; p++) {
                Df d = zero;
                for (int i = 0; i < n; i++) d = df_add(d, df_mul(Qd[i * ld + p], Qd[i * ld + k]));
                const Df md = df_neg(d);
                for (int i0 = 0; i0 < n; i0 += INV_IB) {
                    Df a[INV_IB], b[INV_IB];
#pragma unroll
                    for (int u = 0; u < INV_IB; u++)
                        if (i0 + u < n) {
                            a[u] = Qd[(size_t)(i0 + u) * ld + k];
                            b[u] = Qd[(size_t)(i0 + u) * ld + p];
                        }
#pragma unroll
                    for (int u = 0; u < INV_IB; u++)
                        if (i0 + u < n) Qd[(size_t)(i0 + u) * ld + k] = df_add(a[u], df_mul(md, b[u]));
                }
            }
            float nrm = 0.f;
            for (int i = 0; i < n; i++) { const float y = Qd[i * ld + k].h; nrm = fmaf(y, y, nrm); }
            nrm = sqrtf(nrm);
            if (!(nrm > 0.f) || !isfinite(nrm)) break;
            invit_scale_df(n, Qd, ld, k, {1.0f / nrm, 0.f});
            if (conv) done = true;
            else if (nrm >= grow) conv = true;
        }
        if (!conv) atomicMin(fail, k);
        invit_sign_df(n, Qd, ld, k);
    }
    for (int k = k0; k < k1; k++)
        for (int i = 0; i < n; i++) Q[i * ld + k] = df_to_double(Qd[i * ld + k]);
}

}  // namespace tri
}  // namespace sk
