// tridiag.cu -- eigenpairs of the symmetric tridiagonal S = tridiag(alpha, 0,
// alpha) obtained from the skew tridiagonal T by Lemma 1 (Eq. 1:
// -i D^H T D = S, D = diag(i^r)), and the D back transformation of
// Algorithm 1 step 3.
//
// Sec. 3 (the solver BSEPACK adapted from ScaLAPACK): bisection + inverse
// iteration.
//   * Bisection: Sturm counts from the LDL^T pivots d_0 = -x,
//     d_i = -x - alpha_{i-1}^2/d_{i-1} (tiny pivots replaced by -pivmin) on
//     [-g, g], g = ||S||_1, for the nev largest eigenvalues.  GB300 runs FP64
//     at 1/64 of the FP32 rate and the FP64 recurrence is latency-bound
//     (the division chain), so the counts run in three precisions: FP32
//     counts of S / g bracket each eigenvalue to 8 eps32 (four lanes
//     multisect), double-float counts (FP32 pairs) check the bracket widened
//     by 64 eps32 and narrow it to 2^-42, and, where the eigenvalues are not
//     refined afterwards, FP64 counts check it again (widened by 2^-36 g) and
//     finish it with two-lane multisection.  Each floating-point Sturm count
//     is exact for a matrix perturbed by a few units of its roundoff
//     (Kahan), hence the widening before each check.
//   * Inverse iteration: Gaussian elimination with partial pivoting of
//     S - lambda I (pivots below eps g raised to eps g), a counter-based
//     (splitmix64) start vector, at most maxit solves, one extra solve after
//     the growth test passes.  Eigenvalues closer than ctol form a cluster: a
//     lone eigenvalue's vector is one thread's work; a cluster's members
//     iterate in lockstep (each member's solves on its own thread, then the
//     cluster's CTA orthogonalises them in index order by modified
//     Gram-Schmidt, normalises them and applies the growth test).
//     The largest-modulus entry of each vector is made positive.  When the
//     vectors are refined afterwards, the same steps run in double-float
//     arithmetic (eps = 2^-44).
// Vectors are kept interleaved, Q[i * nev + k], so consecutive threads
// (consecutive k) touch consecutive addresses in every sweep over i.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "tridiag_dev.cuh"

namespace sk {
namespace {

using namespace tri;

#ifndef BISECT_LANES
#define BISECT_LANES 2
#endif


__global__ void tri_prep_kernel(int n, const double* __restrict__ alpha, double* __restrict__ a2,
                                float* __restrict__ a2s, float* __restrict__ a2l, float* __restrict__ alh,
                                float* __restrict__ all_, TriScalars* sc, double* __restrict__ a2e,
                                double* __restrict__ b2e) {
    // the bidiagonal of the zero-diagonal form: a_i = alpha_{2i}, b_i = alpha_{2i+1}
    for (int i = threadIdx.x; i < (n + 1) / 2; i += blockDim.x) {
        const double a = (2 * i <= n - 2) ? alpha[2 * i] : 0.0;
        const double b = (2 * i + 1 <= n - 2) ? alpha[2 * i + 1] : 0.0;
        a2e[i] = a * a;
        b2e[i] = b * b;
    }
    __shared__ double red[32];
    double gmax = 0.0, amax = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double al = (i < n - 1) ? alpha[i] : 0.0;
        double ap = (i > 0) ? alpha[i - 1] : 0.0;
        if (i < n - 1) a2[i] = al * al;
        gmax = fmax(gmax, fabs(al) + fabs(ap));
        amax = fmax(amax, al * al);
    }
    // block max (reuse the sum helper pattern with fmax)
    for (int o = 16; o > 0; o >>= 1) {
        gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
        amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double red2[32];
    if (lane == 0) { red[warp] = gmax; red2[warp] = amax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double g = 0.0, a = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; w++) { g = fmax(g, red[w]); a = fmax(a, red2[w]); }
        sc->g = g;
        sc->pivmin = DBL_MIN * fmax(1.0, a);
        red[0] = g;
    }
    __syncthreads();
    // alpha^2 / g^2 as an FP32 pair (a2s + a2l) for the bracketing passes
    // (entries below FLT_MIN become 0: a perturbation far below their
    // tolerances)
    const double g = red[0], ig2 = (g > 0.0) ? 1.0 / (g * g) : 0.0;
    for (int i = threadIdx.x; i < n - 1; i += blockDim.x) {
        const double v = a2[i] * ig2;
        const float h = (float)v;
        a2s[i] = h;
        a2l[i] = (float)(v - (double)h);
        const float ah = (float)alpha[i];  // alpha itself as a pair (double-float inverse iteration)
        alh[i] = ah;
        all_[i] = (float)(alpha[i] - (double)ah);
    }
}

constexpr float PIV_DF = 7.888609052210118e-31f;  // 2^-100: pivots of S / g raised to this

// Double-float Sturm count of S / g at x (the recurrence of sturm()).
__device__ __forceinline__ int sturm_df(int n, const float* __restrict__ a2s, const float* __restrict__ a2l, Df x) {
    int cnt = 0;
    Df d = {-x.h, -x.l};
    if (fabsf(d.h) < PIV_DF) d = {-PIV_DF, 0.f};
    cnt += (d.h < 0.f);
    for (int i = 1; i < n; i++) {
        const Df t = df_add(x, df_div({a2s[i - 1], a2l[i - 1]}, d));
        d = {-t.h, -t.l};
        if (fabsf(d.h) < PIV_DF) d = {-PIV_DF, 0.f};
        cnt += (d.h < 0.f);
    }
    return cnt;
}

// FP32 Sturm count of the scaled matrix S / g at x (|x| ~ 1): the recurrence
// of sturm() with pivots below FLT_MIN raised to FLT_MIN.
__device__ __forceinline__ int sturm32(int n, const float* __restrict__ a2s, float x) {
    int cnt = 0;
    float d = -x;
    if (fabsf(d) < FLT_MIN) d = -FLT_MIN;
    cnt += (d < 0.f);
    for (int i = 1; i < n; i++) {
        d = -x - __fdividef(a2s[i - 1], d);
        if (fabsf(d) < FLT_MIN) d = -FLT_MIN;
        cnt += (d < 0.f);
    }
    return cnt;
}

// Bracketing pass in FP32 (64 times the FP64 rate on this part): four lanes
// per wanted eigenvalue multisect [-1, 1] for S / g down to 8 eps32.  A
// floating-point Sturm count is the exact count of a matrix whose entries are
// perturbed by a few units of roundoff (Kahan), so lambda_j lies within a few
// eps32 g of the FP32 bracket; the FP64 pass widens it by FP32_SLACK eps32 g
// and checks it with FP64 counts before trusting it.
__global__ void bisect32_kernel(int n, int nev, const float* __restrict__ a2s, const TriScalars* sc,
                                double* __restrict__ lohi) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = gt >> 2, q = gt & 3, lane = threadIdx.x & 31;
    if (k >= nev) return;
    const unsigned gmask = 0xFu << (lane & ~3);
    const int j = n - 1 - k;
    float lo = -1.0f - 4.0f * FLT_EPSILON, hi = 1.0f + 4.0f * FLT_EPSILON;
    for (int it = 0; it < 64; it++) {
        const float w = hi - lo;
        if (w <= 8.0f * FLT_EPSILON) break;
        const float step = w * 0.2f;
        const float x = lo + (float)(q + 1) * step;
        const bool le = (x > lo && x < hi) ? (sturm32(n, a2s, x) <= j) : (x <= lo);
        const int nle = __popc(__ballot_sync(gmask, le) & gmask);
        const float nlo = (nle > 0) ? lo + (float)nle * step : lo;
        const float nhi = (nle < 4) ? lo + (float)(nle + 1) * step : hi;
        if (!(nlo > lo || nhi < hi)) break;
        lo = nlo;
        hi = (nhi < hi) ? nhi : hi;
    }
    if (q == 0) {
        lohi[2 * k] = (double)lo;  // in units of g
        lohi[2 * k + 1] = (double)hi;
    }
}

// Second pass: four lanes multisect the FP32 bracket (widened by FP32_SLACK
// eps32, checked with double-float counts and widened eightfold until the
// check holds) with double-float counts down to DF_WIDTH.  Writes the
// bracket (units of g) back and, in lambda, its midpoint times g.
constexpr double FP32_SLACK = 64.0;
constexpr double DF_WIDTH = 1.0 / 4398046511104.0;  // 2^-42
__global__ void bisect_df_kernel(int n, int nev, const float* __restrict__ a2s, const float* __restrict__ a2l,
                                 const TriScalars* sc, double* __restrict__ lohi, double* __restrict__ lambda) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = gt >> 2, q = gt & 3, lane = threadIdx.x & 31;
    if (k >= nev) return;
    const unsigned gmask = 0xFu << (lane & ~3);
    const int j = n - 1 - k;
    const double g = sc->g;
    if (n == 1 || g == 0.0) {
        if (q == 0) lambda[k] = 0.0;
        return;
    }
    const double glo = -1.0 - 1e-6, ghi = 1.0 + 1e-6;
    double lo = glo, hi = ghi;
    double slack = FP32_SLACK * FLT_EPSILON;
    for (int tries = 0; tries < 8; tries++) {
        const double a = fmax(glo, lohi[2 * k] - slack), b = fmin(ghi, lohi[2 * k + 1] + slack);
        bool mine = true;
        if (q == 0) mine = (a == glo) || sturm_df(n, a2s, a2l, df_of(a)) <= j;
        if (q == 1) mine = (b == ghi) || sturm_df(n, a2s, a2l, df_of(b)) > j;
        if ((__ballot_sync(gmask, !mine) & gmask) == 0u) {
            lo = a;
            hi = b;
            break;
        }
        slack *= 8.0;
    }
    for (int it = 0; it < 64; it++) {
        const double w = hi - lo;
        if (w <= DF_WIDTH) break;
        const double step = w * 0.2;
        const double x = lo + (double)(q + 1) * step;
        const bool le = (x > lo && x < hi) ? (sturm_df(n, a2s, a2l, df_of(x)) <= j) : (x <= lo);
        const int nle = __popc(__ballot_sync(gmask, le) & gmask);
        const double nlo = (nle > 0) ? lo + (double)nle * step : lo;
        const double nhi = (nle < 4) ? lo + (double)(nle + 1) * step : hi;
        if (!(nlo > lo || nhi < hi)) break;
        lo = nlo;
        hi = (nhi < hi) ? nhi : hi;
    }
    if (q == 0) {
        lohi[2 * k] = lo;
        lohi[2 * k + 1] = hi;
        lambda[k] = (lo + 0.5 * (hi - lo)) * g;
    }
}

constexpr double DF_SLACK = 1.0 / 68719476736.0;  // 2^-36: widening of a double-float bracket (units of g)

// FP64 multisection with L lanes per wanted eigenvalue (L = 1: bisection):
// each lane counts at one of L equally spaced interior points, the interval
// shrinks to 1 / (L + 1) per step (stopping rule of bisect_one).  With lohi,
// the start is the double-float bracket (units of g) widened by DF_SLACK g
// once its ends pass the FP64 counts count(lo) <= j < count(hi); a bracket
// that fails is widened eightfold, up to the whole Gershgorin interval.
// BD: counts from the zero-diagonal form (B B^T at x^2, m = ceil(n/2) steps;
// the wanted eigenvalues are >= 0, so the search stays in [0, g]).
template <int L, bool BD = false>
__global__ void bisect_kernel(int n, int nev, const double* __restrict__ a2, const TriScalars* sc,
                              const double* __restrict__ lohi, double* __restrict__ lambda,
                              const double* __restrict__ a2e = nullptr, const double* __restrict__ b2e = nullptr) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = gt / L, q = gt % L, lane = threadIdx.x & 31;
    if (k >= nev) return;  // whole lane groups leave together (blockDim is a multiple of L)
    const unsigned gmask = (L == 1) ? (1u << lane) : (((1u << L) - 1u) << (lane & ~(L - 1)));
    const double g = sc->g, pivmin = sc->pivmin;
    const int m = (n + 1) / 2;
    const int j = BD ? m - 1 - k : n - 1 - k;  // ascending index of the wanted eigenvalue
    // count(x) <= j: the wanted eigenvalue is >= x
    auto below = [&](double x) -> bool {
        return BD ? bd_count(m, a2e, b2e, pivmin, x * x) <= j : sturm(n, a2, pivmin, x) <= j;
    };
    if (n == 1 || g == 0.0) {
        if (q == 0) lambda[k] = 0.0;
        return;
    }
    const double glo = BD ? 0.0 : -g - 2.0 * DBL_EPSILON * g - pivmin, ghi = g + 2.0 * DBL_EPSILON * g + pivmin;
    double lo = glo, hi = ghi;
    if (lohi) {
        double slack = DF_SLACK * g;
        for (int tries = 0; tries < 8; tries++) {
            const double a = fmax(glo, lohi[2 * k] * g - slack), b = fmin(ghi, lohi[2 * k + 1] * g + slack);
            bool ok;
            if (L == 1) {
                ok = (a == glo || below(a)) && (b == ghi || !below(b));
            } else {
                // lane 0 checks the lower end, lane 1 the upper one
                bool mine = true;
                if (q == 0) mine = (a == glo) || below(a);
                if (q == 1) mine = (b == ghi) || !below(b);
                ok = (__ballot_sync(gmask, !mine) & gmask) == 0u;
            }
            if (ok) {
                lo = a;
                hi = b;
                break;
            }
            slack *= 8.0;
        }
    }
    for (int it = 0; it < 4000; it++) {
        const double w = hi - lo;
        const double tol = 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + DBL_MIN;
        if (w <= tol) break;
        const double step = w / (double)(L + 1);
        const double x = lo + (double)(q + 1) * step;
        const bool le = (x > lo && x < hi) ? below(x) : (x <= lo);
        // counts grow with x: the lanes with lambda_j >= x_q are a prefix
        const int nle = (L == 1) ? (le ? 1 : 0) : __popc(__ballot_sync(gmask, le) & gmask);
        const double nlo = (nle > 0) ? lo + (double)nle * step : lo;
        const double nhi = (nle < L) ? lo + (double)(nle + 1) * step : hi;
        if (!(nlo > lo || nhi < hi)) break;  // no representable progress
        lo = nlo;
        hi = (nhi < hi) ? nhi : hi;
    }
    if (q == 0) lambda[k] = lo + 0.5 * (hi - lo);
}

// ---- lockstep inverse iteration of clusters ---------------------------------
// A cluster (two or more eigenvalues closer than ctol) is iterated in lockstep
// rather than by one thread: in every iteration each member solves with its
// own LU on its own thread, then the cluster's CTA orthogonalises the members
// in index order (modified Gram-Schmidt, parallel over the rows), normalises
// them and applies the growth test to each; the cluster stops one iteration
// after all its members passed.  The vectors are an orthonormal basis of the
// same invariant subspace, and the critical path is one member's solves
// instead of the whole cluster's (16 x at the 1e-10 clusters of a clustered
// spectrum).  Singletons keep the one-thread path.
constexpr int CLU_T = 256;

__global__ void clu_list_kernel(int nev, const double* __restrict__ lambda, const TriScalars* sc, double ctol_rel,
                                int2* __restrict__ list, int* __restrict__ count, int* __restrict__ state) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double ctol = ctol_rel * sc->g;
    int c = 0, k0 = 0;
    for (int k = 1; k <= nev; k++) {
        if (k == nev || starts_cluster(lambda, k, ctol)) {
            if (k - k0 >= 2) {
                list[c] = make_int2(k0, k - k0);
                state[c] = 0;
                c++;
            }
            k0 = k;
        }
    }
    *count = c;
}

// Row of the largest abs(x_i) (the lowest on ties), CTA-wide.
template <class F>
__device__ __forceinline__ int block_argmax(int n, F absval, double* rv, int* ri) {
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double a = absval(i);
        if (a > best) {
            best = a;
            bi = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) {
        rv[warp] = best;
        ri[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; w++)
            if (rv[w] > rv[0] || (rv[w] == rv[0] && ri[w] < ri[0])) {
                rv[0] = rv[w];
                ri[0] = ri[w];
            }
    }
    __syncthreads();
    const int r = ri[0];
    __syncthreads();
    return r < n ? r : 0;
}

// Decision after an iteration: state 0 iterating, 1 all members passed (one
// more iteration), 2 done.  ff = first member that failed the growth test
// (m if none), bad = a member's norm was zero or not finite.
__device__ __forceinline__ int clu_next_state(int st, int ff, int m, int bad, int it, int maxit, bool& fin,
                                              bool& failed) {
    int nst = (st == 1) ? 2 : (ff == m ? 1 : 0);
    if (bad) nst = 0;
    fin = bad || nst == 2 || it == maxit - 1;
    failed = fin && nst == 0;
    return nst;
}

__global__ void __launch_bounds__(CLU_T)
invit_clu_kernel(int n, int nev, const double* __restrict__ alpha, const double* __restrict__ lambda,
                 const TriScalars* sc, int maxit, int it, InvitBufs bf, double* __restrict__ Q,
                 const int2* __restrict__ list, const int* __restrict__ count, int* __restrict__ state,
                 int* __restrict__ fail) {
    __shared__ double red[32];
    __shared__ int redi[32];
    __shared__ int s_ff, s_bad;
    const int nc = *count;
    const double g = sc->g;
    const size_t ld = (size_t)nev;
    const double eps = DBL_EPSILON, ptol = eps * g;
    const double grow = 1.0 / (100.0 * sqrt((double)n) * eps * g);
    const int t = threadIdx.x, T = blockDim.x;
    for (int b = blockIdx.x; b < nc; b += gridDim.x) {
        const int2 cl = list[b];
        const int k0 = cl.x, m = cl.y;
        const int st = state[b];
        if (st == 2) continue;
        if (n == 1 || g == 0.0) {
            for (int e = t; e < m * n; e += T) {
                const int j = e / n, i = e % n;
                Q[i * ld + k0 + j] = (i == k0 + j) ? 1.0 : 0.0;
            }
            __syncthreads();
            if (t == 0) state[b] = 2;
            continue;
        }
        // the members' solves, one thread each
        for (int j = t; j < m; j += T) {
            const int k = k0 + j;
            if (it == 0) {
                invit_lu(n, alpha, lambda[k], ptol, bf, ld, k);
                invit_start(n, Q, ld, k);
            }
            invit_solve(n, bf, Q, ld, k);
        }
        if (t == 0) {
            s_ff = m;
            s_bad = 0;
        }
        __syncthreads();
        // modified Gram-Schmidt in index order, normalisation, growth test
        for (int j = 0; j < m; j++) {
            double* qj = Q + k0 + j;
            for (int p = 0; p < j; p++) {
                const double* qp = Q + k0 + p;
                double d = 0.0;
                for (int i = t; i < n; i += T) d = fma(qp[i * ld], qj[i * ld], d);
                d = sk_block_sum(d, red);
                for (int i = t; i < n; i += T) qj[i * ld] = fma(-d, qp[i * ld], qj[i * ld]);
                __syncthreads();
            }
            double s = 0.0;
            for (int i = t; i < n; i += T) s = fma(qj[i * ld], qj[i * ld], s);
            const double nrm = sqrt(sk_block_sum(s, red));
            if (!(nrm > 0.0) || !isfinite(nrm)) {
                if (t == 0) {
                    s_bad = 1;
                    s_ff = min(s_ff, j);
                }
            } else {
                const double inv = 1.0 / nrm;
                for (int i = t; i < n; i += T) qj[i * ld] *= inv;
                if (t == 0 && !(nrm >= grow)) s_ff = min(s_ff, j);
            }
            __syncthreads();
        }
        bool fin, failed;
        const int nst = clu_next_state(st, s_ff, m, s_bad, it, maxit, fin, failed);
        if (failed && t == 0) atomicMin(fail, k0 + s_ff);
        if (fin) {
            // largest-modulus entry of each vector positive (lowest index on ties)
            for (int j = 0; j < m; j++) {
                double* qj = Q + k0 + j;
                const int imax = block_argmax(n, [&](int i) { return fabs(qj[i * ld]); }, red, redi);
                const bool neg = qj[imax * ld] < 0.0;  // read by all before any flip
                __syncthreads();
                if (neg)
                    for (int i = t; i < n; i += T) qj[i * ld] = -qj[i * ld];
                __syncthreads();
            }
        }
        if (t == 0) state[b] = fin ? 2 : nst;
        __syncthreads();
    }
}

// CTA-wide double-float sum (fixed order: deterministic).
__device__ __forceinline__ Df df_block_sum(Df v, float* rh, float* rl) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = df_add(v, Df{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)});
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) {
        rh[warp] = v.h;
        rl[warp] = v.l;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Df s = {rh[0], rl[0]};
        for (int w = 1; w < nw; w++) s = df_add(s, Df{rh[w], rl[w]});
        rh[0] = s.h;
        rl[0] = s.l;
    }
    __syncthreads();
    const Df r = {rh[0], rl[0]};
    __syncthreads();
    return r;
}

// The lockstep cluster iteration in double-float (the vectors refined
// afterwards); the members are converted to FP64 when the cluster is done.
__global__ void __launch_bounds__(CLU_T)
invit_clu_df_kernel(int n, int nev, const float* __restrict__ alh, const float* __restrict__ all_,
                    const double* __restrict__ lambda, const TriScalars* sc, int maxit, int it, InvitBufs bf,
                    double* __restrict__ Q, const int2* __restrict__ list, const int* __restrict__ count,
                    int* __restrict__ state, int* __restrict__ fail) {
    __shared__ float rh[32], rl[32];
    __shared__ double red[32];
    __shared__ int redi[32];
    __shared__ int s_ff, s_bad;
    const int nc = *count;
    const double g = sc->g;
    const size_t ld = (size_t)nev;
    const double eps = 1.0 / 17592186044416.0;  // 2^-44
    const float ptol = (float)(eps * g);
    const float grow = (float)(1.0 / (100.0 * sqrt((double)n) * eps * g));
    const InvitDf v = invit_df_view(bf, Q);
    Df* Qd = v.Qd;
    const int t = threadIdx.x, T = blockDim.x;
    for (int b = blockIdx.x; b < nc; b += gridDim.x) {
        const int2 cl = list[b];
        const int k0 = cl.x, m = cl.y;
        const int st = state[b];
        if (st == 2) continue;
        if (n == 1 || g == 0.0) {
            for (int e = t; e < m * n; e += T) {
                const int j = e / n, i = e % n;
                Q[i * ld + k0 + j] = (i == k0 + j) ? 1.0 : 0.0;
            }
            __syncthreads();
            if (t == 0) state[b] = 2;
            continue;
        }
        for (int j = t; j < m; j += T) {
            const int k = k0 + j;
            if (it == 0) {
                invit_lu_df(n, alh, all_, lambda[k], ptol, v, ld, k);
                invit_start_df(n, Qd, ld, k);
            }
            invit_solve_df(n, v, ld, k);
        }
        if (t == 0) {
            s_ff = m;
            s_bad = 0;
        }
        __syncthreads();
        for (int j = 0; j < m; j++) {
            Df* qj = Qd + k0 + j;
            for (int p = 0; p < j; p++) {
                const Df* qp = Qd + k0 + p;
                Df d = {0.f, 0.f};
                for (int i = t; i < n; i += T) d = df_add(d, df_mul(qp[i * ld], qj[i * ld]));
                const Df md = df_neg(df_block_sum(d, rh, rl));
                for (int i = t; i < n; i += T) qj[i * ld] = df_add(qj[i * ld], df_mul(md, qp[i * ld]));
                __syncthreads();
            }
            float s = 0.f;
            for (int i = t; i < n; i += T) {
                const float y = qj[i * ld].h;
                s = fmaf(y, y, s);
            }
            const float nrm = sqrtf(sk_block_sum(s, rh));
            if (!(nrm > 0.f) || !isfinite(nrm)) {
                if (t == 0) {
                    s_bad = 1;
                    s_ff = min(s_ff, j);
                }
            } else {
                const Df sc1 = {1.0f / nrm, 0.f};
                for (int i = t; i < n; i += T) qj[i * ld] = df_mul(qj[i * ld], sc1);
                if (t == 0 && !(nrm >= grow)) s_ff = min(s_ff, j);
            }
            __syncthreads();
        }
        bool fin, failed;
        const int nst = clu_next_state(st, s_ff, m, s_bad, it, maxit, fin, failed);
        if (failed && t == 0) atomicMin(fail, k0 + s_ff);
        if (fin) {
            for (int j = 0; j < m; j++) {
                Df* qj = Qd + k0 + j;
                const int imax = block_argmax(n, [&](int i) { return (double)fabsf(qj[i * ld].h); }, red, redi);
                const bool neg = qj[imax * ld].h < 0.f;  // read by all before any flip
                __syncthreads();
                for (int i = t; i < n; i += T) {
                    const Df y = qj[i * ld];
                    Q[i * ld + k0 + j] = df_to_double(neg ? df_neg(y) : y);
                }
                __syncthreads();
            }
        }
        if (t == 0) state[b] = fin ? 2 : nst;
        __syncthreads();
    }
}

__global__ void invit_df_kernel(int n, int nev, const float* __restrict__ alh, const float* __restrict__ all_,
                                const double* __restrict__ lambda, const TriScalars* sc, double ctol_rel, int maxit,
                                InvitBufs bf, double* __restrict__ Q, int* __restrict__ fail) {
    const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (k0 >= nev) return;
    invit_cluster_df(n, nev, alh, all_, lambda, sc->g, ctol_rel, maxit, bf, Q, fail, k0, true);
}

__global__ void invit_kernel(int n, int nev, const double* __restrict__ alpha,
                             const double* __restrict__ lambda, const TriScalars* sc, double ctol_rel,
                             int maxit, InvitBufs bf, double* __restrict__ Q, int* __restrict__ fail) {
    const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (k0 >= nev) return;
    invit_cluster(n, nev, alpha, lambda, sc->g, ctol_rel, maxit, bf, Q, fail, k0, true);
}

__global__ void set_int_kernel(int* p, int v) {
    if (threadIdx.x == 0) *p = v;
}

__global__ void invit_status_kernel(const int* fail, int nev, int* status) {
    if (threadIdx.x == 0 && *fail < nev) sk_set_error(status, SKEW_INFO_INVIT_BASE + *fail);
}

// Qi (n x nev interleaved: Qi[i * nev + k]) -> X (n x nev, ld ldz) [+ Y]:
// with dmap, entry i of column k is i^i * q: i mod 4 = 0 -> X = q, 1 -> Y = q,
// 2 -> X = -q, 3 -> Y = -q (Algorithm 1 step 3).
__global__ void transpose_dmap_kernel(int n, int nev, const double* __restrict__ Qi, double* __restrict__ X,
                                      double* __restrict__ Y, int ldz, int dmap) {
    __shared__ double tile[32][33];
    const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        int i = i0 + r, k = k0 + tx;
        tile[r][tx] = (i < n && k < nev) ? Qi[(size_t)i * nev + k] : 0.0;
    }
    __syncthreads();
    for (int c = ty; c < 32; c += 8) {
        int k = k0 + c, i = i0 + tx;
        if (i < n && k < nev) {
            double q = tile[tx][c];
            size_t at = (size_t)k * ldz + i;
            if (!dmap) {
                X[at] = q;
            } else {
                int m4 = i & 3;
                X[at] = (m4 == 0) ? q : (m4 == 2 ? -q : 0.0);
                Y[at] = (m4 == 1) ? q : (m4 == 3 ? -q : 0.0);
            }
        }
    }
}

__global__ void dmap_colmajor_kernel(int n, int k, const double* __restrict__ Q, int ldq, double* __restrict__ X,
                                     double* __restrict__ Y, int ldz) {
    size_t total = (size_t)n * k;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        double q = Q[(size_t)j * ldq + i];
        int m4 = i & 3;
        X[(size_t)j * ldz + i] = (m4 == 0) ? q : (m4 == 2 ? -q : 0.0);
        Y[(size_t)j * ldz + i] = (m4 == 1) ? q : (m4 == 3 ? -q : 0.0);
    }
}

struct TriWs {
    double* a2;
    double *a2e, *b2e;  // alpha_{2i}^2, alpha_{2i+1}^2 (zero-diagonal form, ceil(n/2) each)
    float *a2s, *a2l;  // alpha^2 / g^2 as an FP32 pair (bracketing passes)
    float *alh, *all_;  // alpha as an FP32 pair (double-float inverse iteration)
    double* lohi;   // FP32 brackets, 2 per wanted eigenvalue
    TriScalars* sc;
    int* fail;
    InvitBufs bf;
    int2* clist;  // clusters of two or more: (first index, size)
    int *ccount, *cstate;
};

TriWs carve_tri(Carve& cv, int n, int nev) {
    TriWs w{};
    size_t nn = (size_t)(n > 0 ? n : 1), ne = (size_t)(nev > 0 ? nev : 1);
    w.a2 = cv.take<double>(nn);
    w.a2e = cv.take<double>(nn / 2 + 1);
    w.b2e = cv.take<double>(nn / 2 + 1);
    w.a2s = cv.take<float>(nn);
    w.a2l = cv.take<float>(nn);
    w.alh = cv.take<float>(nn);
    w.all_ = cv.take<float>(nn);
    w.lohi = cv.take<double>(2 * ne);
    w.sc = cv.take<TriScalars>(1);
    w.fail = cv.take<int>(1);
    w.bf.u0 = cv.take<double>(nn * ne);
    w.bf.u1 = cv.take<double>(nn * ne);
    w.bf.u2 = cv.take<double>(nn * ne);
    w.bf.ml = cv.take<double>(nn * ne);
    w.bf.sw = cv.take<unsigned char>(nn * ne);
    w.clist = cv.take<int2>(ne / 2 + 1);
    w.ccount = cv.take<int>(1);
    w.cstate = cv.take<int>(ne / 2 + 1);
    return w;
}

}  // namespace

size_t tridiag_ws(int n, int nev) {
    Carve cv(nullptr, ~size_t(0));
    carve_tri(cv, n, nev);
    return cv.off + 256;
}

int tridiag_eig(cudaStream_t st, int n, const double* alpha, int nev, double* lambda, double* Qi, void* ws,
                size_t ws_bytes, int* d_status, int maxit, bool fp64, bool bidiag) {
    if (n <= 0 || nev <= 0) return 0;
    Carve cv(ws, ws_bytes);
    TriWs w = carve_tri(cv, n, nev);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    tri_prep_kernel<<<1, 1024, 0, st>>>(n, alpha, w.a2, w.a2s, w.a2l, w.alh, w.all_, w.sc, w.a2e, w.b2e);
    count_launch();
    {
        KtScope kt(st, KT_BISECT);
        bisect32_kernel<<<(4 * nev + 127) / 128, 128, 0, st>>>(n, nev, w.a2s, w.sc, w.lohi);
        bisect_df_kernel<<<(4 * nev + 127) / 128, 128, 0, st>>>(n, nev, w.a2s, w.a2l, w.sc, w.lohi, lambda);
        count_launch(2);
        if (fp64 && bidiag && 2 * nev <= n) {
            // FP64 finish on the zero-diagonal form (half-length counts)
            bisect_kernel<BISECT_LANES, true><<<(BISECT_LANES * nev + 63) / 64, 64, 0, st>>>(
                n, nev, w.a2, w.sc, w.lohi, lambda, w.a2e, w.b2e);
            count_launch();
        } else if (fp64) {
            bisect_kernel<BISECT_LANES><<<(BISECT_LANES * nev + 63) / 64, 64, 0, st>>>(n, nev, w.a2, w.sc, w.lohi,
                                                                                        lambda);
            count_launch();
        }
    }
    if (Qi) {
        // cluster tolerance relative to ||S||_1: 1e-3 for small n (the usual
        // inverse-iteration choice), shrinking like n^-1.5 so that clusters stay
        // small for dense spectra while eps*||S||/gap stays below n*eps.
        double ctol = fmin(1e-3, 10.0 / ((double)n * sqrt((double)n)));
        set_int_kernel<<<1, 32, 0, st>>>(w.fail, 0x7fffffff);
        count_launch();
        {
            KtScope kt(st, KT_INVIT);
            // singletons one thread each; clusters in lockstep, one CTA each
            if (fp64)
                invit_kernel<<<(nev + 63) / 64, 64, 0, st>>>(n, nev, alpha, lambda, w.sc, ctol, maxit, w.bf, Qi,
                                                             w.fail);
            else
                invit_df_kernel<<<(nev + 63) / 64, 64, 0, st>>>(n, nev, w.alh, w.all_, lambda, w.sc, ctol, maxit,
                                                                w.bf, Qi, w.fail);
            count_launch();
            clu_list_kernel<<<1, 32, 0, st>>>(nev, lambda, w.sc, ctol, w.clist, w.ccount, w.cstate);
            count_launch();
            const int cgrid = std::max(1, std::min(nev / 2, 2 * device_sms()));
            for (int it = 0; it < maxit; it++) {
                if (fp64)
                    invit_clu_kernel<<<cgrid, CLU_T, 0, st>>>(n, nev, alpha, lambda, w.sc, maxit, it, w.bf, Qi,
                                                              w.clist, w.ccount, w.cstate, w.fail);
                else
                    invit_clu_df_kernel<<<cgrid, CLU_T, 0, st>>>(n, nev, w.alh, w.all_, lambda, w.sc, maxit, it,
                                                                 w.bf, Qi, w.clist, w.ccount, w.cstate, w.fail);
                count_launch();
            }
        }
        invit_status_kernel<<<1, 32, 0, st>>>(w.fail, nev, d_status);
        count_launch();
    }
    return cudaGetLastError() == cudaSuccess ? 0 : SKEW_ERR_CUDA;
}

cudaError_t interleaved_to_colmajor(cudaStream_t st, int n, int nev, const double* Qi, double* X, double* Y,
                                    int ldz, bool dmap) {
    if (n <= 0 || nev <= 0) return cudaSuccess;
    dim3 grid((n + 31) / 32, (nev + 31) / 32), block(32, 8);
    transpose_dmap_kernel<<<grid, block, 0, st>>>(n, nev, Qi, X, Y, ldz, dmap ? 1 : 0);
    count_launch();
    return cudaGetLastError();
}

cudaError_t dmap_colmajor(cudaStream_t st, int n, int k, const double* Q, int ldq, double* X, double* Y, int ldz) {
    if (n <= 0 || k <= 0) return cudaSuccess;
    size_t total = (size_t)n * k;
    int grid = (int)((total + 255) / 256 > 8192 ? 8192 : (total + 255) / 256);
    dmap_colmajor_kernel<<<grid, 256, 0, st>>>(n, k, Q, ldq, X, Y, ldz);
    count_launch();
    return cudaGetLastError();
}

}  // namespace sk
