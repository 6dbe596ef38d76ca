// tridiag.cu -- eigenpairs of the symmetric tridiagonal S = tridiag(alpha, 0,
// alpha) obtained from the skew tridiagonal T by Lemma 1 (Eq. 1:
// -i D^H T D = S, D = diag(i^r)), and the D back transformation of
// Algorithm 1 step 3.
//
// Sec. 3 (the solver BSEPACK adapted from ScaLAPACK): bisection + inverse
// iteration.
//   * Bisection: one thread per wanted eigenvalue (the nev largest); Sturm
//     counts from the LDL^T pivots d_0 = -x, d_i = -x - alpha_{i-1}^2/d_{i-1}
//     (tiny pivots replaced by -pivmin); interval [-g, g], g = ||S||_1.
//   * Inverse iteration: Gaussian elimination with partial pivoting of
//     S - lambda I (pivots below eps g raised to eps g), a counter-based
//     (splitmix64) start vector, at most maxit solves, one extra solve after
//     the growth test passes.  Eigenvalues closer than ctol form a cluster; one
//     thread handles a whole cluster and orthogonalises (modified Gram-Schmidt)
//     each new vector against the cluster's earlier vectors after every solve.
//     The largest-modulus entry of each vector is made positive.
// Vectors are kept interleaved, Q[i * nev + k], so consecutive threads
// (consecutive k) touch consecutive addresses in every sweep over i.
#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace sk {
namespace {

struct TriScalars {
    double g;       // ||S||_1
    double pivmin;  // DBL_MIN * max(1, max alpha^2)
};

__global__ void tri_prep_kernel(int n, const double* __restrict__ alpha, double* __restrict__ a2,
                                TriScalars* sc) {
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
    }
}

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

__global__ void bisect_kernel(int n, int nev, const double* __restrict__ a2, const TriScalars* sc,
                              double* __restrict__ lambda) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nev) return;
    const double g = sc->g, pivmin = sc->pivmin;
    if (n == 1 || g == 0.0) { lambda[k] = 0.0; return; }
    const int j = n - 1 - k;  // ascending index of the wanted eigenvalue
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
    lambda[k] = lo + 0.5 * (hi - lo);
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

__global__ void invit_kernel(int n, int nev, const double* __restrict__ alpha,
                             const double* __restrict__ lambda, const TriScalars* sc, double ctol_rel,
                             int maxit, InvitBufs bf, double* __restrict__ Q, int* __restrict__ fail) {
    const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (k0 >= nev) return;
    const double g = sc->g;
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
    TriScalars* sc;
    int* fail;
    InvitBufs bf;
};

TriWs carve_tri(Carve& cv, int n, int nev) {
    TriWs w{};
    size_t nn = (size_t)(n > 0 ? n : 1), ne = (size_t)(nev > 0 ? nev : 1);
    w.a2 = cv.take<double>(nn);
    w.sc = cv.take<TriScalars>(1);
    w.fail = cv.take<int>(1);
    w.bf.u0 = cv.take<double>(nn * ne);
    w.bf.u1 = cv.take<double>(nn * ne);
    w.bf.u2 = cv.take<double>(nn * ne);
    w.bf.ml = cv.take<double>(nn * ne);
    w.bf.sw = cv.take<unsigned char>(nn * ne);
    return w;
}

}  // namespace

size_t tridiag_ws(int n, int nev) {
    Carve cv(nullptr, ~size_t(0));
    carve_tri(cv, n, nev);
    return cv.off + 256;
}

int tridiag_eig(cudaStream_t st, int n, const double* alpha, int nev, double* lambda, double* Qi, void* ws,
                size_t ws_bytes, int* d_status, int maxit) {
    if (n <= 0 || nev <= 0) return 0;
    Carve cv(ws, ws_bytes);
    TriWs w = carve_tri(cv, n, nev);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    tri_prep_kernel<<<1, 1024, 0, st>>>(n, alpha, w.a2, w.sc);
    count_launch();
    bisect_kernel<<<(nev + 127) / 128, 128, 0, st>>>(n, nev, w.a2, w.sc, lambda);
    count_launch();
    if (Qi) {
        // cluster tolerance relative to ||S||_1: 1e-3 for small n (the usual
        // inverse-iteration choice), shrinking like n^-1.5 so that clusters stay
        // small for dense spectra while eps*||S||/gap stays below n*eps.
        double ctol = fmin(1e-3, 10.0 / ((double)n * sqrt((double)n)));
        set_int_kernel<<<1, 32, 0, st>>>(w.fail, 0x7fffffff);
        count_launch();
        invit_kernel<<<(nev + 63) / 64, 64, 0, st>>>(n, nev, alpha, lambda, w.sc, ctol, maxit, w.bf, Qi, w.fail);
        count_launch();
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
