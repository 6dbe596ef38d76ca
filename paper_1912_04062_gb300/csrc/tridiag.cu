// tridiag.cu -- eigenpairs of the symmetric tridiagonal S = tridiag(alpha, 0,
// alpha) obtained from the skew tridiagonal T by Lemma 1 (Eq. 1:
// -i D^H T D = S, D = diag(i^r)), and the D back transformation of
// Algorithm 1 step 3.
//
// Sec. 3 (the solver BSEPACK adapted from ScaLAPACK): bisection + inverse
// iteration.
//   * Bisection: four lanes per wanted eigenvalue (the nev largest) count at
//     four interior points per step (multisection); Sturm
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
#include "tridiag_dev.cuh"

namespace sk {
namespace {

using namespace tri;


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

// Multisection: four lanes per wanted eigenvalue each count at one of four
// equally spaced interior points of the current interval, which shrinks to one
// fifth per step (same Sturm recurrence and stopping rule as bisect_one).
__global__ void bisect4_kernel(int n, int nev, const double* __restrict__ a2, const TriScalars* sc,
                               double* __restrict__ lambda) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = gt >> 2, q = gt & 3, lane = threadIdx.x & 31;
    if (k >= nev) return;  // whole groups of four leave together (blockDim is a multiple of 4)
    const unsigned gmask = 0xFu << (lane & ~3);
    const double g = sc->g, pivmin = sc->pivmin;
    const int j = n - 1 - k;  // ascending index of the wanted eigenvalue
    if (n == 1 || g == 0.0) {
        if (q == 0) lambda[k] = 0.0;
        return;
    }
    double lo = -g - 2.0 * DBL_EPSILON * g - pivmin;
    double hi = g + 2.0 * DBL_EPSILON * g + pivmin;
    for (int it = 0; it < 2000; it++) {
        const double w = hi - lo;
        const double tol = 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + DBL_MIN;
        if (w <= tol) break;
        const double step = w * 0.2;
        const double x = lo + (double)(q + 1) * step;
        const bool le = (x > lo && x < hi) ? (sturm(n, a2, pivmin, x) <= j) : (x <= lo);
        // counts grow with x: the lanes with lambda_j >= x_q are a prefix
        const int nle = __popc(__ballot_sync(gmask, le) & gmask);
        const double nlo = (nle > 0) ? lo + (double)nle * step : lo;
        const double nhi = (nle < 4) ? lo + (double)(nle + 1) * step : hi;
        if (!(nlo > lo || nhi < hi)) break;  // no representable progress
        lo = nlo;
        hi = (nhi < hi) ? nhi : hi;
    }
    if (q == 0) lambda[k] = lo + 0.5 * (hi - lo);
}

__global__ void invit_kernel(int n, int nev, const double* __restrict__ alpha,
                             const double* __restrict__ lambda, const TriScalars* sc, double ctol_rel,
                             int maxit, InvitBufs bf, double* __restrict__ Q, int* __restrict__ fail) {
    const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (k0 >= nev) return;
    invit_cluster(n, nev, alpha, lambda, sc->g, ctol_rel, maxit, bf, Q, fail, k0);
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
    {
        KtScope kt(st, KT_BISECT);
        bisect4_kernel<<<(4 * nev + 127) / 128, 128, 0, st>>>(n, nev, w.a2, w.sc, lambda);
    }
    count_launch();
    if (Qi) {
        // cluster tolerance relative to ||S||_1: 1e-3 for small n (the usual
        // inverse-iteration choice), shrinking like n^-1.5 so that clusters stay
        // small for dense spectra while eps*||S||/gap stays below n*eps.
        double ctol = fmin(1e-3, 10.0 / ((double)n * sqrt((double)n)));
        set_int_kernel<<<1, 32, 0, st>>>(w.fail, 0x7fffffff);
        count_launch();
        {
            KtScope kt(st, KT_INVIT);
            invit_kernel<<<(nev + 63) / 64, 64, 0, st>>>(n, nev, alpha, lambda, w.sc, ctol, maxit, w.bf, Qi, w.fail);
        }
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
