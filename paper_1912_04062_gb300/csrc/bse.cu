// bse.cu -- device kernels of the Bethe-Salpeter driver around the skew
// solver (Sec. 3: the structure-preserving method for a definite
// H_BS = [[A, B], [-conj(B), -conj(A)]], A Hermitian, B complex symmetric):
//   1. M = J H = [[Re(A+B), Im(A-B)], [-Im(A+B), Re(A-B)]] (Eq. SymmetricM),
//      real symmetric, positive definite when H_BS is definite;
//   2. M = L L^T (Cholesky, lower);
//   3. the skew-symmetric eigenproblem of K = L^T J L, J = [[0, I], [-I, 0]];
//   4. the eigenvectors back: x = L^-T z solves H x = -i lambda x, and
//      psi = Q x with the unitary Q = [[I, -iI], [I, iI]] / sqrt(2) of
//      Theorem 1 is the eigenvector of H_BS for lambda > 0; psi is scaled to
//      psi^H S psi = 1, S = diag(I, -I) (for orthonormal z it is 1/lambda).
// Steps 2 and 4 are blocked by 64: the diagonal blocks and the panels'
// triangular solves are kernels of their own, the trailing updates FP64
// products (lower tiles for the Cholesky, full for the back substitution).
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace sk {
namespace {

constexpr int CB = 64;

__global__ void bse_build_m_kernel(int h, const double* __restrict__ Ar, const double* __restrict__ Ai, int lda,
                                   const double* __restrict__ Br, const double* __restrict__ Bi, int ldb,
                                   double* __restrict__ M, int ldm) {
    const long long N = 2LL * h, total = N * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % N), j = (int)(e / N);
        const int bi = i >= h, bj = j >= h, ii = i - bi * h, jj = j - bj * h;
        const double ar = Ar[ii + (size_t)jj * lda], ai = Ai[ii + (size_t)jj * lda];
        const double br = Br[ii + (size_t)jj * ldb], bm = Bi[ii + (size_t)jj * ldb];
        double v;
        if (!bi && !bj) v = ar + br;          // Re(A + B)
        else if (!bi && bj) v = ai - bm;      // Im(A - B)
        else if (bi && !bj) v = -(ai + bm);   // -Im(A + B)
        else v = ar - br;                     // Re(A - B)
        M[i + (size_t)j * ldm] = v;
    }
}

// Unblocked Cholesky of the kb x kb diagonal block (lower, in place), right
// looking; a pivot that is not positive and finite records
// SKEW_ERR_NOT_DEFINITE and stops the factorisation of the block.
__global__ void __launch_bounds__(256) chol_diag_kernel(int kb, double* __restrict__ D, int ld, int* status) {
    __shared__ double S[CB][CB + 1];
    __shared__ int bad;
    const int t = threadIdx.x;
    for (int e = t; e < kb * kb; e += blockDim.x) {
        const int i = e % kb, j = e / kb;
        S[i][j] = (i >= j) ? D[i + (size_t)j * ld] : 0.0;
    }
    if (t == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < kb; j++) {
        if (t == 0) {
            const double d = S[j][j];
            if (!(d > 0.0) || !isfinite(d)) {
                bad = 1;
                sk_set_error(status, SKEW_ERR_NOT_DEFINITE);
            } else {
                S[j][j] = sqrt(d);
            }
        }
        __syncthreads();
        if (bad) break;
        const double dj = S[j][j];
        for (int i = j + 1 + t; i < kb; i += blockDim.x) S[i][j] /= dj;
        __syncthreads();
        const int m = kb - j - 1;
        for (int e = t; e < m * m; e += blockDim.x) {
            const int i = j + 1 + e % m, l = j + 1 + e / m;
            if (l <= i) S[i][l] = fma(-S[i][j], S[l][j], S[i][l]);
        }
        __syncthreads();
    }
    for (int e = t; e < kb * kb; e += blockDim.x) {
        const int i = e % kb, j = e / kb;
        if (i >= j) D[i + (size_t)j * ld] = S[i][j];
    }
}

// Panel below a factored diagonal block: P <- P L11^-T (row r: x L11^T = p by
// forward substitution), and NP = -P for the trailing update's second factor.
__global__ void __launch_bounds__(128) chol_panel_kernel(int m, int kb, const double* __restrict__ L11, int ld,
                                                         double* __restrict__ P, double* __restrict__ NP, int ldn) {
    __shared__ double Ls[CB][CB + 1];
    const int t = threadIdx.x;
    for (int e = t; e < kb * kb; e += blockDim.x) {
        const int i = e % kb, j = e / kb;
        Ls[i][j] = (i >= j) ? L11[i + (size_t)j * ld] : 0.0;
    }
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + t;
    if (r >= m) return;
    double x[CB];
#pragma unroll
    for (int j = 0; j < CB; j++) x[j] = (j < kb) ? P[r + (size_t)j * ld] : 0.0;
#pragma unroll
    for (int j = 0; j < CB; j++) {
        if (j < kb) {
            double s = x[j];
            for (int l = 0; l < j; l++) s = fma(-x[l], Ls[j][l], s);
            x[j] = s / Ls[j][j];
        }
    }
#pragma unroll
    for (int j = 0; j < CB; j++) {
        if (j < kb) {
            P[r + (size_t)j * ld] = x[j];
            NP[r + (size_t)j * ldn] = -x[j];
        }
    }
}

// L (lower, strict upper part of the factored M set to zero) and
// JL = [L[h:, :]; -L[:h, :]].
__global__ void bse_jl_kernel(int h, double* __restrict__ L, int ld, double* __restrict__ JL, int ldj) {
    const long long N = 2LL * h, total = N * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % N), j = (int)(e / N);
        const int src = (i < h) ? i + h : i - h;
        const double v = (src >= j) ? L[src + (size_t)j * ld] : 0.0;
        JL[i + (size_t)j * ldj] = (i < h) ? v : -v;
        if (i < j) L[i + (size_t)j * ld] = 0.0;
    }
}

// Back substitution with one diagonal block: X_I <- L_II^-T X_I, one thread per
// right-hand side column (L_II^T x = z: x_j = (z_j - sum_{l > j} L_lj x_l) / L_jj).
__global__ void __launch_bounds__(128) trsm_lt_diag_kernel(int kb, const double* __restrict__ Lii, int ld,
                                                           double* __restrict__ X, int ldx, int ncols) {
    __shared__ double Ls[CB][CB + 1];
    const int t = threadIdx.x;
    for (int e = t; e < kb * kb; e += blockDim.x) {
        const int i = e % kb, j = e / kb;
        Ls[i][j] = (i >= j) ? Lii[i + (size_t)j * ld] : 0.0;
    }
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + t;
    if (c >= ncols) return;
    double x[CB];
#pragma unroll
    for (int j = 0; j < CB; j++) x[j] = (j < kb) ? X[j + (size_t)c * ldx] : 0.0;
#pragma unroll
    for (int j = CB - 1; j >= 0; j--) {
        if (j < kb) {
            double s = x[j];
            for (int l = j + 1; l < kb; l++) s = fma(-Ls[l][j], x[l], s);
            x[j] = s / Ls[j][j];
        }
    }
#pragma unroll
    for (int j = 0; j < CB; j++)
        if (j < kb) X[j + (size_t)c * ldx] = x[j];
}

// psi = Q x sqrt(lambda), x = Xr + i Xi (2h x nev), Q = [[I, -iI], [I, iI]] / sqrt(2)
__global__ void bse_psi_kernel(int h, int nev, const double* __restrict__ Xr, const double* __restrict__ Xi, int ldx,
                               const double* __restrict__ lambda, double* __restrict__ Pr, double* __restrict__ Pi,
                               int ldp) {
    const long long total = (long long)h * nev;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % h), k = (int)(e / h);
        const double s = sqrt(fmax(lambda[k], 0.0)) * 0.70710678118654752440;
        const size_t c = (size_t)k * ldx, o = (size_t)k * ldp;
        const double rt = Xr[c + i], rb = Xr[c + i + h], it = Xi[c + i], ib = Xi[c + i + h];
        Pr[o + i] = s * (rt + ib);
        Pi[o + i] = s * (it - rb);
        Pr[o + i + h] = s * (rt - ib);
        Pi[o + i + h] = s * (it + rb);
    }
}

inline int grid_of(long long total) {
    long long g = (total + 255) / 256;
    return (int)(g > 16384 ? 16384 : (g < 1 ? 1 : g));
}

}  // namespace

cudaError_t bse_build_m(cudaStream_t st, int h, const double* Ar, const double* Ai, int lda, const double* Br,
                        const double* Bi, int ldb, double* M, int ldm) {
    bse_build_m_kernel<<<grid_of(4LL * h * h), 256, 0, st>>>(h, Ar, Ai, lda, Br, Bi, ldb, M, ldm);
    count_launch();
    return cudaGetLastError();
}

// M (N x N, ld) <- its lower Cholesky factor; NP: scratch of N x 64.
cudaError_t cholesky_lower(cudaStream_t st, int N, double* M, int ld, double* NP, int* status) {
    for (int k0 = 0; k0 < N; k0 += CB) {
        const int kb = (N - k0 < CB) ? N - k0 : CB;
        double* D = M + k0 + (size_t)k0 * ld;
        chol_diag_kernel<<<1, 256, 0, st>>>(kb, D, ld, status);
        count_launch();
        const int m = N - k0 - kb;
        if (m <= 0) break;
        double* P = D + kb;
        chol_panel_kernel<<<(m + 127) / 128, 128, 0, st>>>(m, kb, D, ld, P, NP, m);
        count_launch();
        // A22 += P (-P)^T on the lower 64-tiles
        if (const cudaError_t e = gemm_lower_tiles(st, m, kb, P, ld, NP, m, D + kb + (size_t)kb * ld, ld, false))
            return e;
    }
    return cudaGetLastError();
}

cudaError_t bse_jl(cudaStream_t st, int h, double* L, int ld, double* JL, int ldj) {
    bse_jl_kernel<<<grid_of(4LL * h * h), 256, 0, st>>>(h, L, ld, JL, ldj);
    count_launch();
    return cudaGetLastError();
}

// X (N x ncols, ld ldx) <- L^-T X for the lower factor L, by blocks of 64 from
// the bottom: X_I <- L_II^-T X_I, then X_{0:I} -= L_{I, 0:I}^T X_I.
cudaError_t trsm_lower_t(cudaStream_t st, int N, const double* L, int ld, double* X, int ldx, int ncols) {
    if (N <= 0 || ncols <= 0) return cudaSuccess;
    const int nb = (N + CB - 1) / CB;
    for (int b = nb - 1; b >= 0; b--) {
        const int i0 = b * CB, kb = (N - i0 < CB) ? N - i0 : CB;
        trsm_lt_diag_kernel<<<(ncols + 127) / 128, 128, 0, st>>>(kb, L + i0 + (size_t)i0 * ld, ld, X + i0, ldx, ncols);
        count_launch();
        if (i0 > 0) {
            // X[0:i0, :] -= (L[i0:i0+kb, 0:i0])^T X[i0:i0+kb, :]
            if (const cudaError_t e = gemm(st, true, false, i0, ncols, kb, -1.0, L + i0, ld, X + i0, ldx, 1.0, X, ldx))
                return e;
        }
    }
    return cudaGetLastError();
}

cudaError_t bse_psi(cudaStream_t st, int h, int nev, const double* Xr, const double* Xi, int ldx,
                    const double* lambda, double* Pr, double* Pi, int ldp) {
    bse_psi_kernel<<<grid_of((long long)h * nev), 256, 0, st>>>(h, nev, Xr, Xi, ldx, lambda, Pr, Pi, ldp);
    count_launch();
    return cudaGetLastError();
}

}  // namespace sk
