// metrics.cu -- accuracy metrics of a computed skew-symmetric eigendecomposition
// on the device (Algorithm 1 "Ensure": Q^H A Q = diag(i lambda)).  With
// Z = X + iY and a column subset S:
//   residual^2      = ||A X_S + Y_S L_S||_F^2 + ||A Y_S - X_S L_S||_F^2
//   orthogonality^2 = ||X_S^T X + Y_S^T Y - I_S||_F^2 + ||X_S^T Y - Y_S^T X||_F^2
//   ||A||_F^2       = 2 * sum of squares of the strict lower triangle.
// S = all columns gives the full metrics; a sample keeps the cost at
// O(n^2 |S|) for large n.
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace sk {
namespace {

__global__ void gather_cols_kernel(int n, const double* __restrict__ X, const double* __restrict__ Y, int ldz,
                                   const int* __restrict__ cols, int s, const double* __restrict__ lambda,
                                   double* __restrict__ XYs, double* __restrict__ lam_s) {
    // XYs = [X_S | Y_S] (n x 2s, ld n)
    size_t total = (size_t)n * s;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        int c = cols[j];
        XYs[(size_t)j * n + i] = X[(size_t)c * ldz + i];
        XYs[(size_t)(j + s) * n + i] = Y[(size_t)c * ldz + i];
        if (i == 0) lam_s[j] = lambda[c];
    }
}

// sum of squares of R1 = AX_S + Y_S L, R2 = AY_S - X_S L (AXY = A [X_S | Y_S])
__global__ void resid_kernel(int n, int s, const double* __restrict__ AXY, const double* __restrict__ XYs,
                             const double* __restrict__ lam_s, double* __restrict__ acc) {
    __shared__ double red[32];
    double a = 0.0;
    size_t total = (size_t)n * s;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        double l = lam_s[j];
        double r1 = AXY[(size_t)j * n + i] + XYs[(size_t)(j + s) * n + i] * l;
        double r2 = AXY[(size_t)(j + s) * n + i] - XYs[(size_t)j * n + i] * l;
        a = fma(r1, r1, fma(r2, r2, a));
    }
    a = sk_block_sum(a, red);
    if (threadIdx.x == 0) atomicAdd(acc, a);
}

// sum of squares of Gre - I_S and Gim (Gre, Gim: s x nev, ld s)
__global__ void orth_kernel(int s, int nev, const double* __restrict__ Gre, const double* __restrict__ Gim,
                            const int* __restrict__ cols, double* __restrict__ acc) {
    __shared__ double red[32];
    double a = 0.0;
    size_t total = (size_t)s * nev;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int j = (int)(e % s), k = (int)(e / s);
        double re = Gre[(size_t)k * s + j] - (cols[j] == k ? 1.0 : 0.0);
        double im = Gim[(size_t)k * s + j];
        a = fma(re, re, fma(im, im, a));
    }
    a = sk_block_sum(a, red);
    if (threadIdx.x == 0) atomicAdd(acc, a);
}

__global__ void fro_lower_kernel(int n, const double* __restrict__ A, int lda, double* __restrict__ acc) {
    __shared__ double red[32];
    double a = 0.0;
    size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        if (i > j) {
            double v = A[(size_t)j * lda + i];
            a = fma(v, v, a);
        }
    }
    a = sk_block_sum(a, red);
    if (threadIdx.x == 0) atomicAdd(acc, 2.0 * a);
}

__global__ void iota_kernel(int* cols, int s) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < s; j += gridDim.x * blockDim.x) cols[j] = j;
}

__global__ void zero3_kernel(double* p) {
    if (threadIdx.x < 3) p[threadIdx.x] = 0.0;
}

inline int grid_for(size_t total) {
    size_t g = (total + 255) / 256;
    return (int)(g > 4096 ? 4096 : (g == 0 ? 1 : g));
}

struct MetricWs {
    int* cols;
    double *XYs, *lam_s, *AXY, *Gre, *Gim, *acc;
};

MetricWs carve_metric(Carve& cv, int n, int nev, int s) {
    MetricWs w{};
    w.cols = cv.take<int>((size_t)s);
    w.XYs = cv.take<double>((size_t)n * 2 * s);
    w.lam_s = cv.take<double>((size_t)s);
    w.AXY = cv.take<double>((size_t)n * 2 * s);
    w.Gre = cv.take<double>((size_t)s * nev);
    w.Gim = cv.take<double>((size_t)s * nev);
    w.acc = cv.take<double>(4);
    return w;
}

}  // namespace

size_t metrics_ws(int n, int nev, int s) {
    Carve cv(nullptr, ~size_t(0));
    carve_metric(cv, n, nev, s);
    return cv.off + 256;
}

int metrics(cudaStream_t st, int n, const double* A, int lda, int nev, const double* lambda, const double* X,
            const double* Y, int ldz, const int* cols, int s, double* out3, void* ws, size_t ws_bytes) {
    Carve cv(ws, ws_bytes);
    MetricWs w = carve_metric(cv, n, nev, s);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    const int* c = cols;
    if (!c) {
        iota_kernel<<<grid_for(s), 256, 0, st>>>(w.cols, s);
        count_launch();
        c = w.cols;
    }
    zero3_kernel<<<1, 32, 0, st>>>(w.acc);
    gather_cols_kernel<<<grid_for((size_t)n * s), 256, 0, st>>>(n, X, Y, ldz, c, s, lambda, w.XYs, w.lam_s);
    count_launch(2);
    if (skew_symm(st, n, 2 * s, A, lda, w.XYs, n, w.AXY, n) != cudaSuccess) return SKEW_ERR_CUDA;
    resid_kernel<<<grid_for((size_t)n * s), 256, 0, st>>>(n, s, w.AXY, w.XYs, w.lam_s, w.acc);
    count_launch();
    // Gre = X_S^T X + Y_S^T Y, Gim = X_S^T Y - Y_S^T X
    const double* Xs = w.XYs;
    const double* Ys = w.XYs + (size_t)n * s;
    if (gemm(st, true, false, s, nev, n, 1.0, Xs, n, X, ldz, 0.0, w.Gre, s) != cudaSuccess) return SKEW_ERR_CUDA;
    if (gemm(st, true, false, s, nev, n, 1.0, Ys, n, Y, ldz, 1.0, w.Gre, s) != cudaSuccess) return SKEW_ERR_CUDA;
    if (gemm(st, true, false, s, nev, n, 1.0, Xs, n, Y, ldz, 0.0, w.Gim, s) != cudaSuccess) return SKEW_ERR_CUDA;
    if (gemm(st, true, false, s, nev, n, -1.0, Ys, n, X, ldz, 1.0, w.Gim, s) != cudaSuccess) return SKEW_ERR_CUDA;
    orth_kernel<<<grid_for((size_t)s * nev), 256, 0, st>>>(s, nev, w.Gre, w.Gim, c, w.acc + 1);
    fro_lower_kernel<<<grid_for((size_t)n * n), 256, 0, st>>>(n, A, lda, w.acc + 2);
    count_launch(2);
    if (cudaMemcpyAsync(out3, w.acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SKEW_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SKEW_ERR_CUDA;
    for (int i = 0; i < 3; i++) out3[i] = std::sqrt(out3[i]);
    return 0;
}

}  // namespace sk
