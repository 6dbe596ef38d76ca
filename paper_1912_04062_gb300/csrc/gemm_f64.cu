// gemm_f64.cu -- FP64 tiled GEMM kernels for the FP64 form of the solver.
//
// On GB300 the FP64 rate is about 1 TFLOP/s for both the SIMT pipe and the
// DMMA (mma.sync f64) path, so these kernels are bound by the FP64 ALU, not by
// memory: a 64 x 64 output tile per 256-thread CTA, 4 x 4 accumulators per
// thread, 16-deep K slices staged through shared memory keep the FP64 pipe
// busy while touching HBM/L2 only once per tile and K slice.
//
// Three shapes are served:
//   * plain C = alpha op(A) op(B) + beta C (split K: partial products in a
//     caller buffer summed in a fixed order, so results do not depend on the
//     order in which CTAs finish; FP64 atomics when no buffer is given);
//   * skew-symmetric A given by its strict lower triangle (Sec. 2.3.2: "symmetry
//     is assumed ... sign changes"): element (i, k) of S is W[i,k] below the
//     diagonal, -W[k,i] above it, 0 on it -- the A V product of Eqs. 8-10;
//   * lower-tile-only output (the skew rank-2k trailing update, Eq. 10 with
//     U1 = -U2): only tiles I >= J of the 64-tile grid are computed.
#include "common.cuh"
#include "internal.h"

namespace sk {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

enum AMode { A_PLAIN_N = 0, A_PLAIN_T = 1, A_SKEW = 2 };

// Load a BM x BK slice of op(A) (rows i0.., cols k0..) into As[k][i].
template <int AM>
__device__ __forceinline__ void load_a(double (*As)[BM + 1], const double* __restrict__ A, int lda,
                                       int M, int K, int i0, int k0) {
    const int t = threadIdx.x;
    if (AM == A_PLAIN_N) {
        // consecutive threads -> consecutive rows i (coalesced)
#pragma unroll
        for (int e = 0; e < (BM * BK) / NT; e++) {
            int idx = t + e * NT;
            int i = idx % BM, k = idx / BM;
            int gi = i0 + i, gk = k0 + k;
            As[k][i] = (gi < M && gk < K) ? A[(size_t)gk * lda + gi] : 0.0;
        }
    } else if (AM == A_PLAIN_T) {
        // op(A)[i,k] = A[k + i*lda]: consecutive threads -> consecutive k
#pragma unroll
        for (int e = 0; e < (BM * BK) / NT; e++) {
            int idx = t + e * NT;
            int k = idx % BK, i = idx / BK;
            int gi = i0 + i, gk = k0 + k;
            As[k][i] = (gi < M && gk < K) ? A[(size_t)gi * lda + gk] : 0.0;
        }
    } else {
        // skew: S[i,k] = W[i,k] (i > k), -W[k,i] (i < k), 0 (i == k)
        const bool all_lower = (i0 > k0 + BK - 1);
        const bool all_upper = (i0 + BM - 1 < k0);
        if (all_lower) {
#pragma unroll
            for (int e = 0; e < (BM * BK) / NT; e++) {
                int idx = t + e * NT;
                int i = idx % BM, k = idx / BM;
                int gi = i0 + i, gk = k0 + k;
                As[k][i] = (gi < M && gk < K) ? A[(size_t)gk * lda + gi] : 0.0;
            }
        } else if (all_upper) {
#pragma unroll
            for (int e = 0; e < (BM * BK) / NT; e++) {
                int idx = t + e * NT;
                int k = idx % BK, i = idx / BK;
                int gi = i0 + i, gk = k0 + k;
                As[k][i] = (gi < M && gk < K) ? -A[(size_t)gi * lda + gk] : 0.0;
            }
        } else {
#pragma unroll
            for (int e = 0; e < (BM * BK) / NT; e++) {
                int idx = t + e * NT;
                int i = idx % BM, k = idx / BM;
                int gi = i0 + i, gk = k0 + k;
                double v = 0.0;
                if (gi < M && gk < K) {
                    if (gi > gk) v = A[(size_t)gk * lda + gi];
                    else if (gi < gk) v = -A[(size_t)gi * lda + gk];
                }
                As[k][i] = v;
            }
        }
    }
}

// Load a BK x BN slice of op(B) (rows k0.., cols j0..) into Bs[k][j].
template <bool TB>
__device__ __forceinline__ void load_b(double (*Bs)[BN + 1], const double* __restrict__ B, int ldb,
                                       int N, int K, int k0, int j0) {
    const int t = threadIdx.x;
    if (!TB) {
        // op(B)[k,j] = B[k + j*ldb]: consecutive threads -> consecutive k
#pragma unroll
        for (int e = 0; e < (BN * BK) / NT; e++) {
            int idx = t + e * NT;
            int k = idx % BK, j = idx / BK;
            int gk = k0 + k, gj = j0 + j;
            Bs[k][j] = (gj < N && gk < K) ? B[(size_t)gj * ldb + gk] : 0.0;
        }
    } else {
        // op(B)[k,j] = B[j + k*ldb]: consecutive threads -> consecutive j
#pragma unroll
        for (int e = 0; e < (BN * BK) / NT; e++) {
            int idx = t + e * NT;
            int j = idx % BN, k = idx / BN;
            int gk = k0 + k, gj = j0 + j;
            Bs[k][j] = (gj < N && gk < K) ? B[(size_t)gk * ldb + gj] : 0.0;
        }
    }
}

// Core tile loop.  Thread (tx, ty) = (t % 16, t / 16) owns rows tx + 16 r and
// columns ty + 16 c (r, c < 4): strided ownership keeps shared-memory reads
// conflict-free and global stores coalesced along rows.
template <int AM, bool TB>
__device__ __forceinline__ void tile_mma(double (&acc)[4][4], const double* A, int lda,
                                         const double* B, int ldb, int M, int N, int K,
                                         int i0, int j0, int kbeg, int kend) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        load_a<AM>(As, A, lda, M, kend, i0, k0);
        load_b<TB>(Bs, B, ldb, N, kend, k0, j0);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; k++) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; r++) a[r] = As[k][tx + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; c++) b[c] = Bs[k][ty + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
    (void)K;
}

template <int AM, bool TB>
__global__ void __launch_bounds__(NT) gemm_kernel(int M, int N, int K, double alpha,
                                                  const double* __restrict__ A, int lda,
                                                  const double* __restrict__ B, int ldb,
                                                  double beta, double* __restrict__ C, int ldc,
                                                  int kchunk, double* __restrict__ part) {
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    double acc[4][4] = {};
    if (kbeg < kend) tile_mma<AM, TB>(acc, A, lda, B, ldb, M, N, K, i0, j0, kbeg, kend);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const bool split = gridDim.z > 1;
    // K range z's partial product, M x N with leading dimension M
    double* Pz = part ? part + (size_t)blockIdx.z * M * N : nullptr;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        int gj = j0 + ty + 16 * c;
        if (gj >= N) continue;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            int gi = i0 + tx + 16 * r;
            if (gi >= M) continue;
            double* p = C + (size_t)gj * ldc + gi;
            double v = alpha * acc[r][c];
            if (Pz) Pz[(size_t)gj * M + gi] = v;
            else if (split) atomicAdd(p, v);
            else *p = (beta == 0.0) ? v : fma(beta, *p, v);
        }
    }
}

// Lower-tile-only C += X Y^T (K = k).  Block b enumerates tiles (I, J),
// I >= J, row-major over the lower triangle of the tile grid.
// zero_diag: the skew rank-2k update (its diagonal is exactly 0); otherwise the
// diagonal is updated like every other entry (symmetric updates)
__global__ void __launch_bounds__(NT) lower_tiles_kernel(int m, int k, const double* __restrict__ X,
                                                         int ldx, const double* __restrict__ Y,
                                                         int ldy, double* __restrict__ C, int ldc, int zero_diag) {
    // invert t = I (I + 1) / 2 + J
    const long long t = blockIdx.x;
    int I = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)(I + 1) * (I + 2) / 2 <= t) I++;
    while ((long long)I * (I + 1) / 2 > t) I--;
    const int J = (int)(t - (long long)I * (I + 1) / 2);
    const int i0 = I * BM, j0 = J * BN;
    double acc[4][4] = {};
    tile_mma<A_PLAIN_N, true>(acc, X, ldx, Y, ldy, m, m, k, i0, j0, 0, k);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        int gj = j0 + ty + 16 * c;
        if (gj >= m) continue;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            int gi = i0 + tx + 16 * r;
            if (gi >= m) continue;
            double* p = C + (size_t)gj * ldc + gi;
            *p = (gi == gj && zero_diag) ? 0.0 : (*p + acc[r][c]);
        }
    }
}

__global__ void scale_kernel(int M, int N, double beta, double* C, int ldc) {
    size_t total = (size_t)M * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        size_t j = e / M, i = e % M;
        double* p = C + j * ldc + i;
        *p = (beta == 0.0) ? 0.0 : beta * *p;
    }
}

// C = beta C + sum of the s partial products, added in order z = 0, 1, ...
__global__ void splitk_sum_kernel(int M, int N, int s, const double* __restrict__ part, double beta,
                                  double* __restrict__ C, int ldc) {
    const size_t MN = (size_t)M * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
        double v = part[e];
        for (int z = 1; z < s; z++) v += part[(size_t)z * MN + e];
        const size_t j = e / M, i = e % M;
        double* p = C + j * ldc + i;
        *p = (beta == 0.0) ? v : fma(beta, *p, v);
    }
}

unsigned sum_blocks(size_t mn) {
    const size_t b = (mn + 255) / 256;
    return (unsigned)(b < 4096 ? b : 4096);
}

int pick_split(int tiles, int K, int requested) {
    if (requested > 0) return requested;
    const int target = 2 * device_sms();
    int s = 1;
    while (tiles * s < target && K / (s * 2) >= 64) s *= 2;
    return s;
}

// K ranges: the requested count, else enough CTAs for two waves while each
// range keeps at least 64 of K; at most part_elems / (M N) when the partial
// products go to a buffer
int pick_split_cap(int tiles, int K, int requested, size_t mn, const double* part, size_t part_elems) {
    int s = pick_split(tiles, K, requested);
    if (part && s > 1) {
        const size_t cap = part_elems / mn;
        if ((size_t)s > cap) s = cap > 1 ? (int)cap : 1;
    }
    return s;
}

}  // namespace

int device_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

cudaError_t gemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, double alpha,
                 const double* A, int lda, const double* B, int ldb, double beta, double* C,
                 int ldc, int splitk, double* part, size_t part_elems) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K <= 0) {
        scale_kernel<<<min(1024, (M * N + 255) / 256 + 1), 256, 0, st>>>(M, N, beta, C, ldc);
        count_launch();
        return cudaGetLastError();
    }
    const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
    const size_t mn = (size_t)M * N;
    int s = pick_split_cap(tm * tn, K, splitk, mn, part, part_elems);
    int kchunk = ((K + s - 1) / s + BK - 1) / BK * BK;
    s = (K + kchunk - 1) / kchunk;
    const bool ordered = part && s > 1;
    if (s > 1 && !ordered) {
        scale_kernel<<<min(4096, (M * N + 255) / 256 + 1), 256, 0, st>>>(M, N, beta, C, ldc);
        count_launch();
    }
    double* pz = ordered ? part : nullptr;
    dim3 grid(tm, tn, s);
    if (!ta && !tb)
        gemm_kernel<A_PLAIN_N, false><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kchunk, pz);
    else if (!ta && tb)
        gemm_kernel<A_PLAIN_N, true><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kchunk, pz);
    else if (ta && !tb)
        gemm_kernel<A_PLAIN_T, false><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kchunk, pz);
    else
        gemm_kernel<A_PLAIN_T, true><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kchunk, pz);
    count_launch();
    if (ordered) {
        splitk_sum_kernel<<<sum_blocks(mn), 256, 0, st>>>(M, N, s, part, beta, C, ldc);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t skew_symm(cudaStream_t st, int m, int nb, const double* W, int ldw, const double* V,
                      int ldv, double* P, int ldp, int splitk, double* part, size_t part_elems) {
    if (m <= 0 || nb <= 0) return cudaSuccess;
    const int tm = (m + BM - 1) / BM, tn = (nb + BN - 1) / BN;
    const size_t mn = (size_t)m * nb;
    int s = pick_split_cap(tm * tn, m, splitk, mn, part, part_elems);
    int kchunk = ((m + s - 1) / s + BK - 1) / BK * BK;
    s = (m + kchunk - 1) / kchunk;
    const bool ordered = part && s > 1;
    if (s > 1 && !ordered) {
        // the K ranges accumulate into P with atomics
        scale_kernel<<<min(4096, (m * nb + 255) / 256 + 1), 256, 0, st>>>(m, nb, 0.0, P, ldp);
        count_launch();
    }
    dim3 grid(tm, tn, s);
    gemm_kernel<A_SKEW, false><<<grid, NT, 0, st>>>(m, nb, m, 1.0, W, ldw, V, ldv, 0.0, P, ldp, kchunk,
                                                    ordered ? part : nullptr);
    count_launch();
    if (ordered) {
        splitk_sum_kernel<<<sum_blocks(mn), 256, 0, st>>>(m, nb, s, part, 0.0, P, ldp);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t gemm_lower_tiles(cudaStream_t st, int m, int k, const double* X, int ldx, const double* Y,
                             int ldy, double* C, int ldc, bool zero_diag) {
    if (m <= 0 || k <= 0) return cudaSuccess;
    const long long T = (m + BM - 1) / BM;
    const long long nt = T * (T + 1) / 2;
    lower_tiles_kernel<<<(unsigned)nt, NT, 0, st>>>(m, k, X, ldx, Y, ldy, C, ldc, zero_diag ? 1 : 0);
    count_launch();
    return cudaGetLastError();
}

}  // namespace sk
