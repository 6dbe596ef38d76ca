// band_reduce.cu -- full-to-band reduction of a skew-symmetric matrix
// (Sec. 2.3.2, "Tridiagonalization in ELPA2", Eqs. 7-10).
//
// For panel p (columns pb..pb+b-1, trailing origin o = (p+1)b, m = n - o):
//   a2  panel QR of W[o:n, pb:pb+b] with Householder reflectors (Sec. 2.1,
//       dlarfg convention) -> V in place, tau, R (the band block);
//       T of the compact WY form Q = I - V T V^T (Eq. 7) from T_ii = tau_i,
//       T[0:i, i] = -tau_i T[0:i,0:i] (V^T V)[0:i, i];
//   a3  P = A22 V using only the lower triangle of A22 (skew SYMM);
//   a4  P <- P T, C = T^T (V^T P), W = P - V C / 2, so that
//       Q^T A22 Q = A22 + V W^T - W V^T (Eqs. 8-10 with U1 = -U2 = W);
//   a5  A22 += [V W] [W -V]^T on the lower 64-tiles (skew rank-2k update).
// The panel QR is one cooperative launch: every CTA keeps its slab of panel
// rows in shared memory for all b columns and the CTAs meet at one capped grid
// barrier per column, so the panel is read from HBM once.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sk {
namespace {

constexpr int QR_THREADS = 256;

// Per-column partial sums live in part[(buf * G + g) * (nb + 1) + c].
__global__ void __launch_bounds__(QR_THREADS)
panel_qr_kernel(int m, int nb, double* __restrict__ P, int ldp, double* __restrict__ tau,
                double* __restrict__ part, double* __restrict__ rowbuf, unsigned* bar,
                int* status, int rpc) {
    extern __shared__ double smem[];
    double* S = smem;                      // rpc x nb, column-major (ld rpc)
    double* vs = S + (size_t)rpc * nb;     // rpc (scaled column i)
    double* ws = vs + rpc;                 // nb  (w_c = v^T P[:, c])
    __shared__ double s_tau, s_scale, s_beta;

    const int G = gridDim.x, g = blockIdx.x, t = threadIdx.x;
    const int r0 = g * rpc;
    const int rows = max(0, min(rpc, m - r0));
    unsigned epoch = 0;

    for (int e = t; e < rpc * nb; e += QR_THREADS) {
        int r = e % rpc, c = e / rpc;
        S[e] = (r < rows) ? P[(size_t)c * ldp + r0 + r] : 0.0;
    }
    __syncthreads();

    const int lane = t & 31, warp = t >> 5, nwarp = QR_THREADS / 32;
    const int ncol = min(nb, m);  // columns with a row on the diagonal
    for (int i = 0; i < ncol; i++) {
        const int buf = i & 1;
        // ---- phase A: partial sums over owned rows with global index > i
        double* pp = part + ((size_t)buf * G + g) * (nb + 1);
        for (int c = i + warp; c < nb; c += nwarp) {
            double acc = 0.0;
            for (int r = lane; r < rows; r += 32) {
                if (r0 + r > i) acc = fma(S[(size_t)i * rpc + r], S[(size_t)c * rpc + r], acc);
            }
            acc = sk_warp_sum(acc);
            if (lane == 0) pp[c] = acc;
        }
        if (r0 <= i && i < r0 + rows) {  // owner of row i publishes it
            for (int c = i + t; c < nb; c += QR_THREADS)
                rowbuf[buf * nb + c] = S[(size_t)c * rpc + (i - r0)];
        }
        if (!sk_grid_barrier(bar, epoch, status)) return;
        // ---- phase B: reduce partials (fixed order -> identical in all CTAs)
        for (int c = i + t; c < nb; c += QR_THREADS) {
            double acc = 0.0;
            for (int h = 0; h < G; h++)
                acc += __ldcg(part + ((size_t)buf * G + h) * (nb + 1) + c);
            ws[c] = acc;  // ws[i] = ||x_tail||^2, ws[c>i] = x_tail . P_tail[:, c]
        }
        __syncthreads();
        if (t == 0) {
            double x0 = __ldcg(rowbuf + buf * nb + i);
            double tail2 = ws[i];
            double tu, sc, be;
            if (tail2 == 0.0) {
                tu = 0.0; sc = 0.0; be = x0;
            } else {
                double rr = sqrt(x0 * x0 + tail2);
                be = (x0 >= 0.0) ? -rr : rr;
                tu = (be - x0) / be;
                sc = 1.0 / (x0 - be);
            }
            s_tau = tu; s_scale = sc; s_beta = be;
            if (g == 0) tau[i] = tu;
        }
        __syncthreads();
        const double tu = s_tau, sc = s_scale;
        // w_c = v^T P[:, c] = P[i, c] + scale * (x_tail . P_tail[:, c]), c > i
        for (int c = i + 1 + t; c < nb; c += QR_THREADS)
            ws[c] = __ldcg(rowbuf + buf * nb + c) + sc * ws[c];
        for (int r = t; r < rows; r += QR_THREADS) {
            int gr = r0 + r;
            double v = 0.0;
            if (gr > i) {
                v = S[(size_t)i * rpc + r] * sc;
                S[(size_t)i * rpc + r] = v;
            }
            vs[r] = v;
        }
        __syncthreads();
        if (tu != 0.0) {
            const int nc = nb - i - 1;
            for (int e = t; e < rows * nc; e += QR_THREADS) {
                int r = e % rows, c = i + 1 + e / rows;
                int gr = r0 + r;
                if (gr > i) S[(size_t)c * rpc + r] -= tu * vs[r] * ws[c];
                else if (gr == i) S[(size_t)c * rpc + r] -= tu * ws[c];
            }
        }
        if (r0 <= i && i < r0 + rows && t == 0) S[(size_t)i * rpc + (i - r0)] = s_beta;
        __syncthreads();
    }
    for (int i = ncol; i < nb; i++)
        if (g == 0 && t == 0) tau[i] = 0.0;
    for (int e = t; e < rows * nb; e += QR_THREADS) {
        int r = e % rows, c = e / rows;
        P[(size_t)c * ldp + r0 + r] = S[(size_t)c * rpc + r];
    }
}

// Explicit V (m x nb): V[r, c] = 1 (r == c), stored (r > c), 0 (r < c).
__global__ void panel_v_kernel(int m, int nb, const double* __restrict__ P, int ldp,
                               double* __restrict__ V, int ldv) {
    size_t total = (size_t)m * nb;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(e % m), c = (int)(e / m);
        double v = (r > c) ? P[(size_t)c * ldp + r] : (r == c ? 1.0 : 0.0);
        V[(size_t)c * ldv + r] = v;
    }
}

// T (nb x nb upper, column-major) from tau and the Gram matrix G = V^T V:
// T_ii = tau_i, T[0:i, i] = -tau_i T[0:i, 0:i] G[0:i, i]   (Eq. 7, forward).
__global__ void tfactor_kernel(int nb, const double* __restrict__ tau,
                               const double* __restrict__ Gm, double* __restrict__ T) {
    extern __shared__ double sh[];
    double* Ts = sh;              // nb x nb
    double* col = sh + nb * nb;   // nb
    const int t = threadIdx.x;
    for (int e = t; e < nb * nb; e += blockDim.x) Ts[e] = 0.0;
    __syncthreads();
    for (int i = 0; i < nb; i++) {
        const double ti = tau[i];
        if (t < i) {
            double acc = 0.0;
            for (int k = t; k < i; k++) acc = fma(Ts[k * nb + t], Gm[(size_t)i * nb + k], acc);
            col[t] = -ti * acc;
        }
        __syncthreads();
        if (t < i) Ts[i * nb + t] = col[t];
        if (t == 0) Ts[i * nb + i] = ti;
        __syncthreads();
    }
    for (int e = t; e < nb * nb; e += blockDim.x) T[e] = Ts[e];
}

// [V W] and [W -V] side by side for the rank-2k update (K = 2 nb).
__global__ void concat_kernel(int m, int nb, const double* __restrict__ V, const double* __restrict__ Wm,
                              int ld, double* __restrict__ X, double* __restrict__ Y) {
    size_t total = (size_t)m * nb;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(e % m), c = (int)(e / m);
        double v = V[(size_t)c * ld + r], w = Wm[(size_t)c * ld + r];
        X[(size_t)c * ld + r] = v;
        X[(size_t)(c + nb) * ld + r] = w;
        Y[(size_t)c * ld + r] = w;
        Y[(size_t)(c + nb) * ld + r] = -v;
    }
}

// Band storage AB[d + c*ldab] = band(c+d, c) for d <= b, 0 for b < d <= 2b.
__global__ void band_pack_kernel(int n, int b, const double* __restrict__ W, int ldw,
                                 double* __restrict__ AB, int ldab, int P) {
    size_t total = (size_t)n * (2 * b + 1);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int d = (int)(e % (2 * b + 1)), c = (int)(e / (2 * b + 1));
        int r = c + d;
        double v = 0.0;
        if (d >= 1 && d <= b && r < n) {
            int p = c / b;                 // column block
            int blk_end = (p + 1) * b;     // first row below the diagonal block
            if (r < blk_end || p >= P) {
                v = W[(size_t)c * ldw + r];   // inside the diagonal block (or tail)
            } else {
                // R block of panel p: keep its upper triangle (row' <= col')
                if (r - blk_end <= c - p * b) v = W[(size_t)c * ldw + r];
            }
        }
        AB[(size_t)c * ldab + d] = v;
    }
}

inline int grid_for(size_t total) {
    size_t g = (total + 255) / 256;
    return (int)(g > 8192 ? 8192 : (g == 0 ? 1 : g));
}

struct ReduceWs {
    double *V, *Pm, *Y, *X2, *Y2, *G, *C1, *C2, *tau, *part, *rowbuf;
    unsigned* bar;
};

int qr_rows_per_cta(int m, int nb, int maxG) {
    int rpc = (m + maxG - 1) / maxG;
    if (rpc < nb) rpc = nb;  // rows 0..nb-1 (the R block) live in CTA 0
    return rpc;
}

size_t qr_smem_bytes(int rpc, int nb) { return sizeof(double) * ((size_t)rpc * nb + rpc + nb); }

ReduceWs carve_reduce(Carve& cv, int n, int b) {
    ReduceWs w{};
    size_t mb = (size_t)n * b;
    w.V = cv.take<double>(mb);
    w.Pm = cv.take<double>(mb);
    w.Y = cv.take<double>(mb);
    w.X2 = cv.take<double>(2 * mb);
    w.Y2 = cv.take<double>(2 * mb);
    w.G = cv.take<double>((size_t)b * b);
    w.C1 = cv.take<double>((size_t)b * b);
    w.C2 = cv.take<double>((size_t)b * b);
    w.tau = cv.take<double>((size_t)b);
    w.part = cv.take<double>((size_t)2 * 1024 * (b + 1));
    w.rowbuf = cv.take<double>((size_t)2 * b);
    w.bar = cv.take<unsigned>(64);
    return w;
}

}  // namespace

int num_panels(int n, int b) { return (n - 2 >= b) ? (n - 2) / b : 0; }

size_t mixed_gemm_ws(int n, int b, int planes) {
    size_t g1, g2;
    if (planes == REDUCE_F64ACC) {
        g1 = ozaki_gemm_ws(n, b, n);
        g2 = ozaki_gemm_ws(n, n, 2 * b);
    } else {
        g1 = split_gemm_ws(n, b, n, planes);
        g2 = split_gemm_ws(n, n, 2 * b, planes);
    }
    return g1 > g2 ? g1 : g2;
}

size_t band_reduce_ws(int n, int b, int planes) {
    Carve cv(nullptr, ~size_t(0));
    carve_reduce(cv, n, b);
    if (planes) cv.take<char>(mixed_gemm_ws(n, b, planes));
    return cv.off + 256;
}

cudaError_t panel_v(cudaStream_t st, int n, int b, int p, const double* W, int ldw, double* V, int ldv) {
    const int o = (p + 1) * b, m = n - o;
    if (m <= 0) return cudaSuccess;
    panel_v_kernel<<<grid_for((size_t)m * b), 256, 0, st>>>(m, b, W + (size_t)p * b * ldw + o, ldw, V, ldv);
    count_launch();
    return cudaGetLastError();
}

int band_reduce(cudaStream_t st, int n, double* W, int ldw, int b, double* Tfac, void* ws,
                size_t ws_bytes, int* d_status, int planes, int slices) {
    const bool mixed = planes > 0;
    if (b <= 0 || b % 64 != 0 || b > 128) return SKEW_ERR_UNSUPPORTED;
    const int P = num_panels(n, b);
    if (P == 0) return 0;
    Carve cv(ws, ws_bytes);
    ReduceWs w = carve_reduce(cv, n, b);
    const size_t gsz = mixed ? mixed_gemm_ws(n, b, planes) : 0;
    void* gws = mixed ? cv.take<char>(gsz) : nullptr;
    if (!cv.ok) return SKEW_ERR_WORKSPACE;

    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int sms = device_sms();

    for (int p = 0; p < P; p++) {
        const int o = (p + 1) * b, m = n - o;
        double* panel = W + (size_t)p * b * ldw + o;
        double* A22 = W + (size_t)o * ldw + o;
        double* Tp = Tfac + (size_t)p * b * b;
        double* taup = w.tau;
        // ---- a2: panel QR (cooperative)
        int rpc = qr_rows_per_cta(m, b, sms);
        int G = (m + rpc - 1) / rpc;
        size_t smem = qr_smem_bytes(rpc, b);
        if ((int)smem > max_smem - 1024 || G > 1024) return SKEW_ERR_UNSUPPORTED;
        cudaFuncSetAttribute(panel_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, panel_qr_kernel, QR_THREADS, smem);
        if (occ * sms < G) return SKEW_ERR_LAUNCH;
        if (cudaMemsetAsync(w.bar, 0, sizeof(unsigned), st) != cudaSuccess) return SKEW_ERR_CUDA;
        int ldp = ldw, nbv = b, mm = m;
        void* args[] = {&mm, &nbv, &panel, &ldp, &taup, &w.part, &w.rowbuf, &w.bar, &d_status, &rpc};
        {
            KtScope kt(st, KT_PANEL_QR);
            if (cudaLaunchCooperativeKernel((void*)panel_qr_kernel, dim3(G), dim3(QR_THREADS), args, smem, st) !=
                cudaSuccess)
                return SKEW_ERR_LAUNCH;
        }
        count_launch();
        // ---- T factor (Eq. 7)
        {
            KtScope kt(st, KT_GEMM_F64);
            panel_v_kernel<<<grid_for((size_t)m * b), 256, 0, st>>>(m, b, panel, ldw, w.V, n);
            count_launch();
            if (gemm(st, true, false, b, b, m, 1.0, w.V, n, w.V, n, 0.0, w.G, b) != cudaSuccess) return SKEW_ERR_CUDA;
            tfactor_kernel<<<1, 128, sizeof(double) * (b * b + b), st>>>(b, taup, w.G, Tp);
            count_launch();
        }
        // ---- a3: P = A22 V (skew, lower triangle only)
        if (planes == REDUCE_F64ACC) {
            int rc = ozaki_gemm(st, m, b, m, 1.0, A22, 0, ldw, 1.0, w.V, n, 1, 1.0, 0.0, w.Pm, n, gws, gsz, d_status,
                                1, slices);
            if (rc) return rc;
        } else if (mixed) {
            int rc = split_gemm(st, m, b, m, 1.0, A22, 0, ldw, 1, w.V, n, 1, 0.0, w.Pm, n, 0, gws, gsz, d_status,
                                planes);
            if (rc) return rc;
        } else {
            KtScope kt(st, KT_GEMM_F64);
            if (skew_symm(st, m, b, A22, ldw, w.V, n, w.Pm, n) != cudaSuccess) return SKEW_ERR_CUDA;
        }
        {
            // ---- a4: Y = P T; C = T^T (V^T Y); W = Y - V C / 2
            KtScope kt(st, KT_GEMM_F64);
            if (gemm(st, false, false, m, b, b, 1.0, w.Pm, n, Tp, b, 0.0, w.Y, n) != cudaSuccess) return SKEW_ERR_CUDA;
            if (gemm(st, true, false, b, b, m, 1.0, w.V, n, w.Y, n, 0.0, w.C1, b) != cudaSuccess) return SKEW_ERR_CUDA;
            if (gemm(st, true, false, b, b, b, 1.0, Tp, b, w.C1, b, 0.0, w.C2, b) != cudaSuccess) return SKEW_ERR_CUDA;
            if (gemm(st, false, false, m, b, b, -0.5, w.V, n, w.C2, b, 1.0, w.Y, n) != cudaSuccess)
                return SKEW_ERR_CUDA;
            // ---- a5: A22 += [V W][W -V]^T (lower tiles)
            concat_kernel<<<grid_for((size_t)m * b), 256, 0, st>>>(m, b, w.V, w.Y, n, w.X2, w.Y2);
            count_launch();
        }
        if (planes == REDUCE_F64ACC) {
            // tiles on or below the diagonal (the upper triangle of W is never read)
            int rc = ozaki_gemm(st, m, m, 2 * b, 1.0, w.X2, 1, n, 1.0, w.Y2, 1, n, 1.0, 1.0, A22, ldw, gws, gsz,
                                d_status, 0, slices, 1);
            if (rc) return rc;
        } else if (mixed) {
            int rc = split_gemm(st, m, m, 2 * b, 1.0, w.X2, 1, n, 0, w.Y2, 1, n, 1.0, A22, ldw, 1, gws, gsz, d_status,
                                planes);
            if (rc) return rc;
        } else {
            KtScope kt(st, KT_GEMM_F64);
            if (gemm_lower_tiles(st, m, 2 * b, w.X2, n, w.Y2, n, A22, ldw) != cudaSuccess) return SKEW_ERR_CUDA;
        }
    }
    return cudaGetLastError() == cudaSuccess ? 0 : SKEW_ERR_CUDA;
}

cudaError_t band_pack(cudaStream_t st, int n, int b, const double* W, int ldw, double* AB, int ldab) {
    if (n <= 0) return cudaSuccess;
    band_pack_kernel<<<grid_for((size_t)n * (2 * b + 1)), 256, 0, st>>>(n, b, W, ldw, AB, ldab, num_panels(n, b));
    count_launch();
    return cudaGetLastError();
}

}  // namespace sk
