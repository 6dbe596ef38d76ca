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
__global__ void __launch_bounds__(QR_THREADS, 1)
panel_qr_kernel(int m, int nb, double* __restrict__ P, int ldp, double* __restrict__ tau,
                double* __restrict__ part, double* __restrict__ rowbuf, unsigned* bar,
                int* status, int rpc, unsigned spin_cap) {
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

    const int ncol = min(nb, m);  // columns with a row on the diagonal
    for (int i = 0; i < ncol; i++) {
        const int buf = i & 1;
        // ---- phase A: partial sums over owned rows with global index > i;
        // four threads per column (rows q, q+4, ..), two shuffle levels (the
        // FP64 pipe, not the rows, bounds this loop)
        double* pp = part + ((size_t)buf * G + g) * (nb + 1);
        for (int cb = i; cb < nb; cb += QR_THREADS / 4) {  // uniform trip count: every lane shuffles
            const int c = cb + (t >> 2), q = t & 3;
            const int rlo = max(0, i + 1 - r0);  // owned rows with global index > i
            double a0 = 0.0, a1 = 0.0;
            int r = (c < nb) ? rlo + ((q - rlo) & 3) : rows;
            for (; r + 4 < rows; r += 8) {
                a0 = fma(S[(size_t)i * rpc + r], S[(size_t)c * rpc + r], a0);
                a1 = fma(S[(size_t)i * rpc + r + 4], S[(size_t)c * rpc + r + 4], a1);
            }
            if (r < rows) a0 = fma(S[(size_t)i * rpc + r], S[(size_t)c * rpc + r], a0);
            double acc = a0 + a1;
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (q == 0 && c < nb) pp[c] = acc;
        }
        if (r0 <= i && i < r0 + rows) {  // owner of row i publishes it
            for (int c = i + t; c < nb; c += QR_THREADS)
                rowbuf[buf * nb + c] = S[(size_t)c * rpc + (i - r0)];
        }
        if (!sk_grid_barrier(bar, epoch, status, spin_cap)) return;
        // row i's entries: loaded now, in flight with the partials below
        const double x0_pre = (t == 0) ? __ldcg(rowbuf + buf * nb + i) : 0.0;
        const double rb_pre = (i + 1 + t < nb) ? __ldcg(rowbuf + buf * nb + i + 1 + t) : 0.0;
        // ---- phase B: reduce partials, four threads per column over CTAs
        // q, q+4, .. (a fixed order: identical in all CTAs)
        for (int cb = i; cb < nb; cb += QR_THREADS / 4) {
            const int c = cb + (t >> 2), q = t & 3;
            double a0 = 0.0, a1 = 0.0;
            int h = (c < nb) ? q : G;
            for (; h + 4 < G; h += 8) {
                a0 += __ldcg(part + ((size_t)buf * G + h) * (nb + 1) + c);
                a1 += __ldcg(part + ((size_t)buf * G + h + 4) * (nb + 1) + c);
            }
            if (h < G) a0 += __ldcg(part + ((size_t)buf * G + h) * (nb + 1) + c);
            double acc = a0 + a1;
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (q == 0 && c < nb) ws[c] = acc;  // ws[i] = ||x_tail||^2, ws[c>i] = x_tail . P_tail[:, c]
        }
        __syncthreads();
        if (t == 0) {
            double x0 = x0_pre;
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
            ws[c] = ((c == i + 1 + t) ? rb_pre : __ldcg(rowbuf + buf * nb + c)) + sc * ws[c];
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
            // row r (from t mod rg) x columns i+1+t/rg, step QR_THREADS/rg
            const int rg = (rows <= QR_THREADS / 2) ? QR_THREADS / 2 : QR_THREADS;
            for (int r = t % rg; r < rows; r += rg) {
                const int gr = r0 + r;
                if (gr < i) continue;
                const double f = (gr > i) ? tu * vs[r] : tu;
                for (int c = i + 1 + t / rg; c < nb; c += QR_THREADS / rg) S[(size_t)c * rpc + r] -= f * ws[c];
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
// T of the compact WY form (Eq. 7): T(i, i) = tau_i and column i above the
// diagonal T(0:i, i) = -tau_i T(0:i, 0:i) G(0:i, i), G = V^T V, column by
// column.  Four threads per row (k = row + q, row + q + 4, ..) and two
// shuffle levels: on GB300 every FP64 warp instruction costs 16 SM cycles,
// so the loops stop at each row's own length.  TFL = nb + 1 pads the rows.
constexpr int TF_THREADS = 256;
__global__ void __launch_bounds__(TF_THREADS) tfactor_kernel(int nb, const double* __restrict__ tau,
                                                            const double* __restrict__ Gm, double* __restrict__ T) {
    extern __shared__ double sh[];
    const int ld = nb + 1;
    const bool gsm = nb <= 64;   // G staged in shared memory (else read from L2)
    double* Ts = sh;             // nb x nb, ld nb + 1
    double* Gs = sh + nb * ld;   // nb x nb, ld nb + 1
    const int t = threadIdx.x;
    for (int e = t; e < nb * nb; e += blockDim.x) {
        const int r = e % nb, c = e / nb;
        Ts[c * ld + r] = 0.0;
        if (gsm) Gs[c * ld + r] = Gm[(size_t)c * nb + r];
    }
    if (t == 0 && nb > 0) Ts[0] = tau[0];
    __syncthreads();
    for (int i = 1; i < nb; i++) {
        const double ti = tau[i];
        const double* gi = gsm ? Gs + i * ld : Gm + (size_t)i * nb;  // column i of G
        // rows 0 .. i-1; warps with no such row skip the step (uniform per warp)
        for (int rb = 0; rb < i; rb += TF_THREADS / 4) {
            const int row = rb + (t >> 2), q = t & 3;
            if ((rb + ((t & ~31) >> 2)) >= i) continue;  // first row of this warp is past the column
            double a0 = 0.0, a1 = 0.0;
            int k = row + q;
            for (; k + 4 < i; k += 8) {
                a0 = fma(Ts[k * ld + row], gi[k], a0);
                a1 = fma(Ts[(k + 4) * ld + row], gi[k + 4], a1);
            }
            if (k < i) a0 = fma(Ts[k * ld + row], gi[k], a0);
            double acc = a0 + a1;
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (q == 0 && row < i) Ts[i * ld + row] = -ti * acc;
        }
        if (t == 0) Ts[i * ld + i] = ti;
        __syncthreads();
    }
    for (int e = t; e < nb * nb; e += blockDim.x) {
        const int r = e % nb, c = e / nb;
        T[(size_t)c * nb + r] = Ts[c * ld + r];
    }
}
size_t tfactor_smem(int nb) { return sizeof(double) * (nb <= 64 ? 2 : 1) * (size_t)nb * (nb + 1); }

// From Q = P^T V and the T factor: C1 = V^T P T = Q^T T, C2 = T^T C1 and the
// right factor Z = [-C2 / 2; T] (2 nb x nb, ld 2 nb) of W = [V P] Z = P T -
// V C2 / 2 (Eq. 9).  One block per column j, one thread per row i.
__global__ void wz_kernel(int nb, const double* __restrict__ Q, const double* __restrict__ T,
                          double* __restrict__ Z) {
    __shared__ double c1[128];
    const int j = blockIdx.x, i = threadIdx.x;
    if (i < nb) {
        // C1(i, j) = sum_{k <= j} Q(k, i) T(k, j)   (T upper triangular)
        double a0 = 0.0, a1 = 0.0;
        int k = 0;
        for (; k + 1 <= j; k += 2) {
            a0 = fma(Q[(size_t)i * nb + k], T[(size_t)j * nb + k], a0);
            a1 = fma(Q[(size_t)i * nb + k + 1], T[(size_t)j * nb + k + 1], a1);
        }
        if (k <= j) a0 = fma(Q[(size_t)i * nb + k], T[(size_t)j * nb + k], a0);
        c1[i] = a0 + a1;
    }
    __syncthreads();
    if (i < nb) {
        // C2(i, j) = sum_{k <= i} T(k, i) C1(k, j)
        double a0 = 0.0, a1 = 0.0;
        int k = 0;
        for (; k + 1 <= i; k += 2) {
            a0 = fma(T[(size_t)i * nb + k], c1[k], a0);
            a1 = fma(T[(size_t)i * nb + k + 1], c1[k + 1], a1);
        }
        if (k <= i) a0 = fma(T[(size_t)i * nb + k], c1[k], a0);
        Z[(size_t)j * 2 * nb + i] = -0.5 * (a0 + a1);
        Z[(size_t)j * 2 * nb + nb + i] = T[(size_t)j * nb + i];
    }
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

// Split-K ranges of the K = m products of the tensor-core form
constexpr int KS_MAX = 256;
// Panels per lazy trailing update in the tensor-core form
constexpr int LAZY_G = 4;

struct ReduceWs {
    double *V, *Pm, *Y, *X2, *Y2, *G, *C1, *C2, *tau, *part, *rowbuf;
    unsigned* bar;
    unsigned spin_cap;  // polls of the panel QR's grid barrier before it gives up
    // tensor-core form: Z = [-C2/2; T], split-K partials of the main and side
    // streams, digit slices of V, P, [V P] and Z
    double *Z, *part_m, *part_s, *part_p;
    size_t part_m_n, part_s_n, part_p_n;  // capacities (doubles)
    // lazy trailing update: [V_q W_q] and [W_q -V_q] of the group's panels
    // (global row index, 2b columns per panel), Y2acc^T V, and a workspace for
    // the small products of the group (the group's A22 split holds the other)
    double *X2acc, *Y2acc, *Cc;
    void* gws2;
    size_t gsz2;
    void *oz_v, *oz_p, *oz_vp, *oz_z;
    size_t oz_vb, oz_vpb, oz_zb;
};

int qr_rows_per_cta(int m, int nb, int maxG) {
    int rpc = (m + maxG - 1) / maxG;
    if (rpc < nb) rpc = nb;  // rows 0..nb-1 (the R block) live in CTA 0
    return rpc;
}

size_t qr_smem_bytes(int rpc, int nb) { return sizeof(double) * ((size_t)rpc * nb + rpc + nb); }

ReduceWs carve_reduce(Carve& cv, int n, int b, bool f64acc) {
    ReduceWs w{};
    size_t mb = (size_t)n * b;
    w.V = cv.take<double>(2 * mb);  // [V P]: P follows V with the same leading dimension n
    w.Pm = w.V + mb;
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
    // split-K partials of the SYMM (splits x tiles <= KS_MAX); in the FP64
    // form also of V^T V and V^T Y
    w.part_p_n = (size_t)KS_MAX * 128 * b;
    w.part_p = cv.take<double>(w.part_p_n);
    if (f64acc) {
        w.Z = cv.take<double>((size_t)2 * b * b);
        // split-K partials: main stream (P^T V, b x b, and Y2^T V, up to
        // 2 b LAZY_G x b), side stream (V^T V)
        w.part_m_n = (size_t)KS_MAX * 2 * b * LAZY_G * b;
        w.part_s_n = (size_t)KS_MAX * b * b;
        w.part_m = cv.take<double>(w.part_m_n);
        w.part_s = cv.take<double>(w.part_s_n);
        w.oz_vb = ozaki_operand_ws(b, n);
        w.oz_v = cv.take<char>(w.oz_vb);
        w.oz_p = cv.take<char>(w.oz_vb);
        w.oz_vpb = ozaki_operand_ws(n, 2 * b);
        w.oz_vp = cv.take<char>(w.oz_vpb);
        w.oz_zb = ozaki_operand_ws(b, 2 * b);
        w.oz_z = cv.take<char>(w.oz_zb);
        w.X2acc = cv.take<double>((size_t)n * 2 * b * LAZY_G);
        w.Y2acc = cv.take<double>((size_t)n * 2 * b * LAZY_G);
        w.Cc = cv.take<double>((size_t)2 * b * LAZY_G * b);
        const size_t g1 = ozaki_gemm_ws(n, b, 2 * b * LAZY_G), g2 = ozaki_operand_ws(2 * b * LAZY_G, n);
        w.gsz2 = g1 > g2 ? g1 : g2;
        w.gws2 = cv.take<char>(w.gsz2);
    }
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
    carve_reduce(cv, n, b, planes == REDUCE_F64ACC);
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

namespace {

// A second stream for the T factor, which needs only V: it runs beside the
// SYMM and is joined before W is formed.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t ev_v = nullptr, ev_t = nullptr;
    int init() {
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SKEW_ERR_CUDA;
        if (cudaEventCreateWithFlags(&ev_v, cudaEventDisableTiming) != cudaSuccess) return SKEW_ERR_CUDA;
        if (cudaEventCreateWithFlags(&ev_t, cudaEventDisableTiming) != cudaSuccess) return SKEW_ERR_CUDA;
        return 0;
    }
    ~SideStream() {
        if (ev_v) cudaEventDestroy(ev_v);
        if (ev_t) cudaEventDestroy(ev_t);
        if (s) cudaStreamDestroy(s);
    }
};

// Cooperative panel QR of panel p (a2): Householder vectors below the
// diagonal block in place, taus into w.tau.
int launch_panel_qr(cudaStream_t st, int n, int b, int p, double* W, int ldw, ReduceWs& w, int* d_status,
                    int max_smem, int sms) {
    const int o = (p + 1) * b, m = n - o;
    double* panel = W + (size_t)p * b * ldw + o;
    int rpc = qr_rows_per_cta(m, b, sms);
    const int G = (m + rpc - 1) / rpc;
    const size_t smem = qr_smem_bytes(rpc, b);
    if ((int)smem > max_smem - 1024 || G > 1024) return SKEW_ERR_UNSUPPORTED;
    cudaFuncSetAttribute(panel_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, panel_qr_kernel, QR_THREADS, smem);
    if (occ * sms < G) return SKEW_ERR_LAUNCH;
    if (cudaMemsetAsync(w.bar, 0, sizeof(unsigned), st) != cudaSuccess) return SKEW_ERR_CUDA;
    int ldp = ldw, nbv = b, mm = m;
    double* taup = w.tau;
    unsigned cap = w.spin_cap;
    void* args[] = {&mm, &nbv, &panel, &ldp, &taup, &w.part, &w.rowbuf, &w.bar, &d_status, &rpc, &cap};
    KtScope kt(st, KT_PANEL_QR);
    if (cudaLaunchCooperativeKernel((void*)panel_qr_kernel, dim3(G), dim3(QR_THREADS), args, smem, st) != cudaSuccess)
        return SKEW_ERR_LAUNCH;
    count_launch();
    return 0;
}

// Band reduction in the tensor-core form with a lazy trailing update.  The
// panels go in groups of LAZY_G.  At a group's start the trailing matrix
// A22_0 = W[o0:, o0:] is up to date and is split into digit slices once;
// panel p = p0 + i of the group then works with
//   A22_p = A22_0[d:, d:] + sum_{q < p in the group} X2_q Y2_q^T  (d = o_p - o0),
// X2_q = [V_q W_q], Y2_q = [W_q -V_q] (Eq. 10): its SYMM reads a view of the
// group split and adds X2 (Y2^T V) (Eq. 8 with the pending terms), its own
// columns get the pending terms just before its QR, and at the group's end one
// rank-2 b LAZY_G product brings the rest of the trailing matrix up to date
// (K = 512 instead of four K = 128 updates: the product's FP64 epilogue and
// the split pass, the costs of a short-K update, run once per group).
// Per panel, as tensor-core products (FP64-accurate digit slices):
//   side stream: G = V^T V (split K), T from G (Eq. 7);
//   main stream: P = A22_p V, Q = P^T V (split K), C1 = V^T P T = Q^T T,
//   C2 = T^T C1 and W = P T - V C2 / 2 = [V P] [-C2/2; T] (Eq. 9) with K = 2b.
int band_reduce_f64acc(cudaStream_t st, int n, double* W, int ldw, int b, double* Tfac, ReduceWs& w, void* gws,
                       size_t gsz, int* status, int slices, SideStream& side, int max_smem, int sms) {
    const int P = num_panels(n, b);
    const long long ldx = n;
    for (int p0 = 0; p0 < P; p0 += LAZY_G) {
        const int p1 = (p0 + LAZY_G < P) ? p0 + LAZY_G : P;
        const int o0 = (p0 + 1) * b, m0 = n - o0;
        OzOperand oa{};  // the group's A22 split (skew, rows and K = m0)
        int rc = ozaki_split(st, m0, m0, W + (size_t)o0 * ldw + o0, 0, ldw, 1.0, 1, gws, gsz, &oa);
        if (rc) return rc;
        for (int p = p0; p < p1; p++) {
            const int i = p - p0, o = (p + 1) * b, m = n - o, d = o - o0, pb = p * b;
            double* panel = W + (size_t)pb * ldw + o;
            double* Tp = Tfac + (size_t)p * b * b;
            if (i > 0) {
                // the pending terms of the panel's own columns (rows from its diagonal block)
                rc = ozaki_gemm(st, n - pb, b, 2 * b * i, 1.0, w.X2acc + pb, 1, ldx, 1.0, w.Y2acc + pb, 1, ldx, 1.0,
                                1.0, W + (size_t)pb * ldw + pb, ldw, w.gws2, w.gsz2, status, 0, 8, 0);
                if (rc) return rc;
            }
            rc = launch_panel_qr(st, n, b, p, W, ldw, w, status, max_smem, sms);
            if (rc) return rc;
            {
                KtScope kt(st, KT_GEMM_F64);
                panel_v_kernel<<<grid_for((size_t)m * b), 256, 0, st>>>(m, b, panel, ldw, w.V, n);
                count_launch();
            }
            // rows of these operands are the b columns of V (of P), K = m
            OzOperand ov{}, op{}, ovp{}, oz{};
            rc = ozaki_split(st, b, m, w.V, n, 1, 1.0, 0, w.oz_v, w.oz_vb, &ov);
            if (rc) return rc;
            const int nch = (m + 63) / 64;
            int ks = (nch + 1) / 2;  // two 64-wide K chunks per CTA at least
            if (ks > sms) ks = sms;
            if (ks > KS_MAX) ks = KS_MAX;
            if (ks < 1) ks = 1;
            if (cudaEventRecord(side.ev_v, st) != cudaSuccess || cudaStreamWaitEvent(side.s, side.ev_v, 0) != cudaSuccess)
                return SKEW_ERR_CUDA;
            rc = ozaki_gemm_pre(side.s, ov, ov, 1.0, 0.0, w.G, b, status, 8, 0, ks, w.part_s, w.part_s_n);
            if (rc) return rc;
            {
                KtScope kt(side.s, KT_GEMM_F64);
                tfactor_kernel<<<1, TF_THREADS, tfactor_smem(b), side.s>>>(b, w.tau, w.G, Tp);
                count_launch();
            }
            if (cudaEventRecord(side.ev_t, side.s) != cudaSuccess) return SKEW_ERR_CUDA;
            // a3: P = A22_0[d:, d:] V (a view of the group split; N = b is a
            // single column of tiles, so K is split to fill the SMs) ...
            {
                const int tiles = (m + 127) / 128;
                int kp = sms / tiles;
                if (kp * tiles > KS_MAX) kp = KS_MAX / tiles;
                if (kp > (nch + 1) / 2) kp = (nch + 1) / 2;
                if (kp < 1) kp = 1;
                rc = ozaki_gemm_pre(st, oz_view(oa, d, d, m, m), ov, 1.0, 0.0, w.Pm, n, status, slices, 0, kp,
                                    w.part_p, w.part_p_n);
                if (rc) return rc;
            }
            if (i > 0) {
                // ... + X2 (Y2^T V) over the group's earlier panels
                const int kq = 2 * b * i;
                OzOperand oy{};
                rc = ozaki_split(st, kq, m, w.Y2acc + o, ldx, 1, 1.0, 0, w.gws2, w.gsz2, &oy);
                if (rc) return rc;
                rc = ozaki_gemm_pre(st, oy, ov, 1.0, 0.0, w.Cc, 2 * b * LAZY_G, status, 8, 0, ks, w.part_m,
                                    w.part_m_n);
                if (rc) return rc;
                rc = ozaki_gemm(st, m, b, kq, 1.0, w.X2acc + o, 1, ldx, 1.0, w.Cc, 2 * b * LAZY_G, 1, 1.0, 1.0, w.Pm, n,
                                w.gws2, w.gsz2, status, 0, 8, 0);
                if (rc) return rc;
            }
            // Q = P^T V
            rc = ozaki_split(st, b, m, w.Pm, n, 1, 1.0, 0, w.oz_p, w.oz_vb, &op);
            if (rc) return rc;
            rc = ozaki_gemm_pre(st, op, ov, 1.0, 0.0, w.C1, b, status, 8, 0, ks, w.part_m, w.part_m_n);
            if (rc) return rc;
            // a4: W = [V P] Z, Z = [-C2/2; T]
            if (cudaStreamWaitEvent(st, side.ev_t, 0) != cudaSuccess) return SKEW_ERR_CUDA;
            {
                KtScope kt(st, KT_GEMM_F64);
                wz_kernel<<<b, b, 0, st>>>(b, w.C1, Tp, w.Z);
                count_launch();
            }
            rc = ozaki_split(st, m, 2 * b, w.V, 1, n, 1.0, 0, w.oz_vp, w.oz_vpb, &ovp);
            if (rc) return rc;
            rc = ozaki_split(st, b, 2 * b, w.Z, 2 * b, 1, 1.0, 0, w.oz_z, w.oz_zb, &oz);
            if (rc) return rc;
            rc = ozaki_gemm_pre(st, ovp, oz, 1.0, 0.0, w.Y, n, status, 8);
            if (rc) return rc;
            {
                // X2_p, Y2_p into the group's accumulators (rows o.. of columns 2 b i ..)
                KtScope kt(st, KT_GEMM_F64);
                concat_kernel<<<grid_for((size_t)m * b), 256, 0, st>>>(m, b, w.V, w.Y, n,
                                                                      w.X2acc + (size_t)2 * b * i * ldx + o,
                                                                      w.Y2acc + (size_t)2 * b * i * ldx + o);
                count_launch();
            }
        }
        // group end: the trailing matrix from the last panel's o (the next
        // group's first panel columns included) takes all the group's terms,
        // tiles on or below the diagonal (the upper triangle of W is never read)
        const int oL = p1 * b, mL = n - oL;
        if (mL > 0) {
            const int rc2 = ozaki_gemm(st, mL, mL, 2 * b * (p1 - p0), 1.0, w.X2acc + oL, 1, ldx, 1.0, w.Y2acc + oL, 1,
                                       ldx, 1.0, 1.0, W + (size_t)oL * ldw + oL, ldw, gws, gsz, status, 0, slices, 1);
            if (rc2) return rc2;
        }
    }
    return 0;
}

}  // namespace

int band_reduce(cudaStream_t st, int n, double* W, int ldw, int b, double* Tfac, void* ws,
                size_t ws_bytes, int* d_status, int planes, int slices, unsigned spin_cap) {
    const bool mixed = planes > 0;
    if (b <= 0 || b % 64 != 0 || b > 128) return SKEW_ERR_UNSUPPORTED;
    const int P = num_panels(n, b);
    if (P == 0) return 0;
    Carve cv(ws, ws_bytes);
    ReduceWs w = carve_reduce(cv, n, b, planes == REDUCE_F64ACC);
    w.spin_cap = spin_cap ? spin_cap : SK_SPIN_CAP;
    const size_t gsz = mixed ? mixed_gemm_ws(n, b, planes) : 0;
    void* gws = mixed ? cv.take<char>(gsz) : nullptr;
    if (!cv.ok) return SKEW_ERR_WORKSPACE;

    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int sms = device_sms();
    if (cudaFuncSetAttribute(tfactor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tfactor_smem(b)) !=
        cudaSuccess)
        return SKEW_ERR_LAUNCH;
    SideStream side;
    if (planes == REDUCE_F64ACC) {
        const int rc = side.init();
        if (rc) return rc;
    }

    if (planes == REDUCE_F64ACC) {
        const int rc = band_reduce_f64acc(st, n, W, ldw, b, Tfac, w, gws, gsz, d_status, slices, side, max_smem, sms);
        if (rc) return rc;
        return cudaGetLastError() == cudaSuccess ? 0 : SKEW_ERR_CUDA;
    }

    for (int p = 0; p < P; p++) {
        const int o = (p + 1) * b, m = n - o;
        double* panel = W + (size_t)p * b * ldw + o;
        double* A22 = W + (size_t)o * ldw + o;
        double* Tp = Tfac + (size_t)p * b * b;
        double* taup = w.tau;
        // ---- a2: panel QR (cooperative)
        if (const int rc0 = launch_panel_qr(st, n, b, p, W, ldw, w, d_status, max_smem, sms)) return rc0;
        {
        // ---- T factor (Eq. 7)
        {
            KtScope kt(st, KT_GEMM_F64);
            panel_v_kernel<<<grid_for((size_t)m * b), 256, 0, st>>>(m, b, panel, ldw, w.V, n);
            count_launch();
            if (gemm(st, true, false, b, b, m, 1.0, w.V, n, w.V, n, 0.0, w.G, b, 0, w.part_p, w.part_p_n) !=
                cudaSuccess)
                return SKEW_ERR_CUDA;
            tfactor_kernel<<<1, TF_THREADS, tfactor_smem(b), st>>>(b, taup, w.G, Tp);
            count_launch();
        }
        // ---- a3: P = A22 V (skew, lower triangle only)
        if (mixed) {
            int rc = split_gemm(st, m, b, m, 1.0, A22, 0, ldw, 1, w.V, n, 1, 0.0, w.Pm, n, 0, gws, gsz, d_status,
                                planes);
            if (rc) return rc;
        } else {
            KtScope kt(st, KT_GEMM_F64);
            if (skew_symm(st, m, b, A22, ldw, w.V, n, w.Pm, n, 0, w.part_p, w.part_p_n) != cudaSuccess)
                return SKEW_ERR_CUDA;
        }
        {
            // ---- a4: Y = P T; C = T^T (V^T Y); W = Y - V C / 2
            KtScope kt(st, KT_GEMM_F64);
            if (gemm(st, false, false, m, b, b, 1.0, w.Pm, n, Tp, b, 0.0, w.Y, n) != cudaSuccess) return SKEW_ERR_CUDA;
            if (gemm(st, true, false, b, b, m, 1.0, w.V, n, w.Y, n, 0.0, w.C1, b, 0, w.part_p, w.part_p_n) !=
                cudaSuccess)
                return SKEW_ERR_CUDA;
            if (gemm(st, true, false, b, b, b, 1.0, Tp, b, w.C1, b, 0.0, w.C2, b) != cudaSuccess) return SKEW_ERR_CUDA;
            if (gemm(st, false, false, m, b, b, -0.5, w.V, n, w.C2, b, 1.0, w.Y, n) != cudaSuccess)
                return SKEW_ERR_CUDA;
            // ---- a5: A22 += [V W][W -V]^T (lower tiles)
            concat_kernel<<<grid_for((size_t)m * b), 256, 0, st>>>(m, b, w.V, w.Y, n, w.X2, w.Y2);
            count_launch();
        }
        }
        if (mixed) {
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
