// backtransform.cu -- eigenvector back transformations (Sec. 2.1, step 3 of
// the two-step form: Q~ = Q_trd Q_diag, then Q = Q_band Q~; Sec. 2.3: applied
// to the real and imaginary parts independently, realising the complex back
// transformation in real arithmetic).
//
// Q_trd (bulge-chase reflectors).  Q_trd = prod over sweeps s (ascending) of
// prod over steps k (ascending) of H_{s,k}; applying it means applying the
// reflectors in reverse generation order.  H_{s,k} acts on rows
// s+1+k b .. s+k b+b.  Grouping ell consecutive sweeps S = [s0, s0+ell) and
// one step k into a block (a parallelogram of rows s0+1+k b .. s0+ell-1+k b+b)
// the order "groups descending; inside a group k ascending; inside a block s
// descending" equals the reverse generation order up to swaps of reflectors
// with disjoint rows (H_{s',k'} and H_{s,k} with s' >= s and k' > k never
// share a row, since s'+1+k'b > s+kb+b, whatever ell is; ell only sets the
// window height ell + b - 1).  Each CTA owns a slab
// of columns and keeps one block's row window in shared memory while it
// applies the block's ell reflectors, so Z crosses HBM once per block instead
// of once per reflector.
//
// Q_band (full-to-band panels, compact WY Q_p = I - V_p T_p V_p^T, Eq. 7):
// for p descending, Z[o:, :] -= V_p (T_p (V_p^T Z[o:, :])) with FP64 GEMMs.
#include "common.cuh"
#include "internal.h"
#include "sm100.cuh"

namespace sk {
namespace {

constexpr int QB = 64;             // band width
constexpr int QELL = 64;           // sweeps per block
constexpr int QH = QELL + QB - 1;  // window height
constexpr int QLD = 132;           // smem leading dimension (= 4 mod 16: conflict-free)
constexpr int QT = 256;

__host__ __device__ inline int qsteps(int n, int b, int s) { return (s <= n - 3) ? 1 + (n - 3 - s) / b : 0; }

// FP32 form.  Thread t: column c = t / 4 of the slab, row phase q = t % 4; it
// keeps window rows 4u + q (u < 32) of its column in registers.  Reflector s
// of a block touches window rows off..off+b-1 with off = s - s0; the loop over
// off is unrolled, so every register index is a compile-time constant, and
// the four threads of a column are lanes of one warp: a reflector costs two
// shuffles and no block barrier.  Consecutive blocks of a group share 63
// window rows: after block k the window's first 64 rows are final for the
// group and stored, the registers shift by 16, and the 64 new rows of block
// k+1 arrive in shared memory by cp.async while block k computes; the next
// block's reflectors and taus (FP32 copies written by the chase, zero taus
// for absent steps) arrive by one bulk copy into the other of two buffers.
constexpr int QS_LD = 68;  // [column][row] staging, = 4 mod 32: conflict-free for the (c, q) pattern

struct QSlideSmem {
    float v[2][QELL * QB];  // reflectors of the current and the next block
    float tau[2][QELL];
    float zin[64 * QS_LD];   // the next block's 64 new window rows
    float zout[64 * QS_LD];  // the block's 64 finished rows
    uint64_t bar[2];
};

SK_DEV void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
SK_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__global__ void __launch_bounds__(256, 2)
qtrd_slide_kernel(int n, const float* __restrict__ V32, const float* __restrict__ tau32, float* __restrict__ Z,
                  int ldz, int ncols, int slab, int* status) {
    extern __shared__ __align__(128) unsigned char qs_raw[];
    QSlideSmem& sm = *reinterpret_cast<QSlideSmem*>(qs_raw);
    const int nsw = n - 2, nsw64 = (nsw + 63) / 64 * 64;
    const int c0 = blockIdx.x * slab;
    const int nc = min(slab, ncols - c0);
    if (nc <= 0) return;
    const int t = threadIdx.x, T = blockDim.x;
    // every lane takes part in the shuffles; lanes past the slab work on zeros
    const int c = t >> 2, q = t & 3;
    const bool own = c < nc;
    float* zc = Z + (size_t)(c0 + (own ? c : 0)) * ldz;
    if (t == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int ngroups = (nsw + QELL - 1) / QELL;
    constexpr uint32_t VBYTES = QELL * QB * sizeof(float), TBYTES = QELL * sizeof(float);
    // reflectors of block (g, k) into buffer buf (one thread)
    auto fetch = [&](int g, int k, int buf) {
        const size_t slot = (size_t)k * nsw64 + (size_t)g * QELL;
        mbar_arrive_expect_tx(&sm.bar[buf], VBYTES + TBYTES);
        bulk_g2s(sm.v[buf], V32 + slot * QB, VBYTES, &sm.bar[buf]);
        bulk_g2s(sm.tau[buf], tau32 + slot, TBYTES, &sm.bar[buf]);
    };
    if (t == 0) fetch(ngroups - 1, 0, 0);
    int blk = 0;  // blocks so far: buffer blk & 1, barrier phase (blk >> 1) & 1
    for (int g = ngroups - 1; g >= 0; g--) {
        const int s0 = g * QELL;
        const int kmax = qsteps(n, QB, s0);
        float zr[32];
        {
            const int top = s0 + 1, H = min(QH, n - top);
#pragma unroll
            for (int u = 0; u < 32; u++) {
                const int r = 4 * u + q;
                zr[u] = (own && r < H) ? zc[top + r] : 0.f;
            }
        }
        for (int k = 0; k < kmax; k++) {
            const int top = s0 + 1 + k * QB;
            const int buf = blk & 1;
            const bool more = k + 1 < kmax;
            // prefetch: the next block's reflectors, and the 64 new rows
            // top + 127 .. top + 190 of block k+1
            if (t == 0) {
                if (more) fetch(g, k + 1, buf ^ 1);
                else if (g > 0) fetch(g - 1, 0, buf ^ 1);
            }
            if (more) {
                for (int e = t; e < 64 * nc; e += T) {
                    const int cc = e >> 6, j = e & 63, row = top + QH + j;
                    float* d = &sm.zin[cc * QS_LD + j];
                    if (row < n) cp_async4(d, Z + (size_t)(c0 + cc) * ldz + row);
                    else *d = 0.f;
                }
            }
            if (!mbar_wait(&sm.bar[buf], (uint32_t)(blk >> 1) & 1u, status)) return;
            const float* vq = sm.v[buf] + q;
            const float* ts = sm.tau[buf];
#pragma unroll
            for (int off = QELL - 1; off >= 0; off--) {
                const float tau = ts[off];
                if (tau == 0.f) continue;
                const float* v = vq + off * QB - off;  // v[4u] = element 4u + q - off of reflector off
                // rows 4u + q with 0 <= 4u + q - off < QB: every phase for u in
                // [U0, U1]; u = U0 - 1 and U1 + 1 depend on q
                const int U0 = (off + 3) / 4, U1 = (off + QB - 4) / 4;
                const bool lo_ok = (U0 >= 1) && (q >= off - 4 * (U0 - 1));
                const bool hi_ok = (U1 + 1 <= 31) && (4 * (U1 + 1) + q - off < QB);
                float a = 0.f, a2 = 0.f;
#pragma unroll
                for (int u = 0; u < 32; u++) {
                    if (u < U0 || u > U1) continue;
                    if (u & 1) a2 = fmaf(v[4 * u], zr[u], a2);
                    else a = fmaf(v[4 * u], zr[u], a);
                }
                if (U0 >= 1 && lo_ok) a = fmaf(v[4 * (U0 - 1)], zr[U0 - 1 < 0 ? 0 : U0 - 1], a);
                if (U1 + 1 <= 31 && hi_ok) a2 = fmaf(v[4 * (U1 + 1)], zr[U1 + 1 > 31 ? 31 : U1 + 1], a2);
                a += a2;
                a += __shfl_xor_sync(0xffffffffu, a, 1);
                a += __shfl_xor_sync(0xffffffffu, a, 2);
                a *= tau;
#pragma unroll
                for (int u = 0; u < 32; u++) {
                    if (u < U0 || u > U1) continue;
                    zr[u] = fmaf(-a, v[4 * u], zr[u]);
                }
                if (U0 >= 1 && lo_ok) zr[U0 - 1 < 0 ? 0 : U0 - 1] = fmaf(-a, v[4 * (U0 - 1)], zr[U0 - 1 < 0 ? 0 : U0 - 1]);
                if (U1 + 1 <= 31 && hi_ok)
                    zr[U1 + 1 > 31 ? 31 : U1 + 1] = fmaf(-a, v[4 * (U1 + 1)], zr[U1 + 1 > 31 ? 31 : U1 + 1]);
            }
            if (more) {
                // rows 0..63 are final for this group: out through shared memory
#pragma unroll
                for (int u = 0; u < 16; u++) sm.zout[c * QS_LD + 4 * u + q] = zr[u];
                cp_async_wait_all();
                __syncthreads();
                for (int e = t; e < 64 * nc; e += T) {
                    const int cc = e >> 6, j = e & 63;
                    Z[(size_t)(c0 + cc) * ldz + top + j] = sm.zout[cc * QS_LD + j];  // top + 63 < n here
                }
                // slide by 64 rows: rows 64..126 move up, 63..126 of the new
                // window come from zin (row 127 is padding)
#pragma unroll
                for (int u = 0; u < 16; u++) zr[u] = zr[u + 16];
                if (q == 3) zr[15] = sm.zin[c * QS_LD];
#pragma unroll
                for (int u = 16; u < 32; u++) {
                    const int j = 4 * u + q - (QH - QB);  // zin row of window row 4u + q
                    zr[u] = (j < 64) ? sm.zin[c * QS_LD + j] : 0.f;
                }
                __syncthreads();
            } else {
                // last block of the group: the whole window is final
                const int H = min(QH, n - top);
                if (own) {
#pragma unroll
                    for (int u = 0; u < 32; u++) {
                        const int r = 4 * u + q;
                        if (r < H) zc[top + r] = zr[u];
                    }
                }
                __syncthreads();
            }
            blk++;
        }
    }
}

// FP64 variant: the window stays in shared memory (ld QLD, conflict-free for
// doubles); thread (c, q) owns rows 4i + q of column c for each reflector.  On
// this part the FP64 pipe is the limit, and the shared-memory form keeps it
// busier than the register-resident one.  The CTA has 4 threads per column
// of its slab (rounded up to whole warps): threads past the slab would spend
// the FP64 pipe on padding.
template <typename T>
__global__ void __launch_bounds__(QT)
qtrd_smem_kernel(int n, const double* __restrict__ Vtrd, const double* __restrict__ tautrd, T* __restrict__ Z,
                 int ldz, int ncols, int slab) {
    extern __shared__ __align__(16) unsigned char qtrd_raw[];
    T* zw = reinterpret_cast<T*>(qtrd_raw);  // QLD x 64
    const int nsw = n - 2;
    const int c0 = blockIdx.x * slab;
    const int nc = min(slab, ncols - c0);
    if (nc <= 0) return;
    const int t = threadIdx.x;
    const int c = t >> 2, q = t & 3;
    const int ngroups = (nsw + QELL - 1) / QELL;
    for (int g = ngroups - 1; g >= 0; g--) {
        const int s0 = g * QELL, s1 = min(nsw, s0 + QELL);
        const int kmax = qsteps(n, QB, s0);
        for (int k = 0; k < kmax; k++) {
            const int top = s0 + 1 + k * QB;
            if (top >= n) break;
            const int H = min(QH, n - top);
            for (int e = t; e < H * nc; e += blockDim.x) {
                int i = e % H, cc = e / H;
                zw[cc * QLD + i] = Z[(size_t)(c0 + cc) * ldz + top + i];
            }
            __syncthreads();
            {
                T* zc = zw + c * QLD;
                for (int s = s1 - 1; s >= s0; s--) {
                    if (k >= qsteps(n, QB, s)) continue;
                    const size_t vi = (size_t)k * nsw + s;
                    const double taud = tautrd[vi];
                    if (taud == 0.0) continue;
                    const T tau = (T)taud;
                    const double* v = Vtrd + vi * QB;
                    const int off = s - s0;
                    const int lim = min(QB, H - off);
                    T vr[QB / 4];
                    T a = 0;
#pragma unroll
                    for (int ii = 0; ii < QB / 4; ii++) {
                        int i = 4 * ii + q;
                        vr[ii] = (i < lim) ? (T)__ldg(v + i) : (T)0;
                        if (i < lim) a = fma(vr[ii], zc[off + i], a);
                    }
                    a += __shfl_xor_sync(0xffffffffu, a, 1);
                    a += __shfl_xor_sync(0xffffffffu, a, 2);
                    a *= tau;
#pragma unroll
                    for (int ii = 0; ii < QB / 4; ii++) {
                        int i = 4 * ii + q;
                        if (i < lim) zc[off + i] = fma(-a, vr[ii], zc[off + i]);
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            for (int e = t; e < H * nc; e += blockDim.x) {
                int i = e % H, cc = e / H;
                Z[(size_t)(c0 + cc) * ldz + top + i] = zw[cc * QLD + i];
            }
            __syncthreads();
        }
    }
}

struct QbandWs {
    double *V, *Y, *Y2;
    double* part;  // split-K partials of V^T Z
    size_t part_n;
};

QbandWs carve_qband(Carve& cv, int n, int b, int k) {
    QbandWs w{};
    w.V = cv.take<double>((size_t)n * b);
    w.Y = cv.take<double>((size_t)b * k);
    w.Y2 = cv.take<double>((size_t)b * k);
    w.part_n = (size_t)b * (4 * (size_t)k > 1024 ? 4 * (size_t)k : 1024);
    w.part = cv.take<double>(w.part_n);
    return w;
}

// Slab width so that the CTA count fills the GPU in whole waves (per CTAs per SM)
int qtrd_slab(int k, int* grid) {
    const int sms = device_sms();
    int per = 1, slab = 64;
    while (true) {
        slab = (k + sms * per - 1) / (sms * per);
        if (slab <= 64) break;
        per++;
    }
    if (slab < 8) slab = (k < 8) ? k : 8;
    *grid = (k + slab - 1) / slab;
    return slab;
}

}  // namespace

cudaError_t apply_qtrd(cudaStream_t st, int n, int b, const double* Vtrd, const double* tautrd, double* Z, int ldz,
                       int k) {
    if (b != QB) return cudaErrorInvalidValue;
    if (n < 3 || k <= 0) return cudaSuccess;
    int grid = 0;
    const int slab = qtrd_slab(k, &grid);
    const size_t smem = sizeof(double) * (size_t)QLD * 64;
    cudaFuncSetAttribute(qtrd_smem_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int threads = (4 * slab + 31) / 32 * 32;
    KtScope kt(st, KT_QTRD);
    qtrd_smem_kernel<double><<<grid, threads, smem, st>>>(n, Vtrd, tautrd, Z, ldz, k, slab);
    count_launch();
    return cudaGetLastError();
}

cudaError_t apply_qtrd_f32(cudaStream_t st, int n, int b, const float* V32, const float* tau32, float* Z, int ldz,
                           int k, int* status) {
    if (b != QB) return cudaErrorInvalidValue;
    if (n < 3 || k <= 0) return cudaSuccess;
    // two CTAs per SM; 4 threads per column of the slab, whole warps
    const int sms = device_sms();
    int slab = (k + 2 * sms - 1) / (2 * sms);
    if (slab > 64) slab = 64;
    if (slab < 8) slab = (k < 8) ? k : 8;
    const int grid = (k + slab - 1) / slab;
    const int threads = (4 * slab + 31) / 32 * 32;
    const size_t smem = sizeof(QSlideSmem);
    cudaFuncSetAttribute(qtrd_slide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    KtScope kt(st, KT_QTRD);
    qtrd_slide_kernel<<<grid, threads, smem, st>>>(n, V32, tau32, Z, ldz, k, slab, status);
    count_launch();
    return cudaGetLastError();
}

size_t qband_ws(int n, int b, int k) {
    Carve cv(nullptr, ~size_t(0));
    carve_qband(cv, n, b, k);
    return cv.off + 256;
}

int apply_qband(cudaStream_t st, int n, int b, const double* W, int ldw, const double* Tfac, double* Z, int ldz,
                int k, void* ws, size_t ws_bytes) {
    const int P = num_panels(n, b);
    if (P == 0 || k <= 0) return 0;
    Carve cv(ws, ws_bytes);
    QbandWs w = carve_qband(cv, n, b, k);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    for (int p = P - 1; p >= 0; p--) {
        const int o = (p + 1) * b, m = n - o;
        const double* Tp = Tfac + (size_t)p * b * b;
        double* Zo = Z + o;
        KtScope kt(st, KT_GEMM_F64);
        if (panel_v(st, n, b, p, W, ldw, w.V, n) != cudaSuccess) return SKEW_ERR_CUDA;
        if (gemm(st, true, false, b, k, m, 1.0, w.V, n, Zo, ldz, 0.0, w.Y, b, 0, w.part, w.part_n) != cudaSuccess)
            return SKEW_ERR_CUDA;
        if (gemm(st, false, false, b, k, b, 1.0, Tp, b, w.Y, b, 0.0, w.Y2, b) != cudaSuccess) return SKEW_ERR_CUDA;
        if (gemm(st, false, false, m, k, b, -1.0, w.V, n, w.Y2, b, 1.0, Zo, ldz) != cudaSuccess) return SKEW_ERR_CUDA;
    }
    return 0;
}

// Mixed form: Q_band with the two contractions on the tensor cores:
// Y^T = Z[o:, :]^T V_p, then Z[o:, :] -= (V_p T_p) Y, V_p T_p in FP64.
// planes: 2 / 3 (BF16x3 / BF16x6 split products, one panel per pass) or
// REDUCE_F64ACC (FP64-accurate digit-slice products, QG panels per pass: the
// product Q_p0 Q_p0+1 ... Q_p0+QG-1 is one compact WY block I - V T V^T with
// V = [V_p0 ... V_p0+QG-1] and T built by the block form of the forward
// recursion of Eq. 7, T_1..j = [[T_1..j-1, -T_1..j-1 (V_1..j-1^T V_j) T_j],
// [0, T_j]], so Z is read and written once per QG panels and the update has
// K = QG b)
constexpr int QG = 8;

static size_t qband_gemm_ws(int n, int b, int k, int planes) {
    size_t g1, g2;
    if (planes == REDUCE_F64ACC) {
        g1 = ozaki_gemm_ws(k, QG * b, n);
        g2 = ozaki_gemm_ws(n, k, QG * b);
    } else {
        g1 = split_gemm_ws(k, b, n, planes);
        g2 = split_gemm_ws(n, k, b, planes);
    }
    return g1 > g2 ? g1 : g2;
}

// Split-K ranges of the group Gram product V^T V
constexpr int QB_KS = 32;

struct QbMixedWs {
    double *V, *VT, *Yt, *Tg, *G, *tmp;
    void* gws;
    size_t gsz;
    // FP64-accurate form: split-K partials, digit slices of V (rows = its
    // columns), of V by rows and of T_g
    double* part;
    size_t part_n;
    void *oz_v, *oz_a, *oz_t;
    size_t oz_vb, oz_ab, oz_tb;
};

static QbMixedWs carve_qband_mixed(Carve& cv, int n, int b, int k, int planes) {
    QbMixedWs q{};
    const bool acc = planes == REDUCE_F64ACC;
    const size_t w = acc ? (size_t)QG * b : (size_t)b;
    q.V = cv.take<double>((size_t)n * w);
    q.VT = cv.take<double>((size_t)n * w);
    q.Yt = cv.take<double>((size_t)k * w);
    q.Tg = cv.take<double>(w * w);
    q.G = cv.take<double>(w * w);
    q.tmp = cv.take<double>(w * w);
    q.gsz = qband_gemm_ws(n, b, k, planes);
    q.gws = cv.take<char>(q.gsz);
    if (acc) {
        q.part_n = (size_t)QB_KS * w * w;
        q.part = cv.take<double>(q.part_n);
        q.oz_vb = ozaki_operand_ws((int)w, n);
        q.oz_v = cv.take<char>(q.oz_vb);
        q.oz_ab = ozaki_operand_ws(n, (int)w);
        q.oz_a = cv.take<char>(q.oz_ab);
        q.oz_tb = ozaki_operand_ws((int)w, (int)w);
        q.oz_t = cv.take<char>(q.oz_tb);
    }
    return q;
}

size_t qband_mixed_ws(int n, int b, int k, int planes) {
    Carve cv(nullptr, ~size_t(0));
    carve_qband_mixed(cv, n, b, k, planes);
    return cv.off + 256;
}

namespace {
// T of a panel group: the diagonal blocks are the panels' own T (b x b each),
// everything else 0 (filled in afterwards).
__global__ void tgroup_init_kernel(int g, int b, const double* __restrict__ Tp, double* __restrict__ Tg) {
    const int gb = g * b;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < gb * gb; e += gridDim.x * blockDim.x) {
        const int r = e % gb, c = e / gb, jr = r / b, jc = c / b;
        Tg[e] = (jr == jc) ? Tp[(size_t)jr * b * b + (r % b) + (size_t)(c % b) * b] : 0.0;
    }
}
}  // namespace

int apply_qband_mixed(cudaStream_t st, int n, int b, const double* W, int ldw, const double* Tfac, double* Z, int ldz,
                      int k, void* ws, size_t ws_bytes, int* status, int planes, int slices) {
    const int P = num_panels(n, b);
    if (P == 0 || k <= 0) return 0;
    const bool acc = planes == REDUCE_F64ACC;
    Carve cv(ws, ws_bytes);
    const QbMixedWs q = carve_qband_mixed(cv, n, b, k, planes);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    double *V = q.V, *VT = q.VT, *Yt = q.Yt, *Tg = q.Tg, *G = q.G, *tmp = q.tmp;
    void* gws = q.gws;
    const size_t gsz = q.gsz;
    if (!acc) {
        for (int p = P - 1; p >= 0; p--) {
            const int o = (p + 1) * b, m = n - o;
            const double* Tp = Tfac + (size_t)p * b * b;
            double* Zo = Z + o;
            {
                KtScope kt(st, KT_GEMM_F64);
                if (panel_v(st, n, b, p, W, ldw, V, n) != cudaSuccess) return SKEW_ERR_CUDA;
                if (gemm(st, false, false, m, b, b, 1.0, V, n, Tp, b, 0.0, VT, n) != cudaSuccess) return SKEW_ERR_CUDA;
            }
            // Yt = Z_o^T V (k x b), then Z_o -= (V T) Yt^T
            int rc = split_gemm(st, k, b, m, 1.0, Zo, ldz, 1, 0, V, n, 1, 0.0, Yt, k, 0, gws, gsz, status, planes);
            if (rc) return rc;
            rc = split_gemm(st, m, k, b, -1.0, VT, 1, n, 0, Yt, 1, k, 1.0, Zo, ldz, 0, gws, gsz, status, planes);
            if (rc) return rc;
        }
        return 0;
    }
    for (int pe = P - 1; pe >= 0; pe -= QG) {
        const int p0 = pe - QG + 1 > 0 ? pe - QG + 1 : 0, g = pe - p0 + 1, gb = g * b;
        const int o = (p0 + 1) * b, m = n - o;
        double* Zo = Z + o;
        {
            KtScope kt(st, KT_GEMM_F64);  // V, T and V T of the group
            // V of the group (m x gb, ld n): panel p0 + j starts at row j b
            if (cudaMemsetAsync(V, 0, sizeof(double) * (size_t)n * gb, st) != cudaSuccess) return SKEW_ERR_CUDA;
            for (int j = 0; j < g; j++)
                if (panel_v(st, n, b, p0 + j, W, ldw, V + (size_t)j * b * n + (size_t)j * b, n) != cudaSuccess)
                    return SKEW_ERR_CUDA;
            // T of the group
            tgroup_init_kernel<<<(gb * gb + 255) / 256, 256, 0, st>>>(g, b, Tfac + (size_t)p0 * b * b, Tg);
            count_launch();
        }
        // digit slices of V with its gb columns as rows (K = m): the Gram
        // product and Yt below
        OzOperand ov{}, oa{}, ot{}, oz{};
        int rc = ozaki_split(st, gb, m, V, n, 1, 1.0, 0, q.oz_v, q.oz_vb, &ov);
        if (rc) return rc;
        if (g > 1) {
            // G = V^T V on the tensor cores (split K: a few output tiles, K = m)
            int ks = ((m + 63) / 64 + 1) / 2;
            if (ks > QB_KS) ks = QB_KS;
            rc = ozaki_gemm_pre(st, ov, ov, 1.0, 0.0, G, gb, status, 8, 0, ks, q.part, (size_t)QB_KS * gb * gb);
            if (rc) return rc;
            KtScope kt(st, KT_GEMM_F64);
            for (int j = 1; j < g; j++) {
                const int jb = j * b;
                const double* Tj = Tfac + (size_t)(p0 + j) * b * b;
                // tmp = (V_1..j-1^T V_j) T_j, then T[0:jb, jb:jb+b] = -T[0:jb, 0:jb] tmp
                // (split K over 16-deep slices: these products have few output tiles)
                if (gemm(st, false, false, jb, b, b, 1.0, G + (size_t)jb * gb, gb, Tj, b, 0.0, tmp, gb, b / 16,
                         q.part, q.part_n) != cudaSuccess)
                    return SKEW_ERR_CUDA;
                if (gemm(st, false, false, jb, b, jb, -1.0, Tg, gb, tmp, gb, 0.0, Tg + (size_t)jb * gb, gb,
                         jb / 16, q.part, q.part_n) != cudaSuccess)
                    return SKEW_ERR_CUDA;
            }
        }
        // VT = V T_g (m x gb, K = gb)
        rc = ozaki_split(st, m, gb, V, 1, n, 1.0, 0, q.oz_a, q.oz_ab, &oa);
        if (rc) return rc;
        rc = ozaki_split(st, gb, gb, Tg, gb, 1, 1.0, 0, q.oz_t, q.oz_tb, &ot);
        if (rc) return rc;
        rc = ozaki_gemm_pre(st, oa, ot, 1.0, 0.0, VT, n, status, 8);
        if (rc) return rc;
        // Yt = Z_o^T V (k x gb), then Z_o -= (V T) Yt^T
        rc = ozaki_split(st, k, m, Zo, ldz, 1, 1.0, 0, gws, gsz, &oz);
        if (rc) return rc;
        rc = ozaki_gemm_pre(st, oz, ov, 1.0, 0.0, Yt, k, status, slices);
        if (rc) return rc;
        rc = ozaki_gemm(st, m, k, gb, -1.0, VT, 1, n, 1.0, Yt, 1, k, 1.0, 1.0, Zo, ldz, gws, gsz, status, 0, slices);
        if (rc) return rc;
    }
    return 0;
}

}  // namespace sk
