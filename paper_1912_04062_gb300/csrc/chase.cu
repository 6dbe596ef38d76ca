// chase.cu -- band-to-tridiagonal reduction of a skew-symmetric band matrix
// by bulge chasing (Sec. 2.3.2, second half: "the reduction of a particular
// column introduces fill-in in the neighboring block"; diagonal blocks take the
// skew rank-2 update A <- A - v u^T + u v^T with u from a skew SYMV).
//
// Band storage (lower): AB[d + c*ldab] = A(c+d, c), 0 <= d <= 2b; rows
// b+1..2b hold the bulge.  Sweep s (s = 0..n-3) annihilates column s below its
// sub-diagonal; its step k works on rows/cols r_k = s+1+k b .. r_k+L-1:
//   B_k = A[r_k:r_k+L, r_{k-1}:r_{k-1}+b] (k >= 1; for k = 0 the column s)
//         -> a reflector H_k = I - tau v v^T from B_k[:, 0], applied from the
//            left to B_k (first column becomes beta e1);
//   D_k = A[r_k:r_k+L, r_k:r_k+L] (skew) -> H D H = D + v p^T - p v^T with
//         p = tau D v (the 0.5 tau^2 (v^T D v) v term is 0 for skew D);
//   C_k = A[r_k+b:r_k+2b, r_k:r_k+L] -> C H (creates the next bulge).
// Dependencies: step k of sweep s may run once sweep s-1 has finished step
// k+2 (the last region they share is the single element
// A(r_{k+2}, r_{k+1}) of sweep s-1), and after step k-1 of its own sweep.
// One persistent cooperative launch: CTA g owns sweeps g, g+G, ...; a per-sweep
// progress counter (release store / acquire load, capped spin) orders them.
#include "common.cuh"
#include "internal.h"

namespace sk {
namespace {

constexpr int CB = 64;          // band width handled by the kernel
constexpr int CLD = CB + 1;     // padded leading dimension in shared memory
constexpr int CH_THREADS = 1024;
constexpr int CH_NQ = CH_THREADS / 64;  // row groups of the dot products (1 CTA per SM)
constexpr int CH_QR = 64 / CH_NQ;       // rows per group

__host__ __device__ inline int nsteps_of(int n, int b, int s) {
    return (s <= n - 3) ? 1 + (n - 3 - s) / b : 0;
}

struct ChaseSmem {
    double buf[3][CB * CLD];  // B, D and C of the current step (B and C trade places)
    double v[CB];
    double wB[CB], wD[CB], wC[CB];
    double red[3][CH_NQ * CB];
    double tau, beta;
};

// Step k of sweep s.  B holds B_k already when have_b (it is the C block of
// step k-1 of the same sweep, which no other sweep touches in between: the
// neighbouring sweeps reach its rows only two steps later), and C is kept for
// step k+1 instead of being stored when keep_c.  The left update of B, the
// two-sided update of D and the right update of C depend only on (v, tau):
// their dot products share one pass and one reduction, their updates one pass.
__device__ void chase_task(int n, int s, int k, int nsw, double* __restrict__ AB, int ldab,
                           double* __restrict__ alpha, double* __restrict__ Vtrd, double* __restrict__ tautrd,
                           double* __restrict__ B, double* __restrict__ D, double* __restrict__ C, bool have_b,
                           bool keep_c, ChaseSmem& sm) {
    const int t = threadIdx.x;
    const int r = s + 1 + k * CB;
    const int L = min(CB, n - r);
    const int c0 = (k == 0) ? s : r - CB;
    const int nbc = (k == 0) ? 1 : CB;
    const int rc = r + CB;
    const int Lc = max(0, min(CB, n - rc));

    // ---- load B_k (L x nbc) unless kept, D_k (strict lower, L x L), C_k (Lc x L)
    if (!have_b)
        for (int e = t; e < L * nbc; e += CH_THREADS) {
            const int i = e % L, j = e / L;
            B[j * CLD + i] = __ldcg(AB + (size_t)(c0 + j) * ldab + (r + i - c0 - j));
        }
    for (int e = t; e < L * L; e += CH_THREADS) {
        const int i = e % L, j = e / L;
        D[j * CLD + i] = (i > j) ? __ldcg(AB + (size_t)(r + j) * ldab + (i - j)) : 0.0;
    }
    for (int e = t; e < Lc * L; e += CH_THREADS) {
        const int i = e % Lc, j = e / Lc;
        C[j * CLD + i] = __ldcg(AB + (size_t)(r + j) * ldab + (CB + i - j));
    }
    __syncthreads();

    // ---- reflector from B_k[:, 0] (dlarfg convention)
    if (t < 32) {
        double a = 0.0;
        for (int i = 1 + t; i < L; i += 32) a = fma(B[i], B[i], a);
        a = sk_warp_sum(a);
        if (t == 0) {
            const double x0 = B[0];
            double tu, be, sc;
            if (a == 0.0) {
                tu = 0.0; be = x0; sc = 0.0;
            } else {
                const double rr = sqrt(x0 * x0 + a);
                be = (x0 >= 0.0) ? -rr : rr;
                tu = (be - x0) / be;
                sc = 1.0 / (x0 - be);
            }
            sm.tau = tu;
            sm.beta = be;
            sm.wB[0] = sc;
        }
    }
    __syncthreads();
    const double tau = sm.tau;
    {
        const double sc = sm.wB[0];
        for (int i = t; i < CB; i += CH_THREADS) sm.v[i] = (i == 0) ? 1.0 : ((i < L) ? B[i] * sc : 0.0);
    }
    __syncthreads();
    {
        double* vg = Vtrd + ((size_t)k * nsw + s) * CB;
        for (int i = t; i < CB; i += CH_THREADS) vg[i] = sm.v[i];
        if (t == 0) {
            tautrd[(size_t)k * nsw + s] = tau;
            if (k == 0) alpha[s] = -sm.beta;  // T[s, s+1] = -T[s+1, s]
        }
    }

    const int jj = t & (CB - 1), q = t >> 6;  // column/row index and row group
    if (tau != 0.0) {
        // ---- partial dots of the three updates (CH_NQ row groups of CH_QR)
        {
            double aB = 0.0, aD = 0.0, aC = 0.0;
            const int lo = q * CH_QR, hi = min(L, q * CH_QR + CH_QR);
            if (nbc > 1 && jj >= 1)  // (v^T B)_j
                for (int i = lo; i < hi; i++) aB = fma(sm.v[i], B[jj * CLD + i], aB);
            if (jj < L)              // (D v)_i, D skew from its lower part
                for (int j = lo; j < hi; j++) {
                    if (j < jj) aD = fma(D[j * CLD + jj], sm.v[j], aD);
                    else if (j > jj) aD = fma(-D[jj * CLD + j], sm.v[j], aD);
                }
            if (jj < Lc)             // (C v)_i
                for (int j = lo; j < hi; j++) aC = fma(C[j * CLD + jj], sm.v[j], aC);
            sm.red[0][q * CB + jj] = aB;
            sm.red[1][q * CB + jj] = aD;
            sm.red[2][q * CB + jj] = aC;
        }
        __syncthreads();
        if (t < 3 * CB) {
            const int which = t / CB, col = t % CB;
            double acc = 0.0;
#pragma unroll
            for (int h = 0; h < CH_NQ; h++) acc += sm.red[which][h * CB + col];
            (which == 0 ? sm.wB : (which == 1 ? sm.wD : sm.wC))[col] = tau * acc;
        }
        __syncthreads();
        // ---- updates: B[:, 1:] -= v wB^T; D += v p^T - p v^T (p = wD = tau D v;
        // the 1/2 tau^2 (v^T D v) v term is 0 for skew D); C -= wC v^T
        if (nbc > 1)
            for (int e = t; e < L * (CB - 1); e += CH_THREADS) {
                const int i = e % L, j = 1 + e / L;
                B[j * CLD + i] -= sm.v[i] * sm.wB[j];
            }
        for (int e = t; e < L * L; e += CH_THREADS) {
            const int i = e % L, j = e / L;
            if (i > j) D[j * CLD + i] += sm.v[i] * sm.wD[j] - sm.wD[i] * sm.v[j];
        }
        for (int e = t; e < Lc * L; e += CH_THREADS) {
            const int i = e % Lc, j = e / Lc;
            C[j * CLD + i] -= sm.wC[i] * sm.v[j];
        }
    }
    // first column of B_k becomes beta e1
    for (int i = t; i < L; i += CH_THREADS) B[i] = (i == 0) ? sm.beta : 0.0;
    __syncthreads();

    // ---- store back (C only when no later step of this sweep takes it)
    for (int e = t; e < L * nbc; e += CH_THREADS) {
        const int i = e % L, j = e / L;
        AB[(size_t)(c0 + j) * ldab + (r + i - c0 - j)] = B[j * CLD + i];
    }
    for (int e = t; e < L * L; e += CH_THREADS) {
        const int i = e % L, j = e / L;
        if (i > j) AB[(size_t)(r + j) * ldab + (i - j)] = D[j * CLD + i];
    }
    if (!keep_c)
        for (int e = t; e < Lc * L; e += CH_THREADS) {
            const int i = e % Lc, j = e / Lc;
            AB[(size_t)(r + j) * ldab + (CB + i - j)] = C[j * CLD + i];
        }
}

__global__ void __launch_bounds__(CH_THREADS)
chase_kernel(int n, double* __restrict__ AB, int ldab, double* __restrict__ alpha,
             double* __restrict__ Vtrd, double* __restrict__ tautrd, int* prog, int* status) {
    extern __shared__ __align__(16) unsigned char chase_raw[];
    ChaseSmem& sm = *reinterpret_cast<ChaseSmem*>(chase_raw);
    const int nsw = n - 2;
    for (int s = blockIdx.x; s < nsw; s += gridDim.x) {
        const int ns = nsteps_of(n, CB, s);
        const int nsp = (s > 0) ? nsteps_of(n, CB, s - 1) : 0;
        double* B = sm.buf[0];
        double* D = sm.buf[1];
        double* C = sm.buf[2];
        bool have_b = false;
        for (int k = 0; k < ns; k++) {
            if (s > 0 && !sk_wait_flag_geq(prog + (s - 1), min(k + 3, nsp), status)) return;
            const bool keep_c = k + 1 < ns;  // step k+1 starts from this C
            chase_task(n, s, k, nsw, AB, ldab, alpha, Vtrd, tautrd, B, D, C, have_b, keep_c, sm);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                sk_st_release_s32(prog + s, k + 1);
            }
            double* tmp = B;  // C_k is B_{k+1}
            B = C;
            C = tmp;
            have_b = keep_c;
        }
    }
}

__global__ void chase_tail_kernel(int n, const double* __restrict__ AB, int ldab, double* __restrict__ alpha) {
    if (threadIdx.x == 0 && n >= 2) alpha[n - 2] = -AB[(size_t)(n - 2) * ldab + 1];
}

}  // namespace

int chase_steps(int n, int b) { return n >= 3 ? nsteps_of(n, b, 0) : 0; }

size_t chase_ws(int n, int b) {
    (void)b;
    return align_up(sizeof(int) * (size_t)(n > 2 ? n : 1)) + 256;
}

int chase(cudaStream_t st, int n, int b, double* AB, int ldab, double* alpha, double* Vtrd, double* tautrd,
          void* ws, size_t ws_bytes, int* d_status, unsigned spin_cap) {
    (void)spin_cap;
    if (b != CB) return SKEW_ERR_UNSUPPORTED;
    if (n < 2) return 0;
    if (ldab < 2 * b + 1) return SKEW_ERR_UNSUPPORTED;
    const int nsw = n - 2;
    if (nsw > 0) {
        Carve cv(ws, ws_bytes);
        int* prog = cv.take<int>((size_t)nsw);
        if (!cv.ok) return SKEW_ERR_WORKSPACE;
        if (cudaMemsetAsync(prog, 0, sizeof(int) * (size_t)nsw, st) != cudaSuccess) return SKEW_ERR_CUDA;
        const size_t smem = sizeof(ChaseSmem);
        cudaFuncSetAttribute(chase_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, chase_kernel, CH_THREADS, smem);
        if (occ < 1) return SKEW_ERR_LAUNCH;
        int G = occ * device_sms();
        if (G > nsw) G = nsw;
        void* args[] = {&n, &AB, &ldab, &alpha, &Vtrd, &tautrd, &prog, &d_status};
        KtScope kt(st, KT_CHASE);
        if (cudaLaunchCooperativeKernel((void*)chase_kernel, dim3(G), dim3(CH_THREADS), args, smem, st) != cudaSuccess)
            return SKEW_ERR_LAUNCH;
        count_launch();
    }
    chase_tail_kernel<<<1, 32, 0, st>>>(n, AB, ldab, alpha);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : SKEW_ERR_CUDA;
}

}  // namespace sk
