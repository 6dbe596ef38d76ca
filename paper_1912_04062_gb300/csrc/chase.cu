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
constexpr int CH_THREADS = 256;

__host__ __device__ inline int nsteps_of(int n, int b, int s) {
    return (s <= n - 3) ? 1 + (n - 3 - s) / b : 0;
}

struct ChaseSmem {
    double B[CB * CLD];
    double D[CB * CLD];
    double C[CB * CLD];
    double v[CB];
    double w[CB];
    double red[4 * CB];
    double tau, beta;
};

__device__ void chase_task(int n, int s, int k, int nsw, double* __restrict__ AB, int ldab,
                           double* __restrict__ alpha, double* __restrict__ Vtrd,
                           double* __restrict__ tautrd, ChaseSmem& sm) {
    const int t = threadIdx.x;
    const int r = s + 1 + k * CB;
    const int L = min(CB, n - r);
    const int c0 = (k == 0) ? s : r - CB;
    const int nbc = (k == 0) ? 1 : CB;
    const int rc = r + CB;
    const int Lc = max(0, min(CB, n - rc));

    // ---- load B_k (L x nbc), D_k (strict lower, L x L), C_k (Lc x L)
    for (int e = t; e < L * nbc; e += CH_THREADS) {
        int i = e % L, j = e / L;
        sm.B[j * CLD + i] = __ldcg(AB + (size_t)(c0 + j) * ldab + (r + i - c0 - j));
    }
    for (int e = t; e < L * L; e += CH_THREADS) {
        int i = e % L, j = e / L;
        sm.D[j * CLD + i] = (i > j) ? __ldcg(AB + (size_t)(r + j) * ldab + (i - j)) : 0.0;
    }
    for (int e = t; e < Lc * L; e += CH_THREADS) {
        int i = e % Lc, j = e / Lc;
        sm.C[j * CLD + i] = __ldcg(AB + (size_t)(r + j) * ldab + (CB + i - j));
    }
    __syncthreads();

    // ---- reflector from B_k[:, 0] (dlarfg convention)
    if (t < 32) {
        double a = 0.0;
        for (int i = 1 + t; i < L; i += 32) a = fma(sm.B[i], sm.B[i], a);
        a = sk_warp_sum(a);
        if (t == 0) {
            double x0 = sm.B[0], tu, be, sc;
            if (a == 0.0) {
                tu = 0.0; be = x0; sc = 0.0;
            } else {
                double rr = sqrt(x0 * x0 + a);
                be = (x0 >= 0.0) ? -rr : rr;
                tu = (be - x0) / be;
                sc = 1.0 / (x0 - be);
            }
            sm.tau = tu;
            sm.beta = be;
            sm.v[0] = 1.0;
            sm.w[0] = sc;
        }
    }
    __syncthreads();
    const double tau = sm.tau;
    {
        const double sc = sm.w[0];
        for (int i = 1 + t; i < CB; i += CH_THREADS) sm.v[i] = (i < L) ? sm.B[i] * sc : 0.0;
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
    // first column of B_k becomes beta e1
    for (int i = t; i < L; i += CH_THREADS) sm.B[i] = (i == 0) ? sm.beta : 0.0;

    const int jj = t & (CB - 1), q = t >> 6;  // column/row index and quarter
    if (tau != 0.0) {
        // ---- left: B_k[:, 1:] -= tau v (v^T B_k[:, 1:])
        if (nbc > 1) {
            double a = 0.0;
            if (jj >= 1)
                for (int i = q * 16; i < min(L, q * 16 + 16); i++) a = fma(sm.v[i], sm.B[jj * CLD + i], a);
            sm.red[q * CB + jj] = a;
            __syncthreads();
            if (t < CB) sm.w[t] = tau * (sm.red[t] + sm.red[CB + t] + sm.red[2 * CB + t] + sm.red[3 * CB + t]);
            __syncthreads();
            for (int e = t; e < L * (CB - 1); e += CH_THREADS) {
                int i = e % L, j = 1 + e / L;
                sm.B[j * CLD + i] -= sm.v[i] * sm.w[j];
            }
            __syncthreads();
        }
        // ---- two-sided on skew D_k: y = D v, p = tau y, D += v p^T - p v^T
        {
            double a = 0.0;
            const int i = jj;
            if (i < L) {
                for (int j = q * 16; j < min(L, q * 16 + 16); j++) {
                    if (j < i) a = fma(sm.D[j * CLD + i], sm.v[j], a);
                    else if (j > i) a = fma(-sm.D[i * CLD + j], sm.v[j], a);
                }
            }
            sm.red[q * CB + jj] = a;
            __syncthreads();
            if (t < CB) sm.w[t] = tau * (sm.red[t] + sm.red[CB + t] + sm.red[2 * CB + t] + sm.red[3 * CB + t]);
            __syncthreads();
            for (int e = t; e < L * L; e += CH_THREADS) {
                int i = e % L, j = e / L;
                if (i > j) sm.D[j * CLD + i] += sm.v[i] * sm.w[j] - sm.w[i] * sm.v[j];
            }
            __syncthreads();
        }
        // ---- right: C_k -= tau (C_k v) v^T
        if (Lc > 0) {
            double a = 0.0;
            const int i = jj;
            if (i < Lc)
                for (int j = q * 16; j < min(L, q * 16 + 16); j++) a = fma(sm.C[j * CLD + i], sm.v[j], a);
            sm.red[q * CB + jj] = a;
            __syncthreads();
            if (t < CB) sm.w[t] = tau * (sm.red[t] + sm.red[CB + t] + sm.red[2 * CB + t] + sm.red[3 * CB + t]);
            __syncthreads();
            for (int e = t; e < Lc * L; e += CH_THREADS) {
                int i = e % Lc, j = e / Lc;
                sm.C[j * CLD + i] -= sm.w[i] * sm.v[j];
            }
        }
    }
    __syncthreads();

    // ---- store back
    for (int e = t; e < L * nbc; e += CH_THREADS) {
        int i = e % L, j = e / L;
        AB[(size_t)(c0 + j) * ldab + (r + i - c0 - j)] = sm.B[j * CLD + i];
    }
    for (int e = t; e < L * L; e += CH_THREADS) {
        int i = e % L, j = e / L;
        if (i > j) AB[(size_t)(r + j) * ldab + (i - j)] = sm.D[j * CLD + i];
    }
    for (int e = t; e < Lc * L; e += CH_THREADS) {
        int i = e % Lc, j = e / Lc;
        AB[(size_t)(r + j) * ldab + (CB + i - j)] = sm.C[j * CLD + i];
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
        for (int k = 0; k < ns; k++) {
            if (s > 0 && !sk_wait_flag_geq(prog + (s - 1), min(k + 3, nsp), status)) return;
            chase_task(n, s, k, nsw, AB, ldab, alpha, Vtrd, tautrd, sm);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                sk_st_release_s32(prog + s, k + 1);
            }
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
