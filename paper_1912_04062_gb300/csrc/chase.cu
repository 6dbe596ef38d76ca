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
// k+1 and after step k-1 of its own sweep; the single element it shares with
// step k+2 of sweep s-1 is completed one step later (see chase_task).
// One persistent cooperative launch: CTA g owns sweeps g, g+G, ...; a per-sweep
// progress counter (release store / acquire load, capped spin) orders them.
#include "common.cuh"
#include "internal.h"

namespace sk {
namespace {

constexpr int CB = 64;          // band width handled by the kernel
constexpr int CLD = CB + 1;     // padded leading dimension in shared memory
constexpr int CH_THREADS = 1024;
constexpr int CH_EPT = CB * CB / CH_THREADS;  // block elements per thread
constexpr int CH_JS = CH_THREADS / CB;        // column stride of a thread's elements

__host__ __device__ inline int nsteps_of(int n, int b, int s) {
    return (s <= n - 3) ? 1 + (n - 3 - s) / b : 0;
}

struct ChaseSmem {
    double buf[3][CB * CLD];  // B, D (both triangles) and C of the current step; B and C trade places
    double v[CB], vprev[CB];
    double wB[CB], wD[CB], wC[CB];
    double tau, beta, tauprev;
    int ok;
};

// Sum over one warp of x_i^2 for 1 <= i < hi, x = B[0:64, 0].
__device__ __forceinline__ double chase_ssq(const double* __restrict__ B, int hi) {
    const int lane = threadIdx.x & 31;
    const double x1 = (lane >= 1 && lane < hi) ? B[lane] : 0.0;
    const double x2 = (lane + 32 < hi) ? B[lane + 32] : 0.0;
    return sk_warp_sum(fma(x2, x2, x1 * x1));
}

// Reflector H = I - tau v v^T with H x = beta e1 for x = B[0:L, 0] (dlarfg
// convention) given a = sum of x_i^2 over 1 <= i < L, formed by one warp:
// sm.v (zero beyond L), sm.tau, sm.beta and the copies kept for the
// back-transformation.
__device__ void chase_reflector(const double* __restrict__ B, int L, double a, ChaseSmem& sm,
                                double* __restrict__ vg, double* __restrict__ tg, float* __restrict__ vf,
                                float* __restrict__ tf, double* __restrict__ alpha_s) {
    const int lane = threadIdx.x & 31;
    const double x0 = B[0];
    const double x1 = (lane < L) ? B[lane] : 0.0;
    const double x2 = (lane + 32 < L) ? B[lane + 32] : 0.0;
    double tu, be, sc;
    if (a == 0.0) {
        tu = 0.0; be = x0; sc = 0.0;
    } else {
        const double rr = sqrt(x0 * x0 + a);
        be = (x0 >= 0.0) ? -rr : rr;
        tu = (be - x0) / be;
        sc = 1.0 / (x0 - be);
    }
    const double v1 = (lane == 0) ? 1.0 : x1 * sc;
    const double v2 = x2 * sc;
    sm.v[lane] = v1;
    sm.v[lane + 32] = v2;
    if (vg) {
        vg[lane] = v1;
        vg[lane + 32] = v2;
    }
    if (vf) {
        vf[lane] = (float)v1;
        vf[lane + 32] = (float)v2;
    }
    if (lane == 0) {
        sm.tau = tu;
        sm.beta = be;
        if (tg) *tg = tu;
        if (tf) *tf = (float)tu;
        if (alpha_s) *alpha_s = -be;  // T[s, s+1] = -T[s+1, s]
    }
}

// Strict-lower element u (0, 1) of thread t in D: "virtual column" p pairs
// column p (rows p+1..63) with column 62-p (rows 63-p..63), 64 elements for
// p < 31 and the 32 of column 31 for p = 31, so the 2016 elements fill the
// warps densely (the FP64 pipe costs a whole warp whatever the active lanes).
__device__ __forceinline__ bool chase_lower(int t, int u, int& i, int& j) {
    const int p = (t >> 6) + 16 * u, ii = t & 63;
    if (ii < 63 - p) {
        i = p + 1 + ii;
        j = p;
        return true;
    }
    i = ii;
    j = 62 - p;
    return p < 31;
}

// Step k of sweep s.  B holds B_k already when have_b (it is the C block of
// step k-1 of the same sweep), so its reflector is formed while the previous
// sweep's progress is awaited; C is kept for step k+1 instead of being stored
// when keep_c.  Step k shares with step k+2 of sweep s-1 only the element
// E = A(r_k+2b-1, r_k+b-1), the last row and column of C_k, whose row is
// (0, .., 0, E) before step k: with defer_e, row 63 of C_k is left at zero
// and step k+1 (fix_e) completes it from the final E as
// E e_63^T - (tau (E v_63)) v^T, the same operations the full update takes,
// so a sweep need only wait for step k+1 of its predecessor.  The work is bound by the
// FP64 pipe (2 FMA per clock per SM): every FP64 warp instruction is spent on
// needed elements, and the 3 x 64 matrix-vector products take two threads
// each (rows split between the half-warps) with a single combining add.
// Thread t owns the elements (t mod 64, t/64 + 16 u) of B and C and two
// elements of D's strict lower part; it keeps the D and C values in registers
// from the load to the update.  Returns false when the wait gave up.
__device__ bool chase_task(int n, int s, int k, int nsw, const int* __restrict__ prog_prev, int want,
                           int* __restrict__ status, double* __restrict__ AB, int ldab, double* __restrict__ alpha,
                           double* __restrict__ Vtrd, double* __restrict__ tautrd, float* __restrict__ V32,
                           float* __restrict__ tau32, int nsw64, double* __restrict__ B, double* __restrict__ D,
                           double* __restrict__ C, bool have_b, bool keep_c, bool fix_e, bool defer_e,
                           ChaseSmem& sm, unsigned spin_cap) {
    const int t = threadIdx.x, warp = t >> 5;
    const int r = s + 1 + k * CB;
    const int L = min(CB, n - r);
    const int Lc = max(0, min(CB, n - r - CB));
    double* vg = Vtrd ? Vtrd + ((size_t)k * nsw + s) * CB : nullptr;
    double* tg = tautrd ? tautrd + (size_t)k * nsw + s : nullptr;
    float* vf = V32 ? V32 + ((size_t)k * nsw64 + s) * CB : nullptr;
    float* tf = tau32 ? tau32 + (size_t)k * nsw64 + s : nullptr;

    // a kept B gives its reflector before the wait, or with fix_e all of its
    // sum of squares but the row-63 term
    double ssq = 0.0;
    if (have_b && warp == 0) {
        ssq = chase_ssq(B, fix_e ? CB - 1 : L);
        if (!fix_e) chase_reflector(B, L, ssq, sm, vg, tg, vf, tf, nullptr);
    }
    if (t == 32) {
        int ok = 1;
        if (want > 0) {
            unsigned polls = 0;
            // error word every 256 polls, sleeps only after 256 tries
            while (sk_ld_acquire_s32(prog_prev) < want) {
                ++polls;
                if (polls > spin_cap || ((polls & 255u) == 0 && *(volatile int*)status != 0)) {
                    ok = 0;
                    break;
                }
                if (polls > 256) __nanosleep(32);
            }
            if (!ok) sk_set_error(status, SKEW_ERR_DEVICE_TIMEOUT);
        }
        sm.ok = ok;
    }
    __syncthreads();
    if (!sm.ok) return false;

    // ---- D_k (strict lower part) and C_k into registers
    const int i = t & (CB - 1), q = t >> 6;
    double d[2], c[CH_EPT];
    int di[2], dj[2];
    bool dok[2], dv[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
        dok[u] = chase_lower(t, u, di[u], dj[u]);
        dv[u] = dok[u] && di[u] < L;
        d[u] = dv[u] ? __ldcg(AB + (size_t)(r + dj[u]) * ldab + (di[u] - dj[u])) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < CH_EPT; u++) {
        const int j = q + CH_JS * u;
        c[u] = (i < Lc && j < L && !(defer_e && i == CB - 1)) ? __ldcg(AB + (size_t)(r + j) * ldab + (CB + i - j))
                                                               : 0.0;
    }
    if (warp == 0 && (!have_b || fix_e)) {
        const int lane = t & 31;
        if (!have_b) {
            // k = 0: B_0 is column s, rows r .. r+L-1
            const double* col = AB + (size_t)s * ldab + (r - s);
            B[lane] = (lane < L) ? __ldcg(col + lane) : 0.0;
            B[lane + 32] = (lane + 32 < L) ? __ldcg(col + lane + 32) : 0.0;
            __syncwarp();
            ssq = chase_ssq(B, L);
        } else {
            // row 63 of B_k = C_{k-1} from the now final E = A(r+b-1, r-1)
            const double E = __ldcg(AB + (size_t)(r - 1) * ldab + CB);
            const double wc = sm.tauprev * (E * sm.vprev[CB - 1]);
            B[lane * CLD + CB - 1] = fma(-wc, sm.vprev[lane], 0.0);
            B[(lane + 32) * CLD + CB - 1] = fma(-wc, sm.vprev[lane + 32], (lane == 31) ? E : 0.0);
            ssq = fma(wc, wc, ssq);  // x_63 = -wc (v_0 = 1)
        }
        __syncwarp();
        chase_reflector(B, L, ssq, sm, vg, tg, vf, tf, have_b ? nullptr : alpha + s);
    }
    // D in both triangles (D^T = -D, zero diagonal and outside the block), C
#pragma unroll
    for (int u = 0; u < 2; u++) {
        if (dok[u]) {
            D[dj[u] * CLD + di[u]] = d[u];
            D[di[u] * CLD + dj[u]] = -d[u];
        }
    }
    if (t < CB) D[t * CLD + t] = 0.0;
#pragma unroll
    for (int u = 0; u < CH_EPT; u++) C[(q + CH_JS * u) * CLD + i] = c[u];
    __syncthreads();

    // ---- (v^T B)_col, (D v)_col, (C v)_col on warps 0..11: warp w takes
    // product w/4 for columns 16 (w mod 4) + 0..15, lanes 16..31 the rows
    // 32..63 of the lanes 0..15; two accumulators per thread keep the FP64
    // pipe fed.  Step 0 has no B product.
    if (warp < 12 && (have_b || warp >= 4)) {
        const int lane = t & 31, h = lane >> 4, col = 16 * (warp & 3) + (lane & 15), which = warp >> 2;
        const double* vr = sm.v + 32 * h;
        double a0 = 0.0, a1 = 0.0;
        if (which == 0) {
            const double* x = B + col * CLD + 32 * h;
#pragma unroll 8
            for (int e = 0; e < 32; e += 2) {
                a0 = fma(vr[e], x[e], a0);
                a1 = fma(vr[e + 1], x[e + 1], a1);
            }
        } else {
            const double* x = ((which == 1) ? D : C) + 32 * h * CLD + col;
#pragma unroll 8
            for (int e = 0; e < 32; e += 2) {
                a0 = fma(x[e * CLD], vr[e], a0);
                a1 = fma(x[(e + 1) * CLD], vr[e + 1], a1);
            }
        }
        double a = a0 + a1;
        a += __shfl_down_sync(0xffffffffu, a, 16);
        if (h == 0) (which == 0 ? sm.wB : (which == 1 ? sm.wD : sm.wC))[col] = sm.tau * a;
    }
    __syncthreads();

    // ---- updates, straight to memory: B[:, 1:] -= v wB^T and B[:, 0] =
    // beta e1; D += v p^T - p v^T with p = wD = tau D v (the 1/2 tau^2
    // (v^T D v) v term is 0 for skew D); C -= wC v^T (kept as the next B)
    {
        const double vi = sm.v[i], wCi = sm.wC[i], beta = sm.beta;
#pragma unroll
        for (int u = 0; u < CH_EPT; u++) {
            const int j = q + CH_JS * u;
            const double vj = sm.v[j];
            if (i < L) {
                if (have_b) {
                    const double bv = (j == 0) ? ((i == 0) ? beta : 0.0) : fma(-vi, sm.wB[j], B[j * CLD + i]);
                    AB[(size_t)(r - CB + j) * ldab + (CB + i - j)] = bv;
                } else if (j == 0) {
                    AB[(size_t)s * ldab + (r - s + i)] = (i == 0) ? beta : 0.0;
                }
            }
            const bool inc = i < Lc && j < L;
            const double cv = inc ? fma(-wCi, vj, c[u]) : 0.0;
            if (keep_c)
                C[j * CLD + i] = cv;
            else if (inc)
                AB[(size_t)(r + j) * ldab + (CB + i - j)] = cv;
        }
        if (defer_e && t < CB) {
            sm.vprev[t] = sm.v[t];
            if (t == 0) sm.tauprev = sm.tau;
        }
#pragma unroll
        for (int u = 0; u < 2; u++) {
            if (dv[u]) {
                const int ii = di[u], jj = dj[u];
                AB[(size_t)(r + jj) * ldab + (ii - jj)] = fma(-sm.wD[ii], sm.v[jj], fma(sm.v[ii], sm.wD[jj], d[u]));
            }
        }
    }
    return true;
}

__global__ void __launch_bounds__(CH_THREADS)
chase_kernel(int n, double* __restrict__ AB, int ldab, double* __restrict__ alpha,
             double* __restrict__ Vtrd, double* __restrict__ tautrd, float* __restrict__ V32,
             float* __restrict__ tau32, int* prog, int* status, unsigned spin_cap) {
    extern __shared__ __align__(16) unsigned char chase_raw[];
    ChaseSmem& sm = *reinterpret_cast<ChaseSmem*>(chase_raw);
    const int nsw = n - 2, nsw64 = (nsw + 63) / 64 * 64;
    for (int s = blockIdx.x; s < nsw; s += gridDim.x) {
        const int ns = nsteps_of(n, CB, s);
        const int nsp = (s > 0) ? nsteps_of(n, CB, s - 1) : 0;
        double* B = sm.buf[0];
        double* D = sm.buf[1];
        double* C = sm.buf[2];
        bool have_b = false, fix_e = false;
        for (int k = 0; k < ns; k++) {
            const bool keep_c = k + 1 < ns;  // step k+1 starts from this C
            // steps 0..k+1 of sweep s-1 done; E of C_k is final only after
            // its step k+2 (when that exists), awaited by step k+1
            const int want = (s > 0) ? min(k + 2, nsp) : 0;
            const bool defer_e = s > 0 && n - (s + 1 + k * CB) >= 2 * CB && k + 2 < nsp;
            if (!chase_task(n, s, k, nsw, prog + (s > 0 ? s - 1 : 0), want, status, AB, ldab, alpha, Vtrd, tautrd,
                            V32, tau32, nsw64, B, D, C, have_b, keep_c, fix_e, defer_e, sm, spin_cap))
                return;
            // all stores of the step precede the release (bar.sync, then a
            // gpu-scope release by one thread)
            __syncthreads();
            if (threadIdx.x == 0) sk_st_release_s32(prog + s, k + 1);
            double* tmp = B;  // C_k is B_{k+1}
            B = C;
            C = tmp;
            have_b = keep_c;
            fix_e = defer_e;
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
          void* ws, size_t ws_bytes, int* d_status, unsigned spin_cap, float* V32, float* tau32) {
    if (spin_cap == 0) spin_cap = SK_SPIN_CAP;
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
        void* args[] = {&n, &AB, &ldab, &alpha, &Vtrd, &tautrd, &V32, &tau32, &prog, &d_status, &spin_cap};
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
