// qtrd_df.cu -- the Q_trd back-transformation (Sec. 2.1 step 3(a), Algorithm 1
// step 4: the bulge-chase reflectors applied in reverse generation order) in
// double-float arithmetic on the FP32 pipe.
//
// Every quantity is an unevaluated sum hi + lo of two FP32 numbers (about 48
// significant bits).  Products use the exact FMA two-product, sums the exact
// two-sum (Knuth), so a dot product or an update is accurate to about 2^-46 of
// its terms' magnitudes: FP64-level accuracy for the eigenvector bounds, from
// a pipe 64 times wider than GB300's FP64 pipe.  It serves the solves whose
// eigenvectors cannot be refined afterwards (no complete basis: nev < n/2)
// and which would otherwise take Q_trd in FP64.
//
// Structure (the FP32 sliding-window kernel's): reflectors grouped into
// blocks of 64 sweeps x one step (a parallelogram of rows top .. top+126);
// each CTA owns a slab of columns, eight threads per column (row phase q), and
// keeps the block's window in registers; consecutive blocks of a group share
// 63 rows, so the window slides by 64 rows, the 64 new rows arriving by
// cp.async while the block computes.  The FP64 reflectors of the next block
// arrive by one bulk copy and are split into hi / lo pairs in place.
//
// Register window.  Thread q holds window rows 8u + q (u < 16).  The
// reflector at offset off = 8m + r (r = off mod 8) touches rows off .. off+63,
// that is for this thread the rows 8(m + w) + q with w = 1..7 always, plus
// w = 0 when q >= r or w = 8 when q < r: exactly 8 elements.  The registers
// are kept rotated so that register w holds row 8(m + w) + q: then every
// register index is a compile-time constant for all eight reflectors of one
// m (r only moves shared-memory offsets, so they run as a loop, keeping the
// code small), and one rotation by a register between consecutive m keeps
// the invariant.  Eight threads per column give twice the warps of four, so
// the four schedulers of an SM get near-equal shares of a slab.
#include "common.cuh"
#include "internal.h"
#include "sm100.cuh"

namespace sk {
namespace {

constexpr int DB = 64;              // band width = reflector length
constexpr int DELL = 64;            // sweeps per block
constexpr int DH = DELL + DB - 1;   // window height
constexpr int P = 8;                // threads per column (row phases)
constexpr int NR = 128 / P;         // window rows per thread
constexpr int MS = DELL / P;        // rotation steps per block
constexpr int DLD = 72;             // staging leading dimension in doubles (conflict-free halves)
constexpr int QD_MAXT = 512;        // threads per CTA at most (64 columns)

__host__ __device__ inline int df_qsteps(int n, int s) { return (s <= n - 3) ? 1 + (n - 3 - s) / DB : 0; }

// ---- conversions with integer operations only (the FP64 pipe stays idle) --
// x = hi + lo + d with hi the truncation of x to 24 bits and lo the rounded
// rest: |d| <= 2^-47 |x|.  |x| < 2^-100 gives (0, 0); the rest of a value
// below 2^-74 is dropped (both errors are absolute and below 2^-97).
SK_DEV float2 df_split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffu);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    if (e < 1023 - 100) return make_float2(0.f, 0.f);
    const unsigned long long mant = b & ((1ull << 52) - 1);
    const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(mant >> 29));
    const unsigned rest = (unsigned)(mant & ((1u << 29) - 1));
    float lo = 0.f;
    if (e >= 949 && rest != 0) {
        // rest x 2^(e - 1075); 2^(e - 1075) is a normal float for e >= 949
        lo = __fmul_rn(__uint2float_rn(rest), __uint_as_float((unsigned)(e - 948) << 23));
        if (sign) lo = -lo;
    }
    return make_float2(hi, lo);
}
// FP32 -> FP64, exact for normal floats; subnormals become 0.
SK_DEV double df_f2d(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0) return 0.0;
    const unsigned long long d = ((unsigned long long)(u >> 31) << 63) |
                                 ((unsigned long long)(e == 255 ? 2047u : e + 896u) << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}
SK_DEV double df_join(float hi, float lo) { return df_f2d(hi) + df_f2d(lo); }

// ---- double-float arithmetic (no contraction: explicit roundings) ---------
SK_DEV void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
SK_DEV void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
SK_DEV void df_add(float& ah, float& al, float bh, float bl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    fast_two_sum(s, e, ah, al);
}
// S + C += v z (v = vh + vl, z = zh + zl; the vl zl term is below 2^-48)
SK_DEV void dot_term(float vh, float vl, float zh, float zl, float& S, float& C) {
    const float p = __fmul_rn(vh, zh);
    float e = __fmaf_rn(vh, zh, -p);
    e = __fmaf_rn(vh, zl, e);
    e = __fmaf_rn(vl, zh, e);
    float s, err;
    two_sum(S, p, s, err);
    S = s;
    C = __fadd_rn(C, __fadd_rn(err, e));
}
// z -= a v
SK_DEV void axpy_term(float ah, float al, float vh, float vl, float& zh, float& zl) {
    const float p = __fmul_rn(ah, vh);
    float e = __fmaf_rn(ah, vh, -p);
    e = __fmaf_rn(ah, vl, e);
    e = __fmaf_rn(al, vh, e);
    float s, err;
    two_sum(zh, -p, s, err);
    zh = s;
    zl = __fadd_rn(zl, __fsub_rn(err, e));
}

struct DfSmem {
    double v[2][DELL * DB];  // a block's FP64 reflectors (bulk copy), then their (hi, lo) pairs in place
    float2 tau[2][DELL];
    double zin[64 * DLD];    // the next block's 64 new window rows
    double zout[64 * DLD];   // the block's 64 finished rows
    uint64_t bar[2];
};

// One reflector at offset off = P m + r of the block: vb points at its element
// 0 (hi, lo pairs), H / L registers in the rotated layout of m.  Thread q's
// elements are i = P w + q - r for w = 1..7 and the edge w = 0 (q >= r) or
// w = 8 (q < r); every register index is a compile-time constant, r and q
// only move the shared-memory offsets and pick the edge register.
SK_DEV void df_reflector(float (&H)[NR], float (&L)[NR], const float2* __restrict__ vb, float2 tau, int q, int r) {
    if (tau.x == 0.f) return;  // absent step or zero tail: H = I
    const bool low = q >= r;
    const float2 ve = vb[low ? q - r : DB + q - r];
    const float2* vw = vb + P + q - r;  // vw[P (w - 1)] = element P w + q - r, w = 1..7
    const float eh0 = low ? H[0] : H[P], el0 = low ? L[0] : L[P];
    float S0 = 0.f, C0 = 0.f, S1 = 0.f, C1 = 0.f;
    dot_term(ve.x, ve.y, eh0, el0, S0, C0);
#pragma unroll
    for (int w = 1; w < P; w++) {
        const float2 v = vw[P * (w - 1)];
        if (w & 1) dot_term(v.x, v.y, H[w], L[w], S1, C1);
        else dot_term(v.x, v.y, H[w], L[w], S0, C0);
    }
    df_add(S0, C0, S1, C1);
#pragma unroll
    for (int o = 1; o < P; o <<= 1)
        df_add(S0, C0, __shfl_xor_sync(0xffffffffu, S0, o), __shfl_xor_sync(0xffffffffu, C0, o));
    // a = tau (v^T z)
    float ah, al;
    {
        const float p = __fmul_rn(tau.x, S0);
        float e = __fmaf_rn(tau.x, S0, -p);
        e = __fmaf_rn(tau.x, C0, e);
        e = __fmaf_rn(tau.y, S0, e);
        fast_two_sum(p, e, ah, al);
    }
    float eh = eh0, el = el0;
    axpy_term(ah, al, ve.x, ve.y, eh, el);
    if (low) {
        H[0] = eh;
        L[0] = el;
    } else {
        H[P] = eh;
        L[P] = el;
    }
#pragma unroll
    for (int w = 1; w < P; w++) {
        const float2 v = vw[P * (w - 1)];
        axpy_term(ah, al, v.x, v.y, H[w], L[w]);
    }
}

__global__ void __launch_bounds__(QD_MAXT, 1)
qtrd_df_kernel(int n, const double* __restrict__ Vtrd, const double* __restrict__ tautrd, double* __restrict__ Z,
               int ldz, int ncols, int slab, int* status) {
    extern __shared__ __align__(128) unsigned char qd_raw[];
    DfSmem& sm = *reinterpret_cast<DfSmem*>(qd_raw);
    const int nsw = n - 2;
    const int c0 = blockIdx.x * slab;
    const int nc = min(slab, ncols - c0);
    if (nc <= 0) return;
    const int t = threadIdx.x, T = blockDim.x;
    // every lane takes part in the shuffles; lanes past the slab work on zeros
    const int c = t / P, q = t % P;
    const bool own = c < nc;
    double* zc = Z + (size_t)(c0 + (own ? c : 0)) * ldz;
    if (t == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int ngroups = (nsw + DELL - 1) / DELL;
    // FP64 reflectors of block (g, k) into buffer buf (one thread); sweeps past
    // the last are not copied (their taus are zero)
    auto fetch = [&](int g, int k, int buf) {
        const int cnt = min(DELL, nsw - g * DELL);
        const size_t slot = (size_t)k * nsw + (size_t)g * DELL;
        const uint32_t bytes = (uint32_t)cnt * DB * sizeof(double);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&sm.bar[buf], bytes);
        bulk_g2s(sm.v[buf], Vtrd + slot * DB, bytes, &sm.bar[buf]);
    };
    auto tau_of = [&](int g, int k) -> double {
        const int s = g * DELL + t;
        return (t < DELL && s < nsw && k < df_qsteps(n, s)) ? __ldg(tautrd + (size_t)k * nsw + s) : 0.0;
    };
    if (t == 0) fetch(ngroups - 1, 0, 0);
    double tau_cur = tau_of(ngroups - 1, 0);
    int blk = 0;  // blocks so far: buffer blk & 1, barrier phase (blk >> 1) & 1
    for (int g = ngroups - 1; g >= 0; g--) {
        const int s0 = g * DELL;
        const int kmax = df_qsteps(n, s0);
        float H[NR], L[NR];
        {
            // window of block (g, 0), rotated for m = MS - 1: register w <- row
            // P ((w + MS - 1) mod NR) + q
            const int top = s0 + 1, Hh = min(DH, n - top);
#pragma unroll
            for (int w = 0; w < NR; w++) {
                const int r = P * ((w + MS - 1) % NR) + q;
                const float2 f = (own && r < Hh) ? df_split(zc[top + r]) : make_float2(0.f, 0.f);
                H[w] = f.x;
                L[w] = f.y;
            }
        }
        for (int k = 0; k < kmax; k++) {
            const int top = s0 + 1 + k * DB;
            const int buf = blk & 1;
            const bool more = k + 1 < kmax;
            // prefetch: the next block's reflectors and taus, and the 64 new
            // rows top + 127 .. top + 190 of block k + 1
            double tau_next = 0.0;
            if (more) {
                if (t == 0) fetch(g, k + 1, buf ^ 1);
                tau_next = tau_of(g, k + 1);
            } else if (g > 0) {
                if (t == 0) fetch(g - 1, 0, buf ^ 1);
                tau_next = tau_of(g - 1, 0);
            }
            if (more) {
                for (int e = t; e < 64 * nc; e += T) {
                    const int cc = e >> 6, j = e & 63, row = top + DH + j;
                    double* d = &sm.zin[cc * DLD + j];
                    if (row < n) {
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(d)),
                                     "l"(Z + (size_t)(c0 + cc) * ldz + row)
                                     : "memory");
                    } else {
                        *d = 0.0;
                    }
                }
            }
            if (!mbar_wait(&sm.bar[buf], (uint32_t)(blk >> 1) & 1u, status)) return;
            // split this block's reflectors in place; the generic writes are
            // fenced before the bulk copy that reuses the buffer two blocks on
            {
                float2* vf = reinterpret_cast<float2*>(sm.v[buf]);
                for (int e = t; e < DELL * DB; e += T) vf[e] = df_split(sm.v[buf][e]);
                if (t < DELL) sm.tau[buf][t] = df_split(tau_cur);
                fence_proxy_async_smem();
            }
            __syncthreads();
            const float2* vblk = reinterpret_cast<const float2*>(sm.v[buf]);
#pragma unroll 1
            for (int m = MS - 1; m >= 0; m--) {
#pragma unroll 1
                for (int r = P - 1; r >= 0; r--) {
                    const int off = P * m + r;
                    df_reflector(H, L, vblk + (size_t)off * DB, sm.tau[buf][off], q, r);
                }
                // renormalise the pairs these P reflectors touched (w = 0..P)
#pragma unroll
                for (int w = 0; w <= P; w++) {
                    float s, e;
                    two_sum(H[w], L[w], s, e);
                    H[w] = s;
                    L[w] = e;
                }
                if (m > 0) {
                    // register w now holds row P (m - 1 + w) + q
                    const float th = H[NR - 1], tl = L[NR - 1];
#pragma unroll
                    for (int w = NR - 1; w > 0; w--) {
                        H[w] = H[w - 1];
                        L[w] = L[w - 1];
                    }
                    H[0] = th;
                    L[0] = tl;
                }
            }
            // register u holds row P u + q now
            if (more) {
                // rows 0..63 are final for this group: out through shared memory
#pragma unroll
                for (int u = 0; u < NR / 2; u++) sm.zout[c * DLD + P * u + q] = df_join(H[u], L[u]);
                asm volatile("cp.async.wait_all;" ::: "memory");
                __syncthreads();
                for (int e = t; e < 64 * nc; e += T) {
                    const int cc = e >> 6, j = e & 63;
                    Z[(size_t)(c0 + cc) * ldz + top + j] = sm.zout[cc * DLD + j];  // top + 63 < n here
                }
                // slide by 64 rows and rotate for m = MS - 1: new row u' goes to
                // register (u' - MS + 1) mod NR; rows 0..62 are old rows
                // 64..126, rows 63..126 come from zin, row 127 is padding
                float NH[NR], NL[NR];
#pragma unroll
                for (int up = 0; up < NR; up++) {
                    const int dst = (up + NR - MS + 1) % NR;
                    if (up < NR / 2 - 1) {
                        NH[dst] = H[up + NR / 2];
                        NL[dst] = L[up + NR / 2];
                    } else {
                        const int j = P * up + q - (DH - DB);  // zin row of window row P up + q
                        float2 f = make_float2(0.f, 0.f);
                        if (up == NR / 2 - 1 && P * up + q <= DH - DB - 1) {
                            f = make_float2(H[NR - 1], L[NR - 1]);
                        } else if (j < 64) {
                            f = df_split(sm.zin[c * DLD + j]);
                        }
                        NH[dst] = f.x;
                        NL[dst] = f.y;
                    }
                }
#pragma unroll
                for (int w = 0; w < NR; w++) {
                    H[w] = NH[w];
                    L[w] = NL[w];
                }
                __syncthreads();
            } else {
                // last block of the group: the whole window is final
                const int Hh = min(DH, n - top);
                if (own) {
#pragma unroll
                    for (int u = 0; u < NR; u++) {
                        const int r = P * u + q;
                        if (r < Hh) zc[top + r] = df_join(H[u], L[u]);
                    }
                }
                __syncthreads();
            }
            tau_cur = tau_next;
            blk++;
        }
    }
}

}  // namespace

cudaError_t apply_qtrd_df(cudaStream_t st, int n, int b, const double* Vtrd, const double* tautrd, double* Z,
                          int ldz, int k, int* status) {
    if (b != DB) return cudaErrorInvalidValue;
    if (n < 3 || k <= 0) return cudaSuccess;
    // one CTA per SM (the staging takes 140 KB); slabs of at most 64 columns
    // sized so that the CTAs fill whole waves
    const int sms = device_sms();
    const int maxslab = QD_MAXT / P;
    int waves = 1, slab = maxslab;
    while (true) {
        slab = (k + sms * waves - 1) / (sms * waves);
        if (slab <= maxslab) break;
        waves++;
    }
    if (slab < 8) slab = (k < 8) ? k : 8;
    const int grid = (k + slab - 1) / slab;
    // at least 64 threads: thread t < 64 brings the tau of sweep t
    const int threads = max(64, (P * slab + 31) / 32 * 32);
    const size_t smem = sizeof(DfSmem);
    cudaFuncSetAttribute(qtrd_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    KtScope kt(st, KT_QTRD);
    qtrd_df_kernel<<<grid, threads, smem, st>>>(n, Vtrd, tautrd, Z, ldz, k, slab, status);
    count_launch();
    return cudaGetLastError();
}

}  // namespace sk
