// ozaki_gemm.cu -- FP64-accurate matrix product on the BF16 tensor cores
// (tcgen05.mma kind::f16, FP32 accumulation in TMEM), for the eigenpair
// refinement of the mixed form.  Not in the paper; on GB300 native FP64 runs at
// about 1 TFLOP/s, so the refinement's n^3 products are done as exact slice
// products (an error-free splitting in the manner of Ozaki, Ogita, Oishi and
// Rump, "Error-free transformations of matrix multiplication", 2012).
//
// Splitting.  Row r of an operand is scaled by 2^-e_r with e_r the smallest
// integer such that every |x| < 2^e_r.  The scaled value x' (|x'| < 1), as a
// 56-bit fixed-point integer, is cut into SL = 8 digits d_0..d_7 with
// rounding shifts (|d_0| <= 128, |d_i| <= 64 for i > 0): every digit is an
// integer that BF16 represents exactly, and
// x = 2^e_r * sum_i d_i 2^-7(i+1) + O(2^(e_r - 56)).
//
// Product.  C[r][c] = 2^(e_r + f_c - 14) * sum_L 2^-7L T_L[r][c] with
// T_L = sum_{i+j=L} D_i E_j^T over the kept levels L < s (s = 8: 36 slice
// pairs, the dropped ones below 2^-63 of |a_r|max |b_c|max per term; fewer
// slices give a cheaper product accurate to about 2^-7s).  The level sums are
// taken over K groups of 256: level 0 is a sum of 256 products of size
// <= 2^14, level L >= 1 of 256 (L + 3) 2^12-sized terms (two pairs with a
// leading digit, |d_0| <= 128), both below 2^24, so FP32 accumulation in TMEM
// is exact.  After each group the level accumulators (s x 64 TMEM columns)
// are folded into a double-float (two FP32) running sum per output, which
// carries about 48 bits.
//
// Kernel: 128 x 64 output tile per CTA, 320 threads: warps 0-7 drain TMEM
// (warp w: lanes 32 (w & 3).. = rows, columns 32 (w >> 2)..) and accumulate;
// warp 8 issues TMA loads (the B digit
// slices of a 128-wide K chunk stay resident, A slices stream through two
// stages); warp 9 issues the MMAs.  TMEM holds one group of two chunks, so the
// MMAs of the next group start once the epilogue has drained the last one.
// With `lower` set, tiles wholly above the diagonal (every column index above
// every row index) are skipped: for symmetric or skew results whose upper
// triangle is not read.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "sm100.cuh"

namespace sk {

bool make_tmap_bf16(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_rows);

namespace {

constexpr int OM = 128;      // tile rows
constexpr int ON = 64;       // tile columns
constexpr int OKC = 128;     // K per chunk (two 64-wide swizzle atoms; the last chunk may hold one)
constexpr int OKA = 64;      // K per swizzle atom; K is padded to a multiple of it
constexpr int SL = 8;        // digit slices per operand
constexpr int OT = 320;      // threads per CTA: 8 epilogue warps, TMA warp, MMA warp
constexpr int OEPI = 256;    // epilogue threads

struct OzParams {
    int M, N, nchunks;
    int katoms;              // 64-wide K atoms in all (the last chunk holds one when odd)
    int Mp, Np;              // padded row counts of the slice planes
    int mt, nt;              // output tiles along M and N
    const int* ea;           // row exponents of A (M)
    const int* eb;           // row exponents of B (N)
    double alpha, beta;
    double* C;
    long long ldc;
    int* status;
    int s;                   // digit slices kept (levels L < s)
    int lower;               // skip tiles above the diagonal
};

struct OzSmem {
    static constexpr uint32_t B_ATOM = ON * 128;          // 64 rows x 128 B
    static constexpr uint32_t A_ATOM = OM * 128;          // 128 rows x 128 B
    static constexpr uint32_t B_BYTES = SL * 2 * B_ATOM;  // all slices of a chunk
    static constexpr uint32_t A_STAGE = 2 * A_ATOM;       // one slice of a chunk
    static constexpr size_t bytes() { return 1024 + B_BYTES + 2 * A_STAGE + 8 * 10 + 16; }
};

// Digits of x 2^-e (|x| < 2^e) without FP64 arithmetic: the significand is
// aligned to a 56-bit fixed-point integer M (|M| < 2^56, bits below 2^(e-56)
// dropped), then d_i = round(M_i / 2^(49 - 7i)), M_(i+1) = M_i - d_i 2^(49-7i)
// for i = 0..7 (shifts 49, 42, ..., 0), which leaves no remainder.
SK_DEV void oz_digits(double x, int e, float (&d)[8]) {
    const long long bits = __double_as_longlong(x);
    const int bexp = (int)((bits >> 52) & 0x7FF);
    long long M = 0;
    if (bexp != 0) {  // zero and subnormals (far below 2^(e-56) here) give 0
        long long mant = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;  // 53 bits, value mant 2^(bexp-1075)
        const int sh = bexp - 1075 - e + 56;  // x 2^-e 2^56 = mant 2^sh
        if (sh >= 0) mant <<= sh;          // sh <= 3 since |x| < 2^e
        else mant = (sh > -63) ? (mant >> (-sh)) : 0;
        M = (bits < 0) ? -mant : mant;
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int sh = 49 - 7 * i;
        const long long q = (sh > 0) ? ((M + (1LL << (sh - 1))) >> sh) : M;
        M -= q << sh;
        d[i] = (float)q;
    }
}

SK_DEV void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// (hi, lo) += x exactly up to the rounding of the final renormalisation
SK_DEV void df_add(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (x - bb);
    const float l = lo + e;
    const float h = s + l;
    lo = l - (h - s);
    hi = h;
}
SK_DEV void df_add_df(float& hi, float& lo, float xh, float xl) {
    const float s = hi + xh;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (xh - bb);
    const float l = lo + xl + e;
    const float h = s + l;
    lo = l - (h - s);
    hi = h;
}

// 10 warps: a sub-partition hosts up to 3 of them in its 16K registers, so at
// most 168 registers per thread
__global__ void __maxnreg__(168)
ozaki_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzParams p) {
    extern __shared__ unsigned char oz_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(oz_raw) + 1023) &
                                                         ~uintptr_t(1023));
    unsigned char* sB = sm;                        // [slice][atom] 64 x 128 B
    unsigned char* sA = sm + OzSmem::B_BYTES;      // [stage][atom] 128 x 128 B
    uint64_t* bar = reinterpret_cast<uint64_t*>(sA + 2 * OzSmem::A_STAGE);
    uint64_t* bfull = bar + 0;
    uint64_t* bfree = bar + 1;
    uint64_t* afull = bar + 2;   // [2]
    uint64_t* aempty = bar + 4;  // [2]
    uint64_t* tfull = bar + 6;
    uint64_t* tempty = bar + 7;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 8);
    __shared__ int s_bi, s_bc, s_ai, s_ac;  // B chunks / A stages issued and consumed

    // tile order: groups of GM tile rows, column-major inside a group, so that
    // the CTAs resident at one time share few distinct A and B rows (one wave
    // of 152 covers about 8 x 19 tiles, whose operands L2 holds as the CTAs
    // step through K together)
    constexpr int GM = 8;
    const int t = blockIdx.x, grp_size = GM * p.nt, first_m = (t / grp_size) * GM;
    const int gm = (p.mt - first_m) < GM ? (p.mt - first_m) : GM;
    const int m0 = (first_m + (t % grp_size) % gm) * OM, n0 = ((t % grp_size) / gm) * ON;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (p.lower && n0 >= m0 + OM) return;  // whole CTA, before any barrier or TMEM use
    const int S = p.s;

    if (threadIdx.x == 0) {
        mbar_init(bfull, 1);
        mbar_init(bfree, 1);
        mbar_init(&afull[0], 1);
        mbar_init(&afull[1], 1);
        mbar_init(&aempty[0], 1);
        mbar_init(&aempty[1], 1);
        mbar_init(tfull, 1);
        mbar_init(tempty, OEPI);
        fence_mbar_init();
        fence_proxy_async_smem();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
        s_bi = s_bc = s_ai = s_ac = 0;
    }
    if (warp == 8) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nch = p.nchunks;

    if (warp == 8) {
        if (lane == 0) {
            // ---- TMA producer
            bool ok = true;
            int bi = 0, ai = 0;
            for (int c = 0; c < nch && ok; c++) {
                if (!(ok = mbar_wait(bfree, ((uint32_t)c & 1u) ^ 1u, p.status))) break;
                const int na = min(2, p.katoms - 2 * c);  // atoms in this chunk
                mbar_arrive_expect_tx(bfull, (uint32_t)(S * na) * OzSmem::B_ATOM);
                for (int j = 0; j < S; j++)
                    for (int a = 0; a < na; a++)
                        tma_load_2d(sB + (j * 2 + a) * OzSmem::B_ATOM, &tmB, bfull, c * OKC + a * 64, j * p.Np + n0);
                bi++;
                for (int i = 0; i < S; i++) {
                    const int it = c * S + i, s = it & 1;
                    if (!(ok = mbar_wait(&aempty[s], ((uint32_t)(it >> 1) & 1u) ^ 1u, p.status))) break;
                    mbar_arrive_expect_tx(&afull[s], (uint32_t)na * OzSmem::A_ATOM);
                    for (int a = 0; a < na; a++)
                        tma_load_2d(sA + s * OzSmem::A_STAGE + a * OzSmem::A_ATOM, &tmA, &afull[s],
                                    c * OKC + a * 64, i * p.Mp + m0);
                    ai++;
                }
            }
            s_bi = bi;
            s_ai = ai;
        }
    } else if (warp == 9) {
        if (lane == 0) {
            // ---- MMA issuer: level L accumulates in TMEM columns [64 L, 64 L + 64)
            constexpr uint32_t idesc = umma_idesc_bf16(OM, ON);
            bool ok = true;
            int bc = 0, ac = 0;
            for (int c = 0; c < nch && ok; c++) {
                const bool first = (c & 1) == 0;  // first chunk of a 256-wide K group
                if (first) {
                    if (!(ok = mbar_wait(tempty, ((uint32_t)(c >> 1) & 1u) ^ 1u, p.status))) break;
                    tc_fence_after();
                }
                if (!(ok = mbar_wait(bfull, (uint32_t)c & 1u, p.status))) break;
                bc++;
                tc_fence_after();
                const int nkk = 4 * min(2, p.katoms - 2 * c);  // 16-wide K steps in this chunk
                for (int i = 0; i < S; i++) {
                    const int it = c * S + i, s = it & 1;
                    if (!(ok = mbar_wait(&afull[s], (uint32_t)(it >> 1) & 1u, p.status))) break;
                    ac++;
                    tc_fence_after();
                    for (int j = 0; i + j < S; j++) {
                        const uint32_t dcol = tmem + (uint32_t)((i + j) * ON);
#pragma unroll
                        for (int kk = 0; kk < OKC / 16; kk++) {
                            if (kk >= nkk) break;
                            const int a = kk >> 2, k4 = kk & 3;
                            const uint64_t ad =
                                umma_desc_sw128(smem_u32(sA + s * OzSmem::A_STAGE + a * OzSmem::A_ATOM)) + 2 * k4;
                            const uint64_t bd = umma_desc_sw128(smem_u32(sB + (j * 2 + a) * OzSmem::B_ATOM)) + 2 * k4;
                            // level L is first written by the pair (0, L) at kk = 0 of a group
                            umma_bf16(dcol, ad, bd, idesc, (!first || i > 0 || kk > 0) ? 1u : 0u);
                        }
                    }
                    umma_commit(&aempty[s]);
                }
                umma_commit(bfree);
                if (!first || c == nch - 1) umma_commit(tfull);
            }
            s_bc = bc;
            s_ac = ac;
        }
    } else {
        // ---- epilogue warps 0-7: row m0 + 32 (w & 3) + lane, columns n0 + 32 (w >> 2) + [0, 32)
        constexpr int EC = ON / 2;
        const int quad = warp & 3, half = warp >> 2;
        float ah[EC], al[EC];
#pragma unroll
        for (int q = 0; q < EC; q++) { ah[q] = 0.f; al[q] = 0.f; }
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * EC);
        bool ok = true;
        const int ngroups = (nch + 1) / 2;
        for (int grp = 0; grp < ngroups; grp++) {
            ok = mbar_wait(tfull, (uint32_t)grp & 1u, p.status);
            tc_fence_after();
            if (!ok) break;
#pragma unroll
            for (int g = 0; g < EC / 16; g++) {
                float sh[16], sl[16];
#pragma unroll
                for (int q = 0; q < 16; q++) { sh[q] = 0.f; sl[q] = 0.f; }
                // levels from the smallest up, three TMEM loads in flight per wait
#pragma unroll 1
                for (int top = S - 1; top >= 0; top -= 3) {
                    uint32_t v0[16], v1[16], v2[16];
                    const uint32_t col = lane_base + (uint32_t)(g * 16);
                    tmem_ld16_async(col + (uint32_t)(top * ON), v0);
                    if (top >= 1) tmem_ld16_async(col + (uint32_t)((top - 1) * ON), v1);
                    if (top >= 2) tmem_ld16_async(col + (uint32_t)((top - 2) * ON), v2);
                    tmem_wait_ld16(v0);
                    tmem_after_wait16(v1);
                    tmem_after_wait16(v2);
                    float sc = __int_as_float((127 - 7 * top) << 23);  // 2^-7L
#pragma unroll
                    for (int q = 0; q < 16; q++) df_add(sh[q], sl[q], __uint_as_float(v0[q]) * sc);
                    if (top >= 1) {
                        sc *= 128.f;
#pragma unroll
                        for (int q = 0; q < 16; q++) df_add(sh[q], sl[q], __uint_as_float(v1[q]) * sc);
                    }
                    if (top >= 2) {
                        sc *= 128.f;
#pragma unroll
                        for (int q = 0; q < 16; q++) df_add(sh[q], sl[q], __uint_as_float(v2[q]) * sc);
                    }
                }
#pragma unroll
                for (int q = 0; q < 16; q++) df_add_df(ah[g * 16 + q], al[g * 16 + q], sh[q], sl[q]);
            }
            tc_fence_before();
            mbar_arrive(tempty);
        }
        const int row = m0 + quad * 32 + lane;
        if (ok && row < p.M) {
            const int er = p.ea[row];
#pragma unroll
            for (int q = 0; q < EC; q++) {
                const int col = n0 + half * EC + q;
                if (col >= p.N) continue;
                const double val = ldexp((double)ah[q] + (double)al[q], er + p.eb[col] - 14);
                double* dst = p.C + (long long)col * p.ldc + row;
                *dst = (p.beta == 0.0) ? p.alpha * val : fma(p.beta, *dst, p.alpha * val);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    // after a timeout, let loads that were issued but never consumed land
    // before the shared memory is released (capped as well)
    if (threadIdx.x == 256) {
        for (int c = s_bc; c < s_bi; c++) mbar_wait(bfull, (uint32_t)c & 1u, p.status, 1u << 16);
        for (int it = s_ac; it < s_ai; it++) mbar_wait(&afull[it & 1], (uint32_t)(it >> 1) & 1u, p.status, 1u << 16);
    }
    __syncthreads();
    if (warp == 8) tmem_dealloc(tmem, 512);
}

// Row exponents when rows are contiguous in memory (sr == 1): one thread per
// row walks k, so a warp reads 32 consecutive rows at each k.
__global__ void oz_exp_cols_kernel(int rows, int K, const double* __restrict__ src, long long sk,
                                   int* __restrict__ e) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        double m = 0.0;
        for (int k = 0; k < K; k++) m = fmax(m, fabs(src[r + (long long)k * sk]));
        int ex = 0;
        if (m > 0.0) frexp(m, &ex);
        e[r] = ex;
    }
}

// Digit slices when rows are contiguous (sr == 1): a 32 x 32 tile is read
// along rows and written along k through shared memory.
__global__ void oz_split_cols_kernel(int rows, int K, int Rp, int Kp, const double* __restrict__ src, long long sk,
                                     double sgn, const int* __restrict__ e, __nv_bfloat16* __restrict__ dst) {
    __shared__ double tile[32][33];
    const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int kk = ty; kk < 32; kk += 8) {
        const int r = r0 + tx, k = k0 + kk;
        tile[kk][tx] = (r < rows && k < K) ? sgn * src[r + (long long)k * sk] : 0.0;
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {
        const int r = r0 + rr, k = k0 + tx;
        if (r >= Rp || k >= Kp) continue;
        float d[8];
        oz_digits(tile[tx][rr], (r < rows) ? e[r] : 0, d);
#pragma unroll
        for (int i = 0; i < SL; i++) dst[((long long)i * Rp + r) * Kp + k] = __float2bfloat16_rn(d[i]);
    }
}

// Row exponents: e_r = smallest e with max_k |x_rk| < 2^e (0 for a zero row).
// Element (r, k) of the operand is sgn * src[r * sr + k * sk].
// skew != 0: the operand is the skew matrix whose strict lower triangle is
// stored column-major in src with leading dimension sk: (r, k) ->
// src[r + k sk] (r > k), -src[k + r sk] (r < k), 0 (r == k).
SK_DEV double oz_elem(const double* __restrict__ src, long long sr, long long sk, int skew, int r, int k) {
    if (!skew) return src[(long long)r * sr + (long long)k * sk];
    if (r > k) return src[(long long)r + (long long)k * sk];
    if (r < k) return -src[(long long)k + (long long)r * sk];
    return 0.0;
}

__global__ void oz_exp_kernel(int rows, int K, const double* __restrict__ src, long long sr, long long sk,
                              int* __restrict__ e, int skew) {
    __shared__ double red[32];
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        double m = 0.0;
        for (int k = threadIdx.x; k < K; k += blockDim.x) m = fmax(m, fabs(oz_elem(src, sr, sk, skew, r, k)));
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            double mm = 0.0;
            for (int w = 0; w < (int)(blockDim.x + 31) / 32; w++) mm = fmax(mm, red[w]);
            int ex = 0;
            if (mm > 0.0) {
                frexp(mm, &ex);  // mm = f 2^ex, f in [0.5, 1): mm < 2^ex
            }
            e[r] = ex;
        }
        __syncthreads();
    }
}

// Digit slices: plane i holds rows [i Rp, i Rp + rows) of a (SL Rp) x Kp
// row-major BF16 array; padding rows / columns are zero.
__global__ void oz_split_kernel(int rows, int K, int Rp, int Kp, const double* __restrict__ src, long long sr,
                                long long sk, double sgn, const int* __restrict__ e, __nv_bfloat16* __restrict__ dst,
                                int skew) {
    const long long total = (long long)Rp * Kp;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t % Kp), r = (int)(t / Kp);
        const double x = (r < rows && k < K) ? sgn * oz_elem(src, sr, sk, skew, r, k) : 0.0;
        float d[8];
        oz_digits(x, (r < rows) ? e[r] : 0, d);
#pragma unroll
        for (int i = 0; i < SL; i++) dst[((long long)i * Rp + r) * Kp + k] = __float2bfloat16_rn(d[i]);
    }
}

// Row maxima of the skew matrix S of a strict lower triangle (W, ld): entry
// W(i, j), i > j, is S(i, j) and -S(j, i), so it bounds rows i and j.  32 x 32
// tiles of the lower triangle, read along i; per-tile row and column maxima go
// to rowmax (as ordered bit patterns of non-negative doubles) with atomicMax.
__global__ void oz_skew_rowmax_kernel(int n, const double* __restrict__ W, long long ld,
                                      unsigned long long* __restrict__ rowmax) {
    __shared__ double tile[32][33];
    const int bi = blockIdx.x, bj = blockIdx.y;
    if (bi < bj) return;
    const int i0 = bi * 32, j0 = bj * 32, tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int jj = ty; jj < 32; jj += 8) {
        const int i = i0 + tx, j = j0 + jj;
        tile[jj][tx] = (i < n && j < n && i > j) ? fabs(W[i + (long long)j * ld]) : 0.0;
    }
    __syncthreads();
    if (ty == 0) {
        double rm = 0.0, cm = 0.0;  // row i0+tx over the tile's columns; column j0+tx over its rows
        for (int jj = 0; jj < 32; jj++) rm = fmax(rm, tile[jj][tx]);
        for (int ii = 0; ii < 32; ii++) cm = fmax(cm, tile[tx][ii]);
        if (i0 + tx < n && rm > 0.0) atomicMax(rowmax + i0 + tx, (unsigned long long)__double_as_longlong(rm));
        if (j0 + tx < n && cm > 0.0) atomicMax(rowmax + j0 + tx, (unsigned long long)__double_as_longlong(cm));
    }
}

__global__ void oz_exp_from_max_kernel(int rows, const unsigned long long* __restrict__ rowmax, int* __restrict__ e) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        const double m = __longlong_as_double((long long)rowmax[r]);
        int ex = 0;
        if (m > 0.0) frexp(m, &ex);
        e[r] = ex;
    }
}

// Digit slices of the skew S: tiles below the diagonal are read along rows of
// W and transposed through shared memory, tiles above read -W(k, r) along k.
__global__ void oz_split_skew_kernel(int rows, int Rp, int Kp, const double* __restrict__ W, long long ld,
                                     const int* __restrict__ e, __nv_bfloat16* __restrict__ dst) {
    __shared__ double tile[32][33];
    const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    if (r0 >= k0 + 32) {
        // strictly lower tile: S(r, k) = W(r, k), contiguous in r
        for (int kk = ty; kk < 32; kk += 8) {
            const int r = r0 + tx, k = k0 + kk;
            tile[kk][tx] = (r < rows && k < rows) ? W[r + (long long)k * ld] : 0.0;
        }
    } else if (r0 + 32 <= k0) {
        // strictly upper tile: S(r, k) = -W(k, r), contiguous in k
        for (int rr = ty; rr < 32; rr += 8) {
            const int r = r0 + rr, k = k0 + tx;
            tile[tx][rr] = (r < rows && k < rows) ? -W[k + (long long)r * ld] : 0.0;
        }
    } else {
        for (int kk = ty; kk < 32; kk += 8) {
            const int r = r0 + tx, k = k0 + kk;
            double v = 0.0;
            if (r < rows && k < rows) v = (r > k) ? W[r + (long long)k * ld] : (r < k ? -W[k + (long long)r * ld] : 0.0);
            tile[kk][tx] = v;
        }
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {
        const int r = r0 + rr, k = k0 + tx;
        if (r >= Rp || k >= Kp) continue;
        float d[8];
        oz_digits((r < rows) ? tile[tx][rr] : 0.0, (r < rows) ? e[r] : 0, d);
#pragma unroll
        for (int i = 0; i < SL; i++) dst[((long long)i * Rp + r) * Kp + k] = __float2bfloat16_rn(d[i]);
    }
}

inline long long rup(long long x, long long a) { return (x + a - 1) / a * a; }
inline int gridn(long long total) {
    long long g = (total + 255) / 256;
    return (int)(g > 16384 ? 16384 : (g < 1 ? 1 : g));
}

}  // namespace

size_t ozaki_gemm_ws(int M, int N, int K) {
    const long long Kp = rup(K > 0 ? K : 1, OKA), Mp = rup(M > 0 ? M : 1, OM), Np = rup(N > 0 ? N : 1, ON);
    return align_up((size_t)(SL * Mp * Kp * 2)) + align_up((size_t)(SL * Np * Kp * 2)) + align_up(sizeof(int) * Mp) +
           align_up(sizeof(int) * Np) + align_up(sizeof(unsigned long long) * Mp) + 256;
}

// C = alpha * (sa A)(sb B)^T + beta C, A[i,k] = A[i*a_rs + k*a_ks], B[j,k] = B[j*b_rs + k*b_ks].
int ozaki_gemm(cudaStream_t st, int M, int N, int K, double alpha, const double* A, long long a_rs, long long a_ks,
               double sa, const double* B, long long b_rs, long long b_ks, double sb, double beta, double* C,
               long long ldc, void* ws, size_t ws_bytes, int* status, int a_skew, int slices, int lower) {
    if (M <= 0 || N <= 0) return 0;
    if (K <= 0 || slices < 1 || slices > SL) return SKEW_ERR_UNSUPPORTED;
    const long long Kp = rup(K, OKA), Mp = rup(M, OM), Np = rup(N, ON);
    Carve cv(ws, ws_bytes);
    __nv_bfloat16* Ad = cv.take<__nv_bfloat16>((size_t)(SL * Mp * Kp));
    __nv_bfloat16* Bd = cv.take<__nv_bfloat16>((size_t)(SL * Np * Kp));
    int* ea = cv.take<int>((size_t)Mp);
    int* eb = cv.take<int>((size_t)Np);
    unsigned long long* skew_max = cv.take<unsigned long long>((size_t)Mp);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    auto split = [&](int rows, long long Rp, const double* src, long long rs, long long ks, double sg, int* e,
                     __nv_bfloat16* d, int skew) {
        if (skew) {
            cudaMemsetAsync(skew_max, 0, sizeof(unsigned long long) * (size_t)Rp, st);
            const unsigned T = (unsigned)((rows + 31) / 32);
            oz_skew_rowmax_kernel<<<dim3(T, T), dim3(32, 8), 0, st>>>(rows, src, ks, skew_max);
            oz_exp_from_max_kernel<<<(rows + 255) / 256, 256, 0, st>>>(rows, skew_max, e);
            oz_split_skew_kernel<<<dim3((unsigned)((Rp + 31) / 32), (unsigned)((Kp + 31) / 32)), dim3(32, 8), 0, st>>>(
                rows, (int)Rp, (int)Kp, src, ks, e, d);
            count_launch(1);
        } else if (rs == 1 && ks != 1) {
            oz_exp_cols_kernel<<<(rows + 127) / 128, 128, 0, st>>>(rows, K, src, ks, e);
            oz_split_cols_kernel<<<dim3((unsigned)((Rp + 31) / 32), (unsigned)((Kp + 31) / 32)), dim3(32, 8), 0, st>>>(
                rows, K, (int)Rp, (int)Kp, src, ks, sg, e, d);
        } else {
            oz_exp_kernel<<<(int)(rows < 16384 ? rows : 16384), 256, 0, st>>>(rows, K, src, rs, ks, e, skew);
            oz_split_kernel<<<gridn(Rp * Kp), 256, 0, st>>>(rows, K, (int)Rp, (int)Kp, src, rs, ks, sg, e, d, skew);
        }
        count_launch(2);
    };
    split(M, Mp, A, a_rs, a_ks, sa, ea, Ad, a_skew);
    if (!a_skew && B == A && b_rs == a_rs && b_ks == a_ks && sb == sa && N == M && Np == Mp) {
        // same operand (a Gram matrix): reuse its slices
        Bd = Ad;
        eb = ea;
    } else {
        split(N, Np, B, b_rs, b_ks, sb, eb, Bd, 0);
    }
    CUtensorMap ta, tb;
    if (!make_tmap_bf16(&ta, Ad, (uint64_t)Kp, (uint64_t)(SL * Mp), (uint64_t)Kp, OM)) return SKEW_ERR_UNSUPPORTED;
    if (!make_tmap_bf16(&tb, Bd, (uint64_t)Kp, (uint64_t)(SL * Np), (uint64_t)Kp, ON)) return SKEW_ERR_UNSUPPORTED;
    OzParams p{};
    p.M = M;
    p.N = N;
    p.katoms = (int)(Kp / OKA);
    p.nchunks = (p.katoms + 1) / 2;
    p.Mp = (int)Mp;
    p.Np = (int)Np;
    p.ea = ea;
    p.eb = eb;
    p.alpha = alpha;
    p.beta = beta;
    p.C = C;
    p.ldc = ldc;
    p.status = status;
    p.s = slices;
    p.lower = lower;
    const size_t smem = OzSmem::bytes();
    cudaFuncSetAttribute(ozaki_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    p.mt = (int)(Mp / OM);
    p.nt = (int)(Np / ON);
    // algorithmic work: the kept slice pairs over the outputs written
    const double pairs = slices * (slices + 1) / 2.0;
    const double outs = lower ? lower_count(M, N) : (double)M * N;
    const int kt = kt_begin(st);
    ozaki_gemm_kernel<<<(unsigned)(p.mt * p.nt), OT, smem, st>>>(ta, tb, p);
    kt_end(st, kt, g_kt_ozaki_kind, 2.0 * pairs * outs * K);
    count_launch();
    return cuda_ok(cudaGetLastError());
}

}  // namespace sk

extern "C" size_t skew_gemm_f64acc_ws(int M, int N, int K) { return sk::ozaki_gemm_ws(M, N, K); }

extern "C" int skew_gemm_f64acc(int M, int N, int K, double alpha, const double* A, long long a_rs, long long a_ks,
                                const double* B, long long b_rs, long long b_ks, double beta, double* C, int ldc,
                                void* ws, size_t ws_bytes, int* d_status, void* stream) {
    if (M < 0) return -1;
    if (N < 0) return -2;
    if (K < 1) return -3;
    if (ldc < (M > 1 ? M : 1)) return -13;
    return sk::ozaki_gemm(static_cast<cudaStream_t>(stream), M, N, K, alpha, A, a_rs, a_ks, 1.0, B, b_rs, b_ks, 1.0,
                          beta, C, ldc, ws, ws_bytes, d_status, 0, 8, 0);
}

extern "C" int skew_gemm_f64acc_ex(int M, int N, int K, double alpha, const double* A, long long a_rs, long long a_ks,
                                   const double* B, long long b_rs, long long b_ks, double beta, double* C, int ldc,
                                   int slices, int lower, void* ws, size_t ws_bytes, int* d_status, void* stream) {
    if (M < 0) return -1;
    if (N < 0) return -2;
    if (K < 1) return -3;
    if (ldc < (M > 1 ? M : 1)) return -13;
    if (slices < 1 || slices > 8) return -14;
    if (lower != 0 && lower != 1) return -15;
    return sk::ozaki_gemm(static_cast<cudaStream_t>(stream), M, N, K, alpha, A, a_rs, a_ks, 1.0, B, b_rs, b_ks, 1.0,
                          beta, C, ldc, ws, ws_bytes, d_status, 0, slices, lower);
}
