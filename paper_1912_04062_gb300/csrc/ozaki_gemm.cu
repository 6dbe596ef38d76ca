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
// taken over K groups of 512: level 0 is a sum of 512 products of size
// <= 2^14, level L >= 1 of 512 (L + 3) 2^12-sized terms (two pairs with a
// leading digit, |d_0| <= 128), so levels 0..5 stay at or below 2^24 and are
// exact in FP32; levels 6 and 7 may round by one unit of their own level,
// below 2^-56 of |a_r|max |b_c|max per group.  After each group the level
// accumulators (s x 64 TMEM columns) are folded into a double-float (two FP32)
// running sum per output, which carries about 48 bits.
//
// Kernel: 128 x 64 output tile per CTA, 320 threads: warps 0-7 drain TMEM
// (warp w: lanes 32 (w & 3).. = rows, columns 32 (w >> 2)..) and accumulate;
// warp 8 issues TMA loads, warp 9 issues the MMAs.  K advances in chunks of 64
// (one 128-byte swizzle atom).  All B digit slices of a chunk sit in one of two
// buffers, so the next chunk's B loads while the current one is multiplied; A
// digit slices stream through a ring of NA one-slice stages.  Within a chunk,
// pass i multiplies A slice i with B slices 0 .. S-1-i as one wide MMA (B
// slices adjacent in shared memory, their levels adjacent in TMEM).
// TMEM holds one level group (8 chunks = 512 of K), so the MMAs of the next
// group start once the epilogue has drained it.
// With `lower` set, tiles wholly above the diagonal (every column index above
// every row index) are skipped: for symmetric or skew results whose upper
// triangle is not read.  Split K (for small outputs over a long K): CTA
// (tile, z) takes chunks [z kz, (z + 1) kz) and stores its unscaled-by-alpha
// partial tile; a reduction kernel sums the partials in a fixed order.
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
constexpr int OKA = 64;      // K per chunk = one 64-wide swizzle atom; K is padded to a multiple of it
constexpr int NA = 6;        // A stages (one digit slice of one chunk each)
constexpr int GRP = 8;       // chunks per level group (512 of K)
constexpr int SL = 8;        // digit slices per operand
constexpr int OT = 320;      // threads per CTA: 8 epilogue warps, TMA warp, MMA warp
constexpr int OEPI = 256;    // epilogue threads

struct OzParams {
    int M, N, nchunks;       // nchunks: 64-wide K chunks
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
    int kz;                  // split K: chunks per split (blockIdx.y), 0 = whole K
    double* part;            // split K: partial tiles, [split][N][M]
    int akoff, bkoff;        // K offsets of views into larger splits (elements)
    const int* skip;         // device flag: nonzero -> the launch does nothing (may be null)
    const int* s_dyn;        // device slice count overriding s (may be null)
};

struct OzSmem {
    static constexpr uint32_t B_ATOM = ON * 128;       // 64 rows x 128 B: one B slice of a chunk
    static constexpr uint32_t A_ATOM = OM * 128;       // 128 rows x 128 B: one A slice of a chunk
    static constexpr uint32_t B_SET = SL * B_ATOM;     // all B slices of a chunk (64 KB)
    static constexpr uint32_t B_BYTES = 2 * B_SET;     // two chunks in flight
    static constexpr uint32_t A_BYTES = NA * A_ATOM;   // 96 KB
    static constexpr int NBAR = 4 + 2 * NA + 2;        // bfull/bfree per set, afull/aempty per stage, tfull, tempty
    static constexpr size_t bytes() { return 1024 + B_BYTES + A_BYTES + 8 * NBAR + 16; }
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
        d[i] = (float)(int)q;  // |q| <= 128: a 32-bit conversion
    }
}

// Sign flips and magnitudes of doubles as integer operations on their bits
// (the split kernels touch every element; GB300's FP64 pipe is 1/64 rate).
SK_DEV double oz_neg_if(double x, bool neg) {
    return __longlong_as_double(__double_as_longlong(x) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
}
// |x| as an ordered bit pattern: for non-negative doubles the integer order of
// the patterns is the numeric order
SK_DEV unsigned long long oz_absbits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFULL;
}
SK_DEV unsigned long long oz_umax(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

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

// x 2^sh as a double, exactly, for a normal or zero float x: the exponent is
// moved with integer operations (GB300 runs FP64 at 1/64 of the FP32 rate, and
// these scalings are an epilogue's bulk); results outside the normal double
// range take ldexp.
SK_DEV double f2d_scaled(float x, int sh) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t ef = (u >> 23) & 0xFFu;
    if ((u & 0x7FFFFFFFu) == 0u) return 0.0;
    const int E = (int)ef - 127 + 1023 + sh;
    if (ef == 0u || E <= 0 || E >= 2047) return ldexp((double)x, sh);
    const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)E << 52) |
                                    ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}

// (hi + lo) 2^sh for a double-float pair (|lo| <= ulp(hi) / 2): the sum of the
// two exact scaled parts spans at most 49 bits, so it is exact too.
SK_DEV double df_scaled(float hi, float lo, int sh) { return f2d_scaled(hi, sh) + f2d_scaled(lo, sh); }

// 10 warps: a sub-partition hosts up to 3 of them in its 16K registers, so at
// most 168 registers per thread.  ONE: one item per CTA (grid = items), for
// long K, where the per-item epilogue is negligible; otherwise the CTAs are
// persistent and walk the items.
template <bool ONE>
__global__ void __maxnreg__(168)
ozaki_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzParams p) {
    extern __shared__ unsigned char oz_raw[];
    // a skipped launch returns before any barrier, copy or tensor-memory use
    if (p.skip && *p.skip) return;
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(oz_raw) + 1023) &
                                                         ~uintptr_t(1023));
    unsigned char* sB = sm;                        // [set][slice] 64 x 128 B
    unsigned char* sA = sm + OzSmem::B_BYTES;      // [stage] 128 x 128 B
    uint64_t* bar = reinterpret_cast<uint64_t*>(sA + OzSmem::A_BYTES);
    uint64_t* bfull = bar;             // [2]
    uint64_t* bfree = bar + 2;         // [2]
    uint64_t* afull = bar + 4;         // [NA]
    uint64_t* aempty = bar + 4 + NA;   // [NA]
    uint64_t* tfull = bar + 4 + 2 * NA;
    uint64_t* tempty = tfull + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 1);
    // loads issued (producer) and consumed (MMA): B in chunks, A in slices
    __shared__ int s_bi, s_bc, s_ai, s_ac;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = p.s_dyn ? *p.s_dyn : p.s;
    const int nz = p.kz ? (p.nchunks + p.kz - 1) / p.kz : 1;
    const int nitems = p.mt * p.nt * nz;  // below 2^31 for every supported size
    // Work item it = (tile, K range z), tile = it / nz.  Tile order: groups of
    // GM tile rows, column-major inside a group, so that the items in flight
    // at one time (one per CTA) share few distinct A and B rows, whose
    // operands L2 holds as the CTAs step through K together.  Every role
    // walks the same items and skips the same ones (tiles wholly above the
    // diagonal with `lower`).
    constexpr int GM = 8;
    auto geom = [&](int it, int& m0, int& n0, int& z, int& c_off, int& nch) -> bool {
        const int t = it / nz;
        z = it - t * nz;
        const int grp_size = GM * p.nt, first_m = (t / grp_size) * GM;
        const int gm = (p.mt - first_m) < GM ? (p.mt - first_m) : GM;
        m0 = (first_m + (t % grp_size) % gm) * OM;
        n0 = ((t % grp_size) / gm) * ON;
        c_off = p.kz ? z * p.kz : 0;
        nch = p.kz ? min(p.kz, p.nchunks - c_off) : p.nchunks;
        return !(p.lower && n0 >= m0 + OM);
    };

    if (threadIdx.x == 0) {
        for (int q = 0; q < 2; q++) {
            mbar_init(&bfull[q], 1);
            mbar_init(&bfree[q], 1);
        }
        for (int q = 0; q < NA; q++) {
            mbar_init(&afull[q], 1);
            mbar_init(&aempty[q], 1);
        }
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

    if (warp == 8) {
        if (lane == 0) {
            // ---- TMA producer: per chunk, its B slices into buffer bi & 1 (free
            // once the chunk two before it is multiplied), then its A slices
            // (each waits for its ring stage); bi and ai run across items
            bool ok = true;
            int ai = 0, bi = 0;
            for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
                int m0, n0, z, c_off, nch;
                if (!geom(it, m0, n0, z, c_off, nch)) continue;
                for (int c = 0; c < nch && ok; c++) {
                    const int q = bi & 1;
                    if (!(ok = mbar_wait(&bfree[q], ((uint32_t)(bi >> 1) & 1u) ^ 1u, p.status))) break;
                    mbar_arrive_expect_tx(&bfull[q], (uint32_t)S * OzSmem::B_ATOM);
                    for (int j = 0; j < S; j++)
                        tma_load_2d(sB + q * OzSmem::B_SET + j * OzSmem::B_ATOM, &tmB, &bfull[q],
                                    p.bkoff + (c_off + c) * OKA, j * p.Np + n0);
                    bi++;
                    for (int i = 0; i < S; i++) {
                        const int st = ai % NA;
                        if (!(ok = mbar_wait(&aempty[st], ((uint32_t)(ai / NA) & 1u) ^ 1u, p.status))) break;
                        mbar_arrive_expect_tx(&afull[st], OzSmem::A_ATOM);
                        tma_load_2d(sA + st * OzSmem::A_ATOM, &tmA, &afull[st], p.akoff + (c_off + c) * OKA,
                                    i * p.Mp + m0);
                        ai++;
                    }
                }
                if (ONE) break;
            }
            s_bi = bi;
            s_ai = ai;
        }
    } else if (warp == 9) {
        if (lane == 0) {
            // ---- MMA issuer: level L accumulates in TMEM columns [64 L, 64 L + 64).
            // Pass i multiplies A slice i with B slices 0 .. S-1-i; those B slices
            // are consecutive 64-row blocks of one buffer and their levels
            // i .. S-1 consecutive TMEM columns, so the pass is one MMA of width
            // N = 64 (S - i) (two when wider than 256).  A level group starts
            // once the epilogue has drained the previous one (of this item or
            // the one before).
            bool ok = true;
            int ac = 0, bc = 0, gc = 0;
            for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
                int m0, n0, z, c_off, nch;
                if (!geom(it, m0, n0, z, c_off, nch)) continue;
                for (int c = 0; c < nch && ok; c++) {
                    const bool first = (c % GRP) == 0;  // first chunk of a level group
                    if (first) {
                        if (!(ok = mbar_wait(tempty, ((uint32_t)gc & 1u) ^ 1u, p.status))) break;
                        tc_fence_after();
                    }
                    const int q = bc & 1;
                    if (!(ok = mbar_wait(&bfull[q], (uint32_t)(bc >> 1) & 1u, p.status))) break;
                    tc_fence_after();
                    for (int i = 0; i < S; i++) {
                        const int st = ac % NA;
                        if (!(ok = mbar_wait(&afull[st], (uint32_t)(ac / NA) & 1u, p.status))) break;
                        ac++;
                        tc_fence_after();
                        const uint64_t ad0 = umma_desc_sw128(smem_u32(sA + st * OzSmem::A_ATOM));
                        const int nj = S - i, n1 = nj < 4 ? nj : 4;
                        const uint64_t b0 = umma_desc_sw128(smem_u32(sB + q * OzSmem::B_SET));
                        const uint64_t b4 = umma_desc_sw128(smem_u32(sB + q * OzSmem::B_SET + 4 * OzSmem::B_ATOM));
                        const uint32_t d0 = tmem + (uint32_t)(i * ON), d4 = tmem + (uint32_t)((i + 4) * ON);
#pragma unroll
                        for (int kk = 0; kk < OKA / 16; kk++) {
                            // every level is first written by pass 0 at kk = 0 of a group
                            const uint32_t acc = (!first || i > 0 || kk > 0) ? 1u : 0u;
                            umma_bf16(d0, ad0 + 2 * kk, b0 + 2 * kk, umma_idesc_bf16(OM, ON * n1), acc);
                            if (nj > 4)
                                umma_bf16(d4, ad0 + 2 * kk, b4 + 2 * kk, umma_idesc_bf16(OM, ON * (nj - 4)), acc);
                        }
                        umma_commit(&aempty[st]);
                    }
                    if (!ok) break;
                    bc++;
                    umma_commit(&bfree[q]);
                    if (c % GRP == GRP - 1 || c == nch - 1) {
                        umma_commit(tfull);
                        gc++;
                    }
                }
                if (ONE) break;
            }
            s_bc = bc;
            s_ac = ac;
        }
    } else {
        // ---- epilogue warps 0-7: row m0 + 32 (w & 3) + lane, columns n0 + 32 (w >> 2) + [0, 32).
        // TMEM is released after the last level fold of an item, so the FP64
        // conversion and the update of C overlap the next item's MMAs.
        constexpr int EC = ON / 2;
        const int quad = warp & 3, half = warp >> 2;
        bool ok = true;
        int gc = 0;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * EC);
        for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
            int ngroups;
            {
                int m0, n0, z, c_off, nch;
                if (!geom(it, m0, n0, z, c_off, nch)) continue;
                ngroups = (nch + GRP - 1) / GRP;
            }
            float ah[EC], al[EC];
#pragma unroll
            for (int q = 0; q < EC; q++) { ah[q] = 0.f; al[q] = 0.f; }
            for (int grp = 0; grp < ngroups; grp++) {
                ok = mbar_wait(tfull, (uint32_t)gc & 1u, p.status);
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
                gc++;
            }
            if (!ok) break;
            int m0, n0, z, c_off, nch;  // recomputed: not live across the drain
            geom(it, m0, n0, z, c_off, nch);
            const int row = m0 + quad * 32 + lane;
            if (row < p.M) {
                const int er = p.ea[row] - 14;
                if (p.part) {
#pragma unroll
                    for (int q = 0; q < EC; q++) {
                        const int col = n0 + half * EC + q;
                        if (col < p.N)
                            p.part[((long long)z * p.N + col) * p.M + row] = df_scaled(ah[q], al[q], er + p.eb[col]);
                    }
                } else {
                    // alpha = +-1 and beta in {0, 1} (every internal use) cost one
                    // or two FP64 additions per output; the old values are loaded
                    // 16 at a time ahead of their use
                    const bool a1 = p.alpha == 1.0, am1 = p.alpha == -1.0;
                    const bool b0 = p.beta == 0.0, b1 = p.beta == 1.0;
#pragma unroll
                    for (int hq = 0; hq < EC; hq += 16) {
                        double old[16];
#pragma unroll
                        for (int q = 0; q < 16; q++) {
                            const int col = n0 + half * EC + hq + q;
                            old[q] = (!b0 && col < p.N) ? p.C[(long long)col * p.ldc + row] : 0.0;
                        }
#pragma unroll
                        for (int q = 0; q < 16; q++) {
                            const int col = n0 + half * EC + hq + q;
                            if (col >= p.N) continue;
                            const double val = df_scaled(ah[hq + q], al[hq + q], er + p.eb[col]);
                            const double av = a1 ? val : (am1 ? -val : p.alpha * val);
                            p.C[(long long)col * p.ldc + row] = b0 ? av : (b1 ? old[q] + av : fma(p.beta, old[q], av));
                        }
                    }
                }
            }
            if (ONE) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    // after a timeout, let loads that were issued but never consumed land
    // before the shared memory is released (capped as well)
    if (threadIdx.x == 256) {
        for (int c = s_bc; c < s_bi; c++) mbar_wait(&bfull[c & 1], (uint32_t)(c >> 1) & 1u, p.status, 1u << 16);
        for (int it = s_ac; it < s_ai; it++) mbar_wait(&afull[it % NA], (uint32_t)(it / NA) & 1u, p.status, 1u << 16);
    }
    __syncthreads();
    if (warp == 8) tmem_dealloc(tmem, 512);
}

// Row maxima when rows are contiguous in memory (sr == 1): 32 rows x 256 k
// per block, read along rows (coalesced); per-row maxima go to rowmax (ordered
// bit patterns of non-negative doubles) with atomicMax.
__global__ void oz_rowmax_cols_kernel(int rows, int K, const double* __restrict__ src, long long sk,
                                      unsigned long long* __restrict__ rowmax, const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ unsigned long long red[8][33];
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int r = blockIdx.x * 32 + tx, k0 = blockIdx.y * 256;
    unsigned long long m = 0;
    if (r < rows)
        for (int kk = ty; kk < 256; kk += 8) {
            const int k = k0 + kk;
            if (k < K) m = oz_umax(m, oz_absbits(src[r + (long long)k * sk]));
        }
    red[ty][tx] = m;
    __syncthreads();
    if (ty == 0) {
        for (int q = 1; q < 8; q++) m = oz_umax(m, red[q][tx]);
        if (r < rows && m > 0) atomicMax(rowmax + r, m);
    }
}

// Digit slices when rows are contiguous (sr == 1): a 32 x 32 tile is read
// along rows and written along k through shared memory.
__global__ void oz_split_cols_kernel(int rows, int K, int Rp, int Kp, const double* __restrict__ src, long long sk,
                                     double sgn, const int* __restrict__ e, __nv_bfloat16* __restrict__ dst,
                                     const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ double tile[32][33];
    const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int kk = ty; kk < 32; kk += 8) {
        const int r = r0 + tx, k = k0 + kk;
        tile[kk][tx] = (r < rows && k < K) ? oz_neg_if(src[r + (long long)k * sk], sgn < 0.0) : 0.0;
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
    if (r < k) return oz_neg_if(src[(long long)k + (long long)r * sk], true);
    return 0.0;
}

__global__ void oz_exp_kernel(int rows, int K, const double* __restrict__ src, long long sr, long long sk,
                              int* __restrict__ e, int skew, const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ unsigned long long red[32];
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        unsigned long long m = 0;
        for (int k = threadIdx.x; k < K; k += blockDim.x) m = oz_umax(m, oz_absbits(oz_elem(src, sr, sk, skew, r, k)));
        for (int o = 16; o > 0; o >>= 1) m = oz_umax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long mm = 0;
            for (int w = 0; w < (int)(blockDim.x + 31) / 32; w++) mm = oz_umax(mm, red[w]);
            int ex = 0;
            if (mm > 0) {
                frexp(__longlong_as_double((long long)mm), &ex);  // mm = f 2^ex, f in [0.5, 1): mm < 2^ex
            }
            e[r] = ex;
        }
        __syncthreads();
    }
}

// Rows contiguous in k (sk == 1): one block per row finds the row maximum,
// then writes the row's digits two k at a time (the second read of the row
// comes from L2).  Padding rows and columns are zero.
__global__ void __launch_bounds__(256) oz_split_rows_kernel(int rows, int K, int Rp, int Kp, const double* __restrict__ src,
                                                            long long sr, double sgn, int* __restrict__ e,
                                                            __nv_bfloat16* __restrict__ dst,
                                                            const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ unsigned long long red[8];
    const bool neg = sgn < 0.0;
    for (int r = blockIdx.x; r < Rp; r += gridDim.x) {
        const double* row = src + (long long)r * sr;
        unsigned long long m = 0;
        if (r < rows)
            for (int k = threadIdx.x; k < K; k += 256) m = oz_umax(m, oz_absbits(row[k]));
        for (int o = 16; o > 0; o >>= 1) m = oz_umax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        m = red[0];
        for (int w = 1; w < 8; w++) m = oz_umax(m, red[w]);
        int ex = 0;
        if (m > 0) frexp(__longlong_as_double((long long)m), &ex);  // m = f 2^ex, f in [0.5, 1): every |x| < 2^ex
        if (threadIdx.x == 0) e[r] = ex;
        for (int k = 2 * threadIdx.x; k < Kp; k += 512) {
            const double x0 = (r < rows && k < K) ? oz_neg_if(row[k], neg) : 0.0;
            const double x1 = (r < rows && k + 1 < K) ? oz_neg_if(row[k + 1], neg) : 0.0;
            float d0[8], d1[8];
            oz_digits(x0, ex, d0);
            oz_digits(x1, ex, d1);
#pragma unroll
            for (int i = 0; i < SL; i++)
                *reinterpret_cast<__nv_bfloat162*>(dst + ((long long)i * Rp + r) * Kp + k) =
                    __floats2bfloat162_rn(d0[i], d1[i]);
        }
        __syncthreads();  // red is reused by the next row
    }
}

// Digit slices: plane i holds rows [i Rp, i Rp + rows) of a (SL Rp) x Kp
// row-major BF16 array; padding rows / columns are zero.
__global__ void oz_split_kernel(int rows, int K, int Rp, int Kp, const double* __restrict__ src, long long sr,
                                long long sk, double sgn, const int* __restrict__ e, __nv_bfloat16* __restrict__ dst,
                                const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Kp) return;
    for (int r = blockIdx.y; r < Rp; r += gridDim.y) {
        const double x = (r < rows && k < K) ? oz_neg_if(src[(long long)r * sr + (long long)k * sk], sgn < 0.0) : 0.0;
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
                                      unsigned long long* __restrict__ rowmax, const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ unsigned long long tile[32][33];
    const int bi = blockIdx.x, bj = blockIdx.y;
    if (bi < bj) return;
    const int i0 = bi * 32, j0 = bj * 32, tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int jj = ty; jj < 32; jj += 8) {
        const int i = i0 + tx, j = j0 + jj;
        tile[jj][tx] = (i < n && j < n && i > j) ? oz_absbits(W[i + (long long)j * ld]) : 0ULL;
    }
    __syncthreads();
    if (ty == 0) {
        unsigned long long rm = 0, cm = 0;  // row i0+tx over the tile's columns; column j0+tx over its rows
        for (int jj = 0; jj < 32; jj++) rm = oz_umax(rm, tile[jj][tx]);
        for (int ii = 0; ii < 32; ii++) cm = oz_umax(cm, tile[tx][ii]);
        if (i0 + tx < n && rm > 0) atomicMax(rowmax + i0 + tx, rm);
        if (j0 + tx < n && cm > 0) atomicMax(rowmax + j0 + tx, cm);
    }
}

__global__ void oz_exp_from_max_kernel(int rows, const unsigned long long* __restrict__ rowmax, int* __restrict__ e,
                                       const int* __restrict__ skip) {
    if (skip && *skip) return;
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
                                     const int* __restrict__ e, __nv_bfloat16* __restrict__ dst,
                                     const int* __restrict__ skip) {
    if (skip && *skip) return;
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
            tile[tx][rr] = (r < rows && k < rows) ? oz_neg_if(W[k + (long long)r * ld], true) : 0.0;
        }
    } else {
        for (int kk = ty; kk < 32; kk += 8) {
            const int r = r0 + tx, k = k0 + kk;
            double v = 0.0;
            if (r < rows && k < rows)
                v = (r > k) ? W[r + (long long)k * ld] : (r < k ? oz_neg_if(W[k + (long long)r * ld], true) : 0.0);
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

// C = alpha * sum_z part[z] + beta C, the partials summed in order z = 0, 1, ..
__global__ void oz_splitk_reduce_kernel(int M, int N, int nz, const double* __restrict__ part, double alpha,
                                        double beta, double* __restrict__ C, long long ldc) {
    const long long total = (long long)M * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int zz = 0; zz < nz; zz++) acc += __ldcg(part + zz * total + e);
        const long long col = e / M, row = e - col * M;
        double* dst = C + col * ldc + row;
        *dst = (beta == 0.0) ? alpha * acc : fma(beta, *dst, alpha * acc);
    }
}

inline long long rup(long long x, long long a) { return (x + a - 1) / a * a; }
inline int gridn(long long total) {
    long long g = (total + 255) / 256;
    return (int)(g > 16384 ? 16384 : (g < 1 ? 1 : g));
}

}  // namespace

size_t ozaki_operand_ws(int rows, int K) {
    const long long Kp = rup(K > 0 ? K : 1, OKA), Rp = rup(rows > 0 ? rows : 1, OM);
    return align_up((size_t)(SL * Rp * Kp * 2)) + align_up(sizeof(int) * Rp) + align_up(sizeof(unsigned long long) * Rp);
}

size_t ozaki_gemm_ws(int M, int N, int K) { return ozaki_operand_ws(M, K) + ozaki_operand_ws(N, K) + 256; }

// Digit slices of the operand X[r, k] = sgn * src[r * rs + k * ks] (rows x K),
// or, with skew, of the skew matrix whose strict lower triangle src holds
// (leading dimension ks).  Rows are padded to a multiple of 128, K to 64.
int ozaki_split(cudaStream_t st, int rows, int K, const double* src, long long rs, long long ks, double sgn, int skew,
                void* ws, size_t ws_bytes, OzOperand* op, const int* skip) {
    if (rows <= 0 || K <= 0) return SKEW_ERR_UNSUPPORTED;
    const long long Kp = rup(K, OKA), Rp = rup(rows, OM);
    Carve cv(ws, ws_bytes);
    __nv_bfloat16* d = cv.take<__nv_bfloat16>((size_t)(SL * Rp * Kp));
    int* e = cv.take<int>((size_t)Rp);
    unsigned long long* rowmax = cv.take<unsigned long long>((size_t)Rp);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    KtScope kt(st, KT_SLICE_SPLIT);
    if (skew || (rs == 1 && ks != 1)) {
        if (const cudaError_t err = cudaMemsetAsync(rowmax, 0, sizeof(unsigned long long) * (size_t)Rp, st))
            return cuda_fail(err);
        if (skew) {
            const unsigned T = (unsigned)((rows + 31) / 32);
            oz_skew_rowmax_kernel<<<dim3(T, T), dim3(32, 8), 0, st>>>(rows, src, ks, rowmax, skip);
        } else {
            oz_rowmax_cols_kernel<<<dim3((unsigned)((rows + 31) / 32), (unsigned)((K + 255) / 256)), dim3(32, 8), 0,
                                    st>>>(rows, K, src, ks, rowmax, skip);
        }
        oz_exp_from_max_kernel<<<(rows + 255) / 256, 256, 0, st>>>(rows, rowmax, e, skip);
        if (skew)
            oz_split_skew_kernel<<<dim3((unsigned)((Rp + 31) / 32), (unsigned)((Kp + 31) / 32)), dim3(32, 8), 0, st>>>(
                rows, (int)Rp, (int)Kp, src, ks, e, d, skip);
        else
            oz_split_cols_kernel<<<dim3((unsigned)((Rp + 31) / 32), (unsigned)((Kp + 31) / 32)), dim3(32, 8), 0, st>>>(
                rows, K, (int)Rp, (int)Kp, src, ks, sgn, e, d, skip);
        count_launch(3);
    } else if (ks == 1) {
        oz_split_rows_kernel<<<(int)(Rp < 32768 ? Rp : 32768), 256, 0, st>>>(rows, K, (int)Rp, (int)Kp, src, rs, sgn, e,
                                                                            d, skip);
        count_launch(1);
    } else {
        oz_exp_kernel<<<(int)(rows < 16384 ? rows : 16384), 256, 0, st>>>(rows, K, src, rs, ks, e, 0, skip);
        oz_split_kernel<<<dim3((unsigned)((Kp + 255) / 256), (unsigned)(Rp < 65535 ? Rp : 65535)), 256, 0, st>>>(
            rows, K, (int)Rp, (int)Kp, src, rs, ks, sgn, e, d, skip);
        count_launch(2);
    }
    op->d = d;
    op->e = e;
    op->rows = rows;
    op->K = K;
    op->Rp = Rp;
    op->Kp = Kp;
    op->roff = 0;
    op->koff = 0;
    return 0;
}

OzOperand oz_view(const OzOperand& o, int r0, int k0, int rows, int K) {
    OzOperand v = o;
    v.d = o.d + (size_t)r0 * (size_t)o.Kp;
    v.e = o.e + r0;
    v.rows = rows;
    v.K = K;
    v.roff = o.roff + r0;
    v.koff = o.koff + k0;
    return v;
}

// C = alpha * A B^T + beta C from split operands (A: M x K, B: N x K).
int ozaki_gemm_pre(cudaStream_t st, const OzOperand& A, const OzOperand& B, double alpha, double beta, double* C,
                   long long ldc, int* status, int slices, int lower, int ksplit, double* part, size_t part_elems,
                   const int* skip, const int* s_dyn) {
    const int M = A.rows, N = B.rows, K = A.K;
    if (M <= 0 || N <= 0) return 0;
    if (B.K != K || slices < 1 || slices > SL) return SKEW_ERR_UNSUPPORTED;
    const long long kpad = rup(K, OKA);  // K chunks read from each operand
    if (A.koff % OKA || B.koff % OKA || A.koff + kpad > A.Kp || B.koff + kpad > B.Kp) return SKEW_ERR_UNSUPPORTED;
    // a view's map starts at its first row and ends where the split ends:
    // rows past it (last plane, last tile) read as zeros instead of memory
    // beyond the buffer
    CUtensorMap ta, tb;
    if (!make_tmap_bf16(&ta, A.d, (uint64_t)A.Kp, (uint64_t)(SL * A.Rp - A.roff), (uint64_t)A.Kp, OM))
        return SKEW_ERR_UNSUPPORTED;
    if (!make_tmap_bf16(&tb, B.d, (uint64_t)B.Kp, (uint64_t)(SL * B.Rp - B.roff), (uint64_t)B.Kp, ON))
        return SKEW_ERR_UNSUPPORTED;
    OzParams p{};
    p.M = M;
    p.N = N;
    p.nchunks = (int)(kpad / OKA);
    p.akoff = A.koff;
    p.bkoff = B.koff;
    p.Mp = (int)A.Rp;
    p.Np = (int)B.Rp;
    p.ea = A.e;
    p.eb = B.e;
    p.alpha = alpha;
    p.beta = beta;
    p.C = C;
    p.ldc = ldc;
    p.status = status;
    p.s = slices;
    p.skip = skip;
    p.s_dyn = s_dyn;
    p.lower = lower;
    p.mt = (M + OM - 1) / OM;
    p.nt = (N + ON - 1) / ON;
    int nz = 1;
    if (ksplit > 1) {
        // no more ranges than the partial buffer holds
        const size_t per = (size_t)M * (size_t)N;
        const long long fit = per ? (long long)(part_elems / per) : 0;
        if (ksplit > fit) ksplit = (int)fit;
    }
    if (ksplit > 1) {
        if (!part) return SKEW_ERR_WORKSPACE;
        p.kz = (p.nchunks + ksplit - 1) / ksplit;
        nz = (p.nchunks + p.kz - 1) / p.kz;
        p.part = part;
    }
    const size_t smem = OzSmem::bytes();
    // long K per item (>= 16 chunks): one CTA per item; short K: persistent
    // CTAs, whose FP64 epilogue overlaps the next item's MMAs
    const bool one = (p.kz ? p.kz : p.nchunks) >= 16;
    auto kern = one ? ozaki_gemm_kernel<true> : ozaki_gemm_kernel<false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // algorithmic work: the kept slice pairs over the outputs written
    const double pairs = slices * (slices + 1) / 2.0;
    const double outs = lower ? lower_count(M, N) : (double)M * N;
    const int kt = kt_begin(st);
    // persistent: one CTA per SM walks the (tile, K range) items
    const long long items = (long long)p.mt * p.nt * nz;
    const int grid = (int)((one || items < device_sms()) ? items : device_sms());
    kern<<<(unsigned)grid, OT, smem, st>>>(ta, tb, p);
    count_launch();
    if (nz > 1) {
        oz_splitk_reduce_kernel<<<gridn((long long)M * N), 256, 0, st>>>(M, N, nz, part, alpha, beta, C, ldc);
        count_launch();
    }
    kt_end(st, kt, g_kt_ozaki_kind, 2.0 * pairs * outs * K);
    return cuda_ok(cudaGetLastError());
}

// C = alpha * (sa A)(sb B)^T + beta C, A[i,k] = A[i*a_rs + k*a_ks], B[j,k] = B[j*b_rs + k*b_ks].
int ozaki_gemm(cudaStream_t st, int M, int N, int K, double alpha, const double* A, long long a_rs, long long a_ks,
               double sa, const double* B, long long b_rs, long long b_ks, double sb, double beta, double* C,
               long long ldc, void* ws, size_t ws_bytes, int* status, int a_skew, int slices, int lower) {
    if (M <= 0 || N <= 0) return 0;
    if (K <= 0 || slices < 1 || slices > SL) return SKEW_ERR_UNSUPPORTED;
    const size_t wa = ozaki_operand_ws(M, K), wb = ozaki_operand_ws(N, K);
    if (!ws || ws_bytes < wa + wb) return SKEW_ERR_WORKSPACE;
    OzOperand oa{}, ob{};
    int rc = ozaki_split(st, M, K, A, a_rs, a_ks, sa, a_skew, ws, wa, &oa);
    if (rc) return rc;
    if (!a_skew && B == A && b_rs == a_rs && b_ks == a_ks && sb == sa && N == M) {
        ob = oa;  // same operand (a Gram matrix): reuse its slices
    } else {
        rc = ozaki_split(st, N, K, B, b_rs, b_ks, sb, 0, static_cast<char*>(ws) + wa, wb, &ob);
        if (rc) return rc;
    }
    return ozaki_gemm_pre(st, oa, ob, alpha, beta, C, ldc, status, slices, lower);
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
