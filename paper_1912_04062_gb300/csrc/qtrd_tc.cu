// qtrd_tc.cu -- the Q_trd back-transformation (Sec. 2.1, step 3a of the
// two-step form; Algorithm 1 step 4) on the tensor cores.
//
// Q_trd is the product of the bulge-chase reflectors H_{s,k} = I - tau v v^T
// (sweep s, step k, v of length b = 64 on rows s+1+k b .. s+k b+b).  As in the
// SIMT kernels, 64 consecutive sweeps s0 .. s0+63 at one step k form a block
// whose reflectors act inside the 128-row window r0 = s0+1+64k .. r0+127, and
// the order "groups descending, inside a group k ascending, inside a block s
// descending" is the reverse generation order up to swaps of reflectors on
// disjoint rows.  Here a block is applied in its compact WY form (Eq. 7):
//   H_{s0} H_{s0+1} ... H_{s0+63} = I - V T V^T,
// V (128 x 64, column j = v of sweep s0+j placed at window rows j .. j+63), T
// upper triangular from the forward recurrence T_jj = tau_j,
// T_{0:j,j} = -tau_j T_{0:j,0:j} (V_{:,0:j}^T v_j).  With U = V T the block
// update of the window is Z <- Z - U (V^T Z): two dense products, on tcgen05.
//
// qtrd_wy_kernel forms V, T and U of every block (FP32) and stores V and -U
// as three BF16 planes each (hi, mid, lo: about 24 bits), already in the
// K-major 128-byte-swizzled layout the MMA reads, so the main kernel fetches a
// block's operands with three bulk copies per matrix.
//
// qtrd_tc_kernel: one CTA per 128 columns of Z.  The window's transpose
// Z^T (128 columns x 128 rows, FP32) lives in TMEM (lane = column, TMEM
// column = row slot).  Per block:
//   1. Z^T is read from TMEM, split into three BF16 planes and stored as the
//      A operand (K = window rows);
//   2. W^T = Z^T V (M = 128 columns, N = 64 reflectors, K = 128): six plane
//      products (orders <= 2) into TMEM;
//   3. W^T is read, split into planes (A operand, K = 64 reflectors);
//   4. Z^T += W^T (-U)^T, accumulated into the window in TMEM (N = 128 window
//      rows as two halves of 64);
//   5. the window slides by 64 rows: the 64 finished rows go to global memory
//      and the next 64 come in.  Slots are reused circularly (window row i of
//      block k sits in slot (i + 64 (k mod 2)) mod 128), which the operand
//      addressing follows: the V image's two K-atoms swap and the U image's
//      two row halves target the matching TMEM column halves.
// The plane products run small orders first, so that the big hi x hi terms are
// added last.  Waits on mbarriers are capped; on a timeout the CTA records
// SKEW_ERR_DEVICE_TIMEOUT, waits for its copies and products in flight and
// leaves.
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "sm100.cuh"

namespace sk {
namespace {

constexpr int TB = 64;        // band width = reflector length = sweeps per block
constexpr int TW = 2 * TB;    // window rows
constexpr int TCOLS = 128;    // columns of Z per CTA (the MMA's M)
constexpr int TPL = 3;        // BF16 planes per operand
constexpr int TTHREADS = 256;
constexpr uint32_t V_PLANE = 2u * TB * 128u;       // 2 K-atoms x 64 rows x 128 B
constexpr uint32_t U_PLANE = (uint32_t)TW * 128u;  // 1 K-atom x 128 rows x 128 B
constexpr uint32_t V_IMG = TPL * V_PLANE;
constexpr uint32_t U_IMG = TPL * U_PLANE;
constexpr uint32_t IMG_BYTES = V_IMG + U_IMG;      // per block
constexpr uint32_t A1_ATOM = (uint32_t)TCOLS * 128u;  // 128 rows x 128 B
constexpr uint32_t A1_PLANE = 2u * A1_ATOM;            // Z^T: K = 128
constexpr uint32_t A2_PLANE = A1_ATOM;                 // W^T: K = 64
constexpr uint32_t A1_BYTES = TPL * A1_PLANE;
constexpr uint32_t SMEM_BYTES = A1_BYTES + V_IMG + U_IMG + 64 + 1024;  // + barriers, alignment slack

__host__ __device__ inline int tc_qsteps(int n, int s) { return (s <= n - 3) ? 1 + (n - 3 - s) / TB : 0; }

// blocks of groups 0 .. g-1 (group g' has Q + 1 - g' steps)
__host__ __device__ inline long long tc_block_index(int g, int k, int Q) {
    return (long long)g * (Q + 1) - (long long)g * (g - 1) / 2 + k;
}

// Byte offset of element (row, kk), kk < 64, of a K-major BF16 atom whose
// 128-byte rows carry the 128-byte swizzle (16-byte chunk index XOR row mod 8).
__host__ __device__ inline uint32_t sw128(int row, int kk) {
    return (uint32_t)row * 128u + ((uint32_t)((kk >> 3) ^ (row & 7)) << 4) + ((uint32_t)(kk & 7) << 1);
}

// x = hi + mid + lo (BF16 each; the remainders are exact in FP32)
SK_DEV void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

SK_DEV uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// 8 consecutive K elements -> one 16-byte chunk per plane
SK_DEV void split8(const float* x, uint4 (&o)[TPL]) {
    __nv_bfloat16 h[8], m[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; i++) split3(x[i], h[i], m[i], l[i]);
    o[0] = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
    o[1] = make_uint4(pack2(m[0], m[1]), pack2(m[2], m[3]), pack2(m[4], m[5]), pack2(m[6], m[7]));
    o[2] = make_uint4(pack2(l[0], l[1]), pack2(l[2], l[3]), pack2(l[4], l[5]), pack2(l[6], l[7]));
}

SK_DEV void tmem_st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
        "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
        "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}
SK_DEV void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Capped wait for an mbarrier phase that ignores errors recorded by others
// (the exit path: asynchronous copies into shared memory must land before the
// CTA leaves).  Gives up after about a second and records the timeout.
SK_DEV void drain_wait(uint64_t* bar, uint32_t parity, int* status) {
    for (uint32_t i = 0; i < (1u << 24); i++) {
        if (mbar_try_wait(bar, parity)) return;
        if (i > 1024) __nanosleep(64);
    }
    sk_set_error(status, SKEW_ERR_DEVICE_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Compact WY form of block (g, k) (grid x = k, y = g), images for the MMAs.
// V32 / tau32: the chase's FP32 reflectors, slot k nsw64 + s (64 floats each,
// zero padded beyond the matrix; taus of absent steps zero).
__global__ void __launch_bounds__(TTHREADS)
qtrd_wy_kernel(int n, const float* __restrict__ V32, const float* __restrict__ tau32, int nsw64, int Q,
               unsigned char* __restrict__ img) {
    const int k = blockIdx.x, g = blockIdx.y;
    if (k > Q - g) return;
    __shared__ float Vs[TB][TB + 1];  // Vs[j][i] = element i of reflector j (window row j + i)
    __shared__ float Gm[TB][TB + 1];  // Gm[i][j] = v_i^T v_j, i <= j
    __shared__ float T[TB][TB + 1];   // T[i][j], upper triangular
    __shared__ float taus[TB];
    const int t = threadIdx.x;
    const int nsw = n - 2, s0 = g * TB;
    unsigned char* out = img + tc_block_index(g, k, Q) * (long long)IMG_BYTES;
    if (t < TB) {
        const int s = s0 + t;
        taus[t] = (s < nsw && k < tc_qsteps(n, s)) ? tau32[(size_t)k * nsw64 + s] : 0.f;
    }
    __syncthreads();
    for (int e = t; e < TB * TB; e += TTHREADS) {
        const int j = e >> 6, i = e & 63;
        // absent reflectors (tau = 0) count as v = 0: their slots may hold stale data
        Vs[j][i] = (taus[j] != 0.f) ? V32[((size_t)k * nsw64 + s0 + j) * TB + i] : 0.f;
        T[j][i] = 0.f;
    }
    __syncthreads();
    // Gram of the parallelogram: v_i covers window rows i .. i+63, so for
    // i <= j (d = j - i) the overlap is rows j .. i+63
    for (int e = t; e < TB * TB; e += TTHREADS) {
        const int i = e & 63, j = e >> 6;
        if (i > j) continue;
        const int d = j - i;
        float a = 0.f;
        for (int u = d; u < TB; u++) a = fmaf(Vs[i][u], Vs[j][u - d], a);
        Gm[i][j] = a;
    }
    __syncthreads();
    // forward recurrence of Eq. 7: column j of T from columns 0 .. j-1
    for (int j = 0; j < TB; j++) {
        if (t < j) {
            float a = 0.f;
            for (int l = t; l < j; l++) a = fmaf(T[t][l], Gm[l][j], a);
            T[t][j] = -taus[j] * a;
        } else if (t == j) {
            T[j][j] = taus[j];
        }
        __syncthreads();
    }
    // -U = -V T, rows r = window rows, K = reflector j
    for (int e = t; e < TW * TB; e += TTHREADS) {
        const int r = e >> 6, j = e & 63;
        const int i0 = r - (TB - 1) > 0 ? r - (TB - 1) : 0, i1 = j < r ? j : r;
        float a = 0.f;
        for (int i = i0; i <= i1; i++) a = fmaf(Vs[i][r - i], T[i][j], a);
        __nv_bfloat16 h, m, l;
        split3(-a, h, m, l);
        const uint32_t off = V_IMG + sw128(r, j);
        *reinterpret_cast<__nv_bfloat16*>(out + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(out + off + U_PLANE) = m;
        *reinterpret_cast<__nv_bfloat16*>(out + off + 2 * U_PLANE) = l;
    }
    // V: rows = reflectors j, K = window rows r (two K-atoms of 64)
    for (int e = t; e < TB * TW; e += TTHREADS) {
        const int j = e >> 7, r = e & (TW - 1);
        const int i = r - j;
        const float v = (i >= 0 && i < TB) ? Vs[j][i] : 0.f;
        __nv_bfloat16 h, m, l;
        split3(v, h, m, l);
        const uint32_t off = (uint32_t)(r >> 6) * (uint32_t)(TB * 128) + sw128(j, r & 63);
        *reinterpret_cast<__nv_bfloat16*>(out + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(out + off + V_PLANE) = m;
        *reinterpret_cast<__nv_bfloat16*>(out + off + 2 * V_PLANE) = l;
    }
}

// plane pairs (a, b) of orders <= 2, small orders first
__constant__ int kPairs[6][2] = {{2, 0}, {1, 1}, {0, 2}, {1, 0}, {0, 1}, {0, 0}};

__global__ void __launch_bounds__(TTHREADS, 1)
qtrd_tc_kernel(int n, const unsigned char* __restrict__ img, float* __restrict__ Z, int ldz, int ncols, int Q,
               int* status) {
    extern __shared__ unsigned char qtc_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(qtc_raw) + 1023) &
                                                         ~uintptr_t(1023));
    unsigned char* A1 = sm;            // Z^T planes, later W^T planes
    unsigned char* VB = sm + A1_BYTES;  // V image of the current block
    unsigned char* UB = VB + V_IMG;     // -U image of the current block
    uint64_t* bar = reinterpret_cast<uint64_t*>(UB + U_IMG);
    uint64_t* mv = bar;      // V image landed
    uint64_t* mu = bar + 1;  // U image landed
    uint64_t* m1 = bar + 2;  // W^T = Z^T V done
    uint64_t* m2 = bar + 3;  // window update done
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int wg = warp >> 2, quad = warp & 3;
    const int c = quad * 32 + lane;  // column of the slab = TMEM lane
    const int c0 = blockIdx.x * TCOLS;
    const bool own = c0 + c < ncols;
    float* zc = Z + (size_t)(own ? c0 + c : 0) * ldz;
    const int G = Q + 1;

    if (t == 0) {
        mbar_init(mv, 1);
        mbar_init(mu, 1);
        mbar_init(m1, 1);
        mbar_init(m2, 1);
        fence_mbar_init();
        *abort_flag = 0;
    }
    if (warp == 0) {
        tmem_alloc(tslot, 256);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);

    // issue / completion counts (thread 0 issues; everyone waits by phase)
    int v_iss = 0, u_iss = 0, m1_iss = 0, m2_iss = 0;
    int v_done = 0, u_done = 0, m1_done = 0, m2_done = 0;
    auto load_v = [&](int g, int k) {
        const unsigned char* src = img + tc_block_index(g, k, Q) * (long long)IMG_BYTES;
        mbar_arrive_expect_tx(mv, V_IMG);
        for (int pl = 0; pl < TPL; pl++) bulk_g2s(VB + pl * V_PLANE, src + pl * V_PLANE, V_PLANE, mv);
    };
    auto load_u = [&](int g, int k) {
        const unsigned char* src = img + tc_block_index(g, k, Q) * (long long)IMG_BYTES + V_IMG;
        mbar_arrive_expect_tx(mu, U_IMG);
        for (int pl = 0; pl < TPL; pl++) bulk_g2s(UB + pl * U_PLANE, src + pl * U_PLANE, U_PLANE, mu);
    };
    if (t == 0) {
        load_v(G - 1, 0);
        load_u(G - 1, 0);
    }
    v_iss = u_iss = 1;

    // window rows [r, r + 64) of this column into TMEM slots [slot, slot + 64)
    auto fill = [&](int r, int slot) {
#pragma unroll
        for (int q4 = 0; q4 < 4; q4++) {
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int row = r + 16 * q4 + i;
                v[i] = (own && row < n) ? zc[row] : 0.f;
            }
            tmem_st16(lane_base + (uint32_t)(slot + 16 * q4), v);
        }
        tmem_wait_st();
    };
    auto drain = [&](int slot, int r) {
#pragma unroll
        for (int q4 = 0; q4 < 4; q4++) {
            float v[16];
            tmem_ld16(lane_base + (uint32_t)(slot + 16 * q4), v);
            if (own) {
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const int row = r + 16 * q4 + i;
                    if (row < n) zc[row] = v[i];
                }
            }
        }
    };
    // all threads: capped wait on a phase; a failure anywhere ends the CTA's
    // work (a phase counts as done only when it was seen to complete)
    auto wait_all = [&](uint64_t* b, int& done) -> bool {
        if (mbar_wait(b, (uint32_t)done & 1u, status)) done++;
        else *abort_flag = 1;
        __syncthreads();
        return *abort_flag == 0;
    };

    bool ok = true;
    for (int g = G - 1; g >= 0 && ok; g--) {
        const int s0 = g * TB, Kg = Q + 1 - g;
        fill(s0 + 1 + 64 * wg, 64 * wg);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        for (int k = 0; k < Kg && ok; k++) {
            const int p = k & 1;
            const int r0 = s0 + 1 + TB * k;
            // 1. Z^T (own 64 slots = K-atom wg) -> three BF16 planes
#pragma unroll
            for (int q4 = 0; q4 < 4; q4++) {
                float v[16];
                tmem_ld16(lane_base + (uint32_t)(64 * wg + 16 * q4), v);
#pragma unroll
                for (int hh = 0; hh < 2; hh++) {
                    uint4 o[TPL];
                    split8(v + 8 * hh, o);
                    const uint32_t off = (uint32_t)wg * A1_ATOM + (uint32_t)c * 128u +
                                         ((uint32_t)((2 * q4 + hh) ^ (c & 7)) << 4);
#pragma unroll
                    for (int pl = 0; pl < TPL; pl++) *reinterpret_cast<uint4*>(A1 + pl * A1_PLANE + off) = o[pl];
                }
            }
            fence_proxy_async_smem();
            tc_fence_before();
            // 2. W^T = Z^T V (needs the V image of this block)
            ok = wait_all(mv, v_done);
            if (!ok) break;
            if (t == 0) {
                tc_fence_after();
                const uint32_t a1 = smem_u32(A1), vb = smem_u32(VB);
                uint32_t acc = 0u;
                for (int pi = 0; pi < 6; pi++) {
                    const int ia = kPairs[pi][0], ib = kPairs[pi][1];
#pragma unroll
                    for (int s = 0; s < 8; s++) {
                        const int atom = s >> 2, kq = s & 3;
                        const uint64_t ad = umma_desc_sw128(a1 + ia * A1_PLANE + atom * A1_ATOM + kq * 32);
                        const uint64_t bd =
                            umma_desc_sw128(vb + ib * V_PLANE + (uint32_t)((atom ^ p) * TB * 128) + kq * 32);
                        umma_bf16(tmem + 128u, ad, bd, umma_idesc_bf16(128, 64), acc);
                        acc = 1u;
                    }
                }
                umma_commit(m1);
            }
            m1_iss++;
            ok = wait_all(m1, m1_done);
            if (!ok) break;
            tc_fence_after();
            // the V buffer is free: next block's V image
            if (t == 0) {
                if (k + 1 < Kg) load_v(g, k + 1);
                else if (g > 0) load_v(g - 1, 0);
            }
            if (k + 1 < Kg || g > 0) v_iss++;
            // 3. W^T (32 reflector columns per warpgroup) -> planes, K = reflector
#pragma unroll
            for (int q2 = 0; q2 < 2; q2++) {
                float v[16];
                tmem_ld16(lane_base + (uint32_t)(128 + 32 * wg + 16 * q2), v);
#pragma unroll
                for (int hh = 0; hh < 2; hh++) {
                    uint4 o[TPL];
                    split8(v + 8 * hh, o);
                    const uint32_t off =
                        (uint32_t)c * 128u + ((uint32_t)((4 * wg + 2 * q2 + hh) ^ (c & 7)) << 4);
#pragma unroll
                    for (int pl = 0; pl < TPL; pl++) *reinterpret_cast<uint4*>(A1 + pl * A2_PLANE + off) = o[pl];
                }
            }
            fence_proxy_async_smem();
            tc_fence_before();
            // 4. Z^T += W^T (-U)^T into the window's slots
            ok = wait_all(mu, u_done);
            if (!ok) break;
            if (t == 0) {
                tc_fence_after();
                const uint32_t a2 = smem_u32(A1), ub = smem_u32(UB);
                for (int pi = 0; pi < 6; pi++) {
                    const int ia = kPairs[pi][0], ib = kPairs[pi][1];
#pragma unroll
                    for (int s = 0; s < 4; s++) {
                        const uint64_t ad = umma_desc_sw128(a2 + ia * A2_PLANE + s * 32);
#pragma unroll
                        for (int hh = 0; hh < 2; hh++) {
                            const uint64_t bd = umma_desc_sw128(ub + ib * U_PLANE + hh * (TB * 128) + s * 32);
                            const uint32_t dcol = (uint32_t)(((hh + p) & 1) * 64);
                            umma_bf16(tmem + dcol, ad, bd, umma_idesc_bf16(128, 64), 1u);
                        }
                    }
                }
                umma_commit(m2);
            }
            m2_iss++;
            ok = wait_all(m2, m2_done);
            if (!ok) break;
            tc_fence_after();
            if (t == 0) {
                if (k + 1 < Kg) load_u(g, k + 1);
                else if (g > 0) load_u(g - 1, 0);
            }
            if (k + 1 < Kg || g > 0) u_iss++;
            // 5. slide (window rows 0..63 are in slots 64 p, held by warpgroup p)
            if (k + 1 < Kg) {
                if (wg == p) {
                    drain(64 * p, r0);
                    fill(r0 + TW, 64 * p);
                }
            } else {
                drain(64 * wg, r0 + (wg == p ? 0 : TB));
            }
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
    }
    // leave only with no copy or product in flight (these waits do not stop
    // early on an error recorded elsewhere: the copies must land first)
    if (t == 0) {
        while (v_done < v_iss) drain_wait(mv, (uint32_t)(v_done++) & 1u, status);
        while (u_done < u_iss) drain_wait(mu, (uint32_t)(u_done++) & 1u, status);
        while (m1_done < m1_iss) drain_wait(m1, (uint32_t)(m1_done++) & 1u, status);
        while (m2_done < m2_iss) drain_wait(m2, (uint32_t)(m2_done++) & 1u, status);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 256);
}

}  // namespace

size_t qtrd_tc_ws(int n) {
    if (n < 3) return 256;
    const long long Q = (n - 3) / TB;
    return (size_t)((Q + 1) * (Q + 2) / 2) * IMG_BYTES + 256;
}

int apply_qtrd_tc(cudaStream_t st, int n, const float* V32, const float* tau32, float* Z, int ldz, int k,
                  void* ws, size_t ws_bytes, int* status) {
    if (n < 3 || k <= 0) return 0;
    if (ws_bytes < qtrd_tc_ws(n) - 256 || !ws) return SKEW_ERR_WORKSPACE;
    const int Q = (n - 3) / TB;
    const int nsw64 = (n - 2 + TB - 1) / TB * TB;
    unsigned char* img = static_cast<unsigned char*>(ws);
    {
        KtScope kt(st, KT_QTRD);
        qtrd_wy_kernel<<<dim3((unsigned)(Q + 1), (unsigned)(Q + 1)), TTHREADS, 0, st>>>(n, V32, tau32, nsw64, Q, img);
        count_launch();
        if (cudaFuncSetAttribute(qtrd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES) !=
            cudaSuccess)
            return SKEW_ERR_LAUNCH;
        const int grid = (k + TCOLS - 1) / TCOLS;
        qtrd_tc_kernel<<<grid, TTHREADS, SMEM_BYTES, st>>>(n, img, Z, ldz, k, Q, status);
        count_launch();
    }
    return cuda_ok(cudaGetLastError());
}

}  // namespace sk
