// umma_gemm.cu -- BF16x3 split GEMM on the 5th-generation tensor cores
// (tcgen05.mma kind::f16, FP32 accumulation in TMEM) for the mixed form of the
// solver: the skew SYMM (a3), the skew rank-2k trailing update (a5) and the
// Q_band back-transform (a12).  Not in the paper; the paper's contractions are
// FP64 BLAS-3 (Sec. 2.3.2).
//
// Split (a13): every FP64 operand x becomes two BF16 planes, hi = bf16(x) and
// lo = bf16(x - hi) (round to nearest), stored side by side along K
// ([hi | lo], each plane padded to a multiple of 64).  The product keeps the
// three leading terms hi*hi + lo*hi + hi*lo; the dropped lo*lo term and the
// truncation of x - hi - lo are below 2^-16 relative, and the FP32
// accumulation adds about K 2^-24.
//
// Kernel: one 128 x BN output tile per CTA, 128 threads.  Thread 0 of warp 0
// issues TMA loads of 128 x 64 (A) and BN x 64 (B) BF16 tiles into 128-byte
// swizzled shared-memory stages; thread 0 of warp 1 issues tcgen05.mma (K = 16
// each) into a TMEM accumulator and releases each stage with tcgen05.commit;
// afterwards all four warps read the accumulator (tcgen05.ld, lanes = rows)
// and update the FP64 output in place.  Stage hand-off uses mbarriers; every
// wait is capped.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "sm100.cuh"

namespace sk {
namespace {

constexpr int UM = 128;   // tile rows (UMMA M)
constexpr int UK = 64;    // K per pipeline stage (128 bytes of BF16)
constexpr int UT = 128;   // threads per CTA

struct UmmaParams {
    int M, N;
    int kblocks;            // UK-blocks per term
    int nterms;
    int aplane[8], bplane[8];
    int Kp;                 // K extent of one plane (multiple of UK)
    int lower;              // 1: lower-triangular tile grid, C += alpha D, zero diagonal
    double alpha, beta;
    double* C;
    long long ldc;
    int* status;
};

template <int BN, int STAGES>
struct UmmaSmem {
    static constexpr uint32_t A_BYTES = UM * UK * 2;
    static constexpr uint32_t B_BYTES = BN * UK * 2;
    static constexpr size_t bytes() {
        return 1024 + (size_t)STAGES * (A_BYTES + B_BYTES) + 8 * (2 * STAGES + 1) + 16;
    }
};

template <int BN, int STAGES>
__global__ void __launch_bounds__(UT, 1)
umma_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, UmmaParams p) {
    using L = UmmaSmem<BN, STAGES>;
    extern __shared__ unsigned char umma_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(umma_raw) + 1023) &
                                                         ~uintptr_t(1023));
    unsigned char* sA = sm;
    unsigned char* sB = sm + STAGES * L::A_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * L::B_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accum = empty + STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    __shared__ int s_issued, s_consumed;

    int I, J;
    if (p.lower) {
        const long long t = blockIdx.x;
        I = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((long long)(I + 1) * (I + 2) / 2 <= t) I++;
        while ((long long)I * (I + 1) / 2 > t) I--;
        J = (int)(t - (long long)I * (I + 1) / 2);
    } else {
        I = blockIdx.x;
        J = blockIdx.y;
    }
    const int m0 = I * UM, n0 = J * BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
        s_issued = 0;
        s_consumed = 0;
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int total = p.nterms * p.kblocks;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        int it = 0;
        for (; it < total; it++) {
            const int s = it % STAGES;
            const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u, p.status)) break;
            const int t = it / p.kblocks, kb = it % p.kblocks;
            mbar_arrive_expect_tx(&full[s], L::A_BYTES + L::B_BYTES);
            tma_load_2d(sA + s * L::A_BYTES, &tmA, &full[s], p.aplane[t] * p.Kp + kb * UK, m0);
            tma_load_2d(sB + s * L::B_BYTES, &tmB, &full[s], p.bplane[t] * p.Kp + kb * UK, n0);
        }
        s_issued = it;
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        constexpr uint32_t idesc = umma_idesc_bf16(UM, BN);
        int it = 0;
        for (; it < total; it++) {
            const int s = it % STAGES;
            const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
            if (!mbar_wait(&full[s], ph, p.status)) break;
            tc_fence_after();
            const uint64_t ad = umma_desc_sw128(smem_u32(sA + s * L::A_BYTES));
            const uint64_t bd = umma_desc_sw128(smem_u32(sB + s * L::B_BYTES));
#pragma unroll
            for (int k = 0; k < UK / 16; k++)
                umma_bf16(tmem, ad + 2 * k, bd + 2 * k, idesc, (it > 0 || k > 0) ? 1u : 0u);
            umma_commit(&empty[s]);
        }
        s_consumed = it;
        umma_commit(accum);
    }
    __syncwarp();

    // ---- epilogue: TMEM lanes 32w..32w+31 = tile rows, 16 columns per load
    const bool ok = mbar_wait(accum, 0, p.status);
    tc_fence_after();
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        const bool rin = row < p.M;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (!rin) continue;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int col = n0 + c0 + j;
                if (col >= p.N) continue;
                double* q = p.C + (long long)col * p.ldc + row;
                const double d = p.alpha * (double)v[j];
                if (p.lower) *q = (row == col) ? 0.0 : (*q + d);
                else *q = (p.beta == 0.0) ? d : fma(p.beta, *q, d);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    // after a timeout, let TMA copies that were issued but never consumed land
    // before the shared memory is released (capped as well)
    if (threadIdx.x == 0 && s_issued > s_consumed) {
        for (int it = s_consumed; it < s_issued; it++)
            mbar_wait(&full[it % STAGES], (uint32_t)(it / STAGES) & 1u, p.status, 1u << 16);
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, BN);
}

// FP64 -> [hi | lo] (nplanes = 2) or [hi | mid | lo] (nplanes = 3) BF16
// planes, row-major with leading dimension ldd (elements), each plane Kp
// wide; rows >= rows and k >= K are zero.  Each plane is the round-to-nearest
// BF16 of what the previous planes leave of x.
// src element (r, k) = src[r * sr + k * sk] (mode 0) or, for mode 1, the skew
// matrix whose strict lower triangle is stored column-major in src (ld sk):
// (r, k) -> src[r + k*sk] (r > k), -src[k + r*sk] (r < k), 0 (r == k).
__global__ void split_bf16_kernel(int rows, int K, int rows_pad, int Kp, const double* __restrict__ src,
                                  long long sr, long long sk, int mode, __nv_bfloat16* __restrict__ dst,
                                  long long ldd, int nplanes) {
    const long long total = (long long)rows_pad * Kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % Kp), r = (int)(e / Kp);
        double x = 0.0;
        if (r < rows && k < K) {
            if (mode == 0) x = src[(long long)r * sr + (long long)k * sk];
            else if (r > k) x = src[(long long)r + (long long)k * sk];
            else if (r < k) x = -src[(long long)k + (long long)r * sk];
        }
        for (int pl = 0; pl < nplanes; pl++) {
            const __nv_bfloat16 h = __double2bfloat16(x);
            dst[(long long)r * ldd + (long long)pl * Kp + k] = h;
            x -= (double)__bfloat162float(h);
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool get_encode() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode != nullptr;
}

// 2-D BF16 tensor map: inner dimension `inner` elements (contiguous), `outer`
// rows `ld` elements apart; box 64 x box_rows, 128-byte swizzle.
bool make_tmap(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_rows) {
    if (!get_encode()) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)UK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

inline long long round_up(long long x, long long a) { return (x + a - 1) / a * a; }

template <int BN, int STAGES>
cudaError_t launch(cudaStream_t st, const CUtensorMap& ta, const CUtensorMap& tb, const UmmaParams& p, dim3 grid,
                   double flops) {
    const size_t smem = UmmaSmem<BN, STAGES>::bytes();
    cudaFuncSetAttribute(umma_gemm_kernel<BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int kt = kt_begin(st);
    umma_gemm_kernel<BN, STAGES><<<grid, UT, smem, st>>>(ta, tb, p);
    kt_end(st, kt, KT_SPLIT, flops);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

bool make_tmap_bf16(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_rows) {
    return make_tmap(m, base, inner, outer, ld, box_rows);
}

size_t split_gemm_ws(int M, int N, int K, int nplanes) {
    const long long Kp = round_up(K > 0 ? K : 1, UK);
    const long long Mp = round_up(M > 0 ? M : 1, UM), Np = round_up(N > 0 ? N : 1, 128);
    return (size_t)(align_up((size_t)(Mp * nplanes * Kp * 2)) + align_up((size_t)(Np * nplanes * Kp * 2)) + 256);
}

int split_gemm(cudaStream_t st, int M, int N, int K, double alpha, const double* A, long long a_rs, long long a_ks,
               int a_skew, const double* B, long long b_rs, long long b_ks, double beta, double* C, long long ldc,
               int lower, void* ws, size_t ws_bytes, int* status, int nplanes) {
    if (M <= 0 || N <= 0) return 0;
    if (K <= 0 || (nplanes != 2 && nplanes != 3)) return SKEW_ERR_UNSUPPORTED;
    if (lower && M != N) return SKEW_ERR_UNSUPPORTED;
    const long long Kp = round_up(K, UK);
    const int BN = (N <= 64 && !lower) ? 64 : 128;
    const long long Mp = round_up(M, UM), Np = round_up(N, BN);
    Carve cv(ws, ws_bytes);
    __nv_bfloat16* Ab = cv.take<__nv_bfloat16>((size_t)(Mp * nplanes * Kp));
    __nv_bfloat16* Bb = cv.take<__nv_bfloat16>((size_t)(round_up(N, 128) * nplanes * Kp));
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    auto grid_for = [](long long total) {
        long long g = (total + 255) / 256;
        return (int)(g > 16384 ? 16384 : (g < 1 ? 1 : g));
    };
    const long long ldb = (long long)nplanes * Kp;
    {
        KtScope kt(st, KT_SLICE_SPLIT);
        split_bf16_kernel<<<grid_for(Mp * Kp), 256, 0, st>>>(M, K, (int)Mp, (int)Kp, A, a_rs, a_ks, a_skew, Ab, ldb,
                                                             nplanes);
        split_bf16_kernel<<<grid_for(Np * Kp), 256, 0, st>>>(N, K, (int)Np, (int)Kp, B, b_rs, b_ks, 0, Bb, ldb,
                                                             nplanes);
    }
    count_launch(2);
    CUtensorMap ta, tb;
    if (!make_tmap(&ta, Ab, (uint64_t)ldb, (uint64_t)Mp, (uint64_t)ldb, UM)) return SKEW_ERR_UNSUPPORTED;
    if (!make_tmap(&tb, Bb, (uint64_t)ldb, (uint64_t)Np, (uint64_t)ldb, (uint32_t)BN)) return SKEW_ERR_UNSUPPORTED;
    UmmaParams p{};
    p.M = M;
    p.N = N;
    p.kblocks = (int)(Kp / UK);
    // plane pairs (a, b) kept: all with a + b <= nplanes - 1
    // (2 planes: hi*hi + lo*hi + hi*lo; 3 planes: the six terms of order <= 2)
    p.nterms = 0;
    for (int lvl = 0; lvl < nplanes; lvl++)
        for (int a = 0; a <= lvl; a++) {
            p.aplane[p.nterms] = a;
            p.bplane[p.nterms] = lvl - a;
            p.nterms++;
        }
    p.Kp = (int)Kp;
    p.lower = lower;
    p.alpha = alpha;
    p.beta = beta;
    p.C = C;
    p.ldc = ldc;
    p.status = status;
    // algorithmic work: the kept plane products over the outputs written
    const double flops = 2.0 * p.nterms * (lower ? lower_count(M, N) : (double)M * N) * K;
    cudaError_t e;
    if (lower) {
        const long long T = Mp / UM;
        e = launch<128, 3>(st, ta, tb, p, dim3((unsigned)(T * (T + 1) / 2)), flops);
    } else if (BN == 64) {
        e = launch<64, 4>(st, ta, tb, p, dim3((unsigned)(Mp / UM), (unsigned)(Np / 64)), flops);
    } else {
        e = launch<128, 3>(st, ta, tb, p, dim3((unsigned)(Mp / UM), (unsigned)(Np / 128)), flops);
    }
    return e == cudaSuccess ? 0 : SKEW_ERR_CUDA;
}

}  // namespace sk

extern "C" size_t skew_gemm_bf16x3_ws(int M, int N, int K) { return sk::split_gemm_ws(M, N, K, 3); }

extern "C" int skew_gemm_bf16x3(int M, int N, int K, double alpha, const double* A, long long a_rs, long long a_ks,
                                const double* B, long long b_rs, long long b_ks, double beta, double* C, int ldc,
                                int lower, int planes, void* ws, size_t ws_bytes, int* d_status, void* stream) {
    if (M < 0) return -1;
    if (N < 0) return -2;
    if (K < 1) return -3;
    if (ldc < (M > 1 ? M : 1)) return -13;
    if (lower && M != N) return -14;
    return sk::split_gemm(static_cast<cudaStream_t>(stream), M, N, K, alpha, A, a_rs, a_ks, 0, B, b_rs, b_ks, beta, C,
                          ldc, lower, ws, ws_bytes, d_status, planes == 3 ? 3 : 2);
}
