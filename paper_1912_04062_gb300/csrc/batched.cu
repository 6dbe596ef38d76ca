// batched.cu -- many independent skew eigenproblems of small and medium order
// in a few launches (the paper solves one matrix per run; this is the batched
// form of the same route for orders up to BATCH_MAX = 1024).
//
// Per matrix, one CTA tridiagonalises the whole skew matrix column by column
// with Householder reflectors (dlarfg convention; the skew two-sided update
// A <- A + v p^T - p v^T with p = tau A v, Eqs. 2-6 with u1 = -u2, whose
// 1/2 tau^2 (v^T A v) v term is 0 for skew A), giving alpha_c = T[c, c+1]
// (Lemma 1).  Orders up to BATCH_SMALL_MAX keep the matrix in shared memory;
// larger ones work on a copy in global memory (L2), one CTA each, so that the
// GPU runs as many matrices at a time as it has SMs.  One launch then bisects
// every wanted eigenvalue of every matrix, one launch runs inverse iteration
// for all of them (Sec. 3), and one CTA per matrix applies the D map
// (Algorithm 1 step 3) and the reflectors in reverse order to the eigenvectors.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tridiag_dev.cuh"

namespace sk {
namespace {

constexpr int BT = 256;  // threads per CTA of the per-matrix kernels

struct BItem {
    int n, nev, lda, vectors;
    double* S;                   // global working matrix (n x n) for n > BATCH_SMALL_MAX
    const double* A;
    double *lambda, *Zre, *Zim;  // Z: n x nev, leading dimension n
    int* info;                   // caller's status word of this matrix (may be null)
    // per-matrix scratch
    double *V, *tau, *alpha, *a2, *Qi;
    tri::TriScalars* sc;
    tri::InvitBufs bf;
    int* fail;
    long long e0;  // first global eigenvalue index of this matrix
};

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();  // red may still be read from a previous call
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < BT / 32; k++) s += red[k];
    return s;
}

__device__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < BT / 32; k++) s = fmax(s, red[k]);
    return s;
}

// One CTA per matrix (order[] lists the matrices, largest first).  G = false:
// shared memory holds S (n x n, ld n + 1), v and p; G = true: S is the
// matrix's global copy (ld n), v and p in shared memory.
template <bool G>
__global__ void __launch_bounds__(BT) bt_reduce_kernel(const BItem* __restrict__ items, const int* __restrict__ order) {
    extern __shared__ double bsm[];
    const BItem it = items[order[blockIdx.x]];
    const int n = it.n, ld = G ? n : n + 1, t = threadIdx.x;
    double* S = G ? it.S : bsm;
    double* v = G ? bsm : S + (size_t)n * ld;
    double* p = v + n;
    double* red = p + n;
    // S(i, j) = A(i, j) below the diagonal, -A(j, i) above: only the strict
    // lower triangle of A is read
    for (int e = t; e < n * n; e += BT) {
        const int i = e % n, j = e / n;
        double x = 0.0;
        if (i > j) x = it.A[i + (size_t)j * it.lda];
        else if (i < j) x = -it.A[j + (size_t)i * it.lda];
        S[i + (size_t)j * ld] = x;
    }
    __syncthreads();
    for (int c = 0; c + 2 < n; c++) {
        double a = 0.0;
        for (int i = c + 2 + t; i < n; i += BT) a = fma(S[i + (size_t)c * ld], S[i + (size_t)c * ld], a);
        a = block_sum(a, red);
        const double x0 = S[(c + 1) + (size_t)c * ld];
        double tau, beta, sc;
        if (a == 0.0) {
            tau = 0.0;
            beta = x0;
            sc = 0.0;
        } else {
            const double rr = sqrt(x0 * x0 + a);
            beta = (x0 >= 0.0) ? -rr : rr;
            tau = (beta - x0) / beta;
            sc = 1.0 / (x0 - beta);
        }
        for (int i = c + 1 + t; i < n; i += BT) {
            const double vi = (i == c + 1) ? 1.0 : S[i + (size_t)c * ld] * sc;
            v[i] = vi;
            it.V[i + (size_t)c * n] = vi;
        }
        if (t == 0) {
            it.tau[c] = tau;
            it.alpha[c] = -beta;  // T[c, c+1] = -T[c+1, c]
        }
        __syncthreads();
        if (tau != 0.0) {
            // p = tau S22 v, S22 = S[c+1:, c+1:]
            for (int i = c + 1 + t; i < n; i += BT) {
                double s2 = 0.0;
                for (int j = c + 1; j < n; j++) s2 = fma(S[i + (size_t)j * ld], v[j], s2);
                p[i] = tau * s2;
            }
            __syncthreads();
            // S22 += v p^T - p v^T on the whole square: each product is rounded
            // on its own, so element (j, i) receives exactly minus what (i, j)
            // receives and S stays exactly skew
            const int m = n - c - 1;
            for (int e = t; e < m * m; e += BT) {
                const int i = c + 1 + e % m, j = c + 1 + e / m;
                S[i + (size_t)j * ld] += __dsub_rn(__dmul_rn(v[i], p[j]), __dmul_rn(p[i], v[j]));
            }
        }
        __syncthreads();
    }
    if (t == 0 && n >= 2) it.alpha[n - 2] = S[(n - 2) + (size_t)(n - 1) * ld];
    __syncthreads();
    // ||S||_1 of tridiag(alpha, 0, alpha), pivmin, alpha^2
    double gm = 0.0, am = 0.0;
    for (int i = t; i < n; i += BT) {
        const double al = (i < n - 1) ? it.alpha[i] : 0.0;
        const double ap = (i > 0) ? it.alpha[i - 1] : 0.0;
        if (i < n - 1) it.a2[i] = al * al;
        gm = fmax(gm, fabs(al) + fabs(ap));
        am = fmax(am, al * al);
    }
    gm = block_max(gm, red);
    am = block_max(am, red);
    if (t == 0) {
        it.sc->g = gm;
        it.sc->pivmin = DBL_MIN * fmax(1.0, am);
        *it.fail = 0x7fffffff;
    }
}

// Matrix owning global eigenvalue index e (items sorted by e0).
__device__ int item_of(const BItem* __restrict__ items, int count, long long e) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].e0 <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void bt_bisect_kernel(const BItem* __restrict__ items, int count, long long total) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const BItem& it = items[item_of(items, count, e)];
    const int k = (int)(e - it.e0);
    it.lambda[k] = tri::bisect_one(it.n, it.n - 1 - k, it.a2, it.sc->g, it.sc->pivmin);
}

__global__ void bt_invit_kernel(const BItem* __restrict__ items, int count, long long total, int maxit) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const BItem& it = items[item_of(items, count, e)];
    if (!it.vectors) return;
    const int k = (int)(e - it.e0);
    const double ctol = fmin(1e-3, 10.0 / ((double)it.n * sqrt((double)it.n)));
    tri::invit_cluster(it.n, it.nev, it.alpha, it.lambda, it.sc->g, ctol, maxit, it.bf, it.Qi, it.fail, k);
}

// One CTA per matrix: eigenvector k of S (interleaved Qi) -> D map -> X_k, Y_k,
// then Z <- H_0 H_1 ... H_{n-3} Z.  Warp w takes columns w, w + 8, ... of
// [X Y] and keeps one column in registers (lane l holds rows l + 32 r, r < BR).
// G = false: the reflectors are staged in shared memory; G = true: read from
// global memory (L2).
template <int BR, bool G>
__global__ void __launch_bounds__(BT) bt_back_kernel(const BItem* __restrict__ items, const int* __restrict__ order) {
    extern __shared__ double bsm[];
    const BItem it = items[order[blockIdx.x]];
    const int n = it.n, nev = it.nev, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0 && it.info) *it.info = (*it.fail < nev) ? SKEW_INFO_INVIT_BASE + *it.fail : 0;
    if (!it.vectors || nev == 0) return;
    const double* Vs = it.V;  // n x n, reflector c in column c (rows c+1..)
    const double* ts = it.tau;
    if (!G) {
        double* V2 = bsm;
        double* t2 = V2 + (size_t)n * n;
        for (int e = t; e < n * n; e += BT) {
            const int i = e % n, c = e / n;
            V2[e] = (c + 2 < n && i > c) ? it.V[e] : 0.0;
        }
        for (int c = t; c < n; c += BT) t2[c] = (c + 2 < n) ? it.tau[c] : 0.0;
        __syncthreads();
        Vs = V2;
        ts = t2;
    }
    for (int col = warp; col < 2 * nev; col += BT / 32) {
        const int k = col % nev, part = col / nev;  // part 0: X = Re, 1: Y = Im
        double z[BR];
#pragma unroll
        for (int r = 0; r < BR; r++) {
            const int i = lane + 32 * r;
            double q = (i < n) ? it.Qi[(size_t)i * nev + k] : 0.0;
            const int m4 = i & 3;  // i^i: 1, i, -1, -i
            z[r] = (part == 0) ? (m4 == 0 ? q : (m4 == 2 ? -q : 0.0)) : (m4 == 1 ? q : (m4 == 3 ? -q : 0.0));
        }
        for (int c = n - 3; c >= 0; c--) {
            const double tau = ts[c];
            if (tau == 0.0) continue;
            const double* vc = Vs + (size_t)c * n;
            double d = 0.0;
#pragma unroll
            for (int r = 0; r < BR; r++) {
                const int i = lane + 32 * r;
                if (i > c && i < n) d = fma(vc[i], z[r], d);
            }
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            d *= tau;
#pragma unroll
            for (int r = 0; r < BR; r++) {
                const int i = lane + 32 * r;
                if (i > c && i < n) z[r] = fma(-d, vc[i], z[r]);
            }
        }
        double* out = (part == 0 ? it.Zre : it.Zim) + (size_t)k * n;
#pragma unroll
        for (int r = 0; r < BR; r++) {
            const int i = lane + 32 * r;
            if (i < n) out[i] = z[r];
        }
    }
}

struct BCarve {
    std::vector<BItem> items;
    std::vector<int> order;
    BItem* d_items;
    int* d_order;
    long long total;
    bool ok;
};

// Places every per-matrix buffer (base == nullptr: sizing only).
size_t carve_small(Carve& cv, int count, const BatchProblem* pr, BCarve* out) {
    std::vector<BItem> items((size_t)count);
    long long e0 = 0;
    BItem* d_items = cv.take<BItem>((size_t)(count > 0 ? count : 1));
    int* d_order = cv.take<int>((size_t)(count > 0 ? count : 1));
    for (int b = 0; b < count; b++) {
        const BatchProblem& q = pr[b];
        BItem& it = items[(size_t)b];
        const size_t n = (size_t)q.n, ne = (size_t)(q.nev > 0 ? q.nev : 1);
        it.n = q.n;
        it.nev = q.nev;
        it.lda = q.lda;
        it.vectors = q.Zre != nullptr;
        it.A = q.A;
        it.lambda = q.lambda;
        it.Zre = q.Zre;
        it.Zim = q.Zim;
        it.info = q.info;
        it.S = (q.n > BATCH_SMALL_MAX) ? cv.take<double>(n * n) : nullptr;
        it.V = cv.take<double>(n * n);
        it.tau = cv.take<double>(n);
        it.alpha = cv.take<double>(n);
        it.a2 = cv.take<double>(n);
        it.sc = cv.take<tri::TriScalars>(1);
        it.fail = cv.take<int>(1);
        if (it.vectors) {
            it.Qi = cv.take<double>(n * ne);
            it.bf.u0 = cv.take<double>(n * ne);
            it.bf.u1 = cv.take<double>(n * ne);
            it.bf.u2 = cv.take<double>(n * ne);
            it.bf.ml = cv.take<double>(n * ne);
            it.bf.sw = cv.take<unsigned char>(n * ne);
        }
        it.e0 = e0;
        e0 += q.nev;
    }
    if (out) {
        out->items = std::move(items);
        out->d_items = d_items;
        out->d_order = d_order;
        out->total = e0;
    }
    return cv.off;
}

size_t smem_reduce(int n) { return sizeof(double) * ((size_t)n * (n + 1) + 2 * (size_t)n + 32); }
size_t smem_back(int n) { return sizeof(double) * ((size_t)n * n + (size_t)n); }

}  // namespace

size_t batched_small_ws(int count, const BatchProblem* pr) {
    Carve cv(nullptr, ~size_t(0));
    carve_small(cv, count, pr, nullptr);
    return cv.off + 256;
}

int batched_small(cudaStream_t st, int count, const BatchProblem* pr, void* ws, size_t ws_bytes, int maxit) {
    if (count <= 0) return 0;
    for (int b = 0; b < count; b++)
        if (pr[b].n < 2 || pr[b].n > BATCH_MAX) return SKEW_ERR_UNSUPPORTED;
    Carve cv(ws, ws_bytes);
    BCarve bc{};
    carve_small(cv, count, pr, &bc);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    // per-matrix launches by class, each listing its matrices largest first:
    // [0, n1) shared-memory path, then the global-memory path by rows per lane
    // of the back-transform (8, 16, 32: n <= 256, 512, 1024)
    bc.order.resize((size_t)count);
    for (int b = 0; b < count; b++) bc.order[(size_t)b] = b;
    std::stable_sort(bc.order.begin(), bc.order.end(), [&](int x, int y) { return pr[x].n > pr[y].n; });
    auto cls = [&](int n) { return n <= BATCH_SMALL_MAX ? 0 : (n <= 256 ? 1 : (n <= 512 ? 2 : 3)); };
    std::stable_sort(bc.order.begin(), bc.order.end(), [&](int x, int y) { return cls(pr[x].n) < cls(pr[y].n); });
    int first[5] = {0, 0, 0, 0, 0};
    for (int c = 0; c < 4; c++) {
        first[c + 1] = first[c];
        while (first[c + 1] < count && cls(pr[bc.order[(size_t)first[c + 1]]].n) == c) first[c + 1]++;
    }
    // pageable copies: the host vectors may go once the calls return
    if (const cudaError_t e = cudaMemcpyAsync(bc.d_items, bc.items.data(), sizeof(BItem) * (size_t)count,
                                              cudaMemcpyHostToDevice, st))
        return cuda_fail(e);
    if (const cudaError_t e = cudaMemcpyAsync(bc.d_order, bc.order.data(), sizeof(int) * (size_t)count,
                                              cudaMemcpyHostToDevice, st))
        return cuda_fail(e);
    int nmax_small = 2, nmax = 2;
    for (int b = 0; b < count; b++) {
        nmax = pr[b].n > nmax ? pr[b].n : nmax;
        if (pr[b].n <= BATCH_SMALL_MAX) nmax_small = pr[b].n > nmax_small ? pr[b].n : nmax_small;
    }
    const int nsmall = first[1], nlarge = count - first[1];
    if (nsmall > 0) {
        const size_t s1 = smem_reduce(nmax_small);
        cudaFuncSetAttribute(bt_reduce_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1);
        bt_reduce_kernel<false><<<nsmall, BT, s1, st>>>(bc.d_items, bc.d_order);
        count_launch();
    }
    if (nlarge > 0) {
        const size_t s1 = sizeof(double) * (2 * (size_t)nmax + 32);
        cudaFuncSetAttribute(bt_reduce_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1);
        bt_reduce_kernel<true><<<nlarge, BT, s1, st>>>(bc.d_items, bc.d_order + first[1]);
        count_launch();
    }
    if (bc.total > 0) {
        const unsigned g = (unsigned)((bc.total + 127) / 128);
        bt_bisect_kernel<<<g, 128, 0, st>>>(bc.d_items, count, bc.total);
        const unsigned g2 = (unsigned)((bc.total + 63) / 64);
        bt_invit_kernel<<<g2, 64, 0, st>>>(bc.d_items, count, bc.total, maxit);
        count_launch(2);
    }
    if (nsmall > 0) {
        const size_t s2 = smem_back(nmax_small);
        cudaFuncSetAttribute(bt_back_kernel<(BATCH_SMALL_MAX + 31) / 32, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2);
        bt_back_kernel<(BATCH_SMALL_MAX + 31) / 32, false><<<nsmall, BT, s2, st>>>(bc.d_items, bc.d_order);
        count_launch();
    }
    if (first[2] > first[1]) {
        bt_back_kernel<8, true><<<first[2] - first[1], BT, 0, st>>>(bc.d_items, bc.d_order + first[1]);
        count_launch();
    }
    if (first[3] > first[2]) {
        bt_back_kernel<16, true><<<first[3] - first[2], BT, 0, st>>>(bc.d_items, bc.d_order + first[2]);
        count_launch();
    }
    if (first[4] > first[3]) {
        bt_back_kernel<32, true><<<first[4] - first[3], BT, 0, st>>>(bc.d_items, bc.d_order + first[3]);
        count_launch();
    }
    return cuda_ok(cudaGetLastError());
}

}  // namespace sk
