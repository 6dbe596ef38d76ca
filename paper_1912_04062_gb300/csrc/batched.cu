// batched.cu -- many independent skew eigenproblems of small and medium order
// in ONE persistent launch (the paper solves one matrix per run; this is the
// batched form of the same route for orders up to BATCH_MAX = 1024).
//
// Every CTA of the launch (ctas_per_sm per SM) takes matrices from a device
// work counter over a list sorted largest first (longest-processing-time
// order) and runs the whole route for each one: it tridiagonalises the skew
// matrix column by column with Householder reflectors (dlarfg convention; the
// skew two-sided update A <- A + v p^T - p v^T with p = tau A v, Eqs. 2-6 with
// u1 = -u2, whose 1/2 tau^2 (v^T A v) v term is 0 for skew A), giving
// alpha_c = T[c, c+1] (Lemma 1); bisects every wanted eigenvalue and runs
// inverse iteration (Sec. 3), one thread per eigenvalue; then applies the D
// map (Algorithm 1 step 3) and the reflectors in reverse order to the
// eigenvectors.  Orders up to smem_max_n keep the working matrix in shared
// memory; larger ones work on a copy in global memory (L2).  ctas_per_sm and
// smem_max_n are the launch's tunables (skew_batched_config; chosen per GPU by
// timing the candidates on the batch, skew_batched_plan_tune).
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
    double* S;                   // global working matrix (n x n), used when n > the launch's smem_max_n
    const double* A;
    double *lambda, *Zre, *Zim;  // Z: n x nev, leading dimension n
    int* info;                   // caller's status word of this matrix (may be null)
    // per-matrix scratch
    double *V, *tau, *alpha, *a2, *Qi;
    double *a2e, *b2e;  // the bidiagonal of the zero-diagonal form, squared (ceil(n/2) each)
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

// Tridiagonalisation of one matrix by the whole CTA.  S: the working matrix
// (shared memory, ld n + 1, or the matrix's global copy, ld n); v, p: n
// doubles of shared memory; red: 32 doubles of shared memory.
__device__ void bt_reduce_body(const BItem& it, double* S, int ld, double* v, double* p, double* red) {
    const int n = it.n, t = threadIdx.x;
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
            // S22 += v p^T - p v^T: each product is rounded on its own, so the
            // update of (j, i) is exactly minus that of (i, j); the strict lower
            // triangle is computed and its negation stored above (the diagonal
            // stays 0), which keeps S exactly skew with half the FP64 work of
            // updating the whole square, and the same values
            const int m = n - c - 1;
            for (int e = t; e < m * m; e += BT) {
                const int i = c + 1 + e % m, j = c + 1 + e / m;
                if (i > j) {
                    const double x =
                        S[i + (size_t)j * ld] + __dsub_rn(__dmul_rn(v[i], p[j]), __dmul_rn(p[i], v[j]));
                    S[i + (size_t)j * ld] = x;
                    S[j + (size_t)i * ld] = -x;
                }
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
    // the zero-diagonal form's bidiagonal: a_i = alpha_{2i}, b_i = alpha_{2i+1}
    for (int i = t; i < (n + 1) / 2; i += BT) {
        const double a = (2 * i <= n - 2) ? it.alpha[2 * i] : 0.0;
        const double b = (2 * i + 1 <= n - 2) ? it.alpha[2 * i + 1] : 0.0;
        it.a2e[i] = a * a;
        it.b2e[i] = b * b;
    }
    gm = block_max(gm, red);
    am = block_max(am, red);
    if (t == 0) {
        it.sc->g = gm;
        it.sc->pivmin = DBL_MIN * fmax(1.0, am);
        *it.fail = 0x7fffffff;
    }
    __syncthreads();
}

// Eigenvector k of S (interleaved Qi) -> D map -> X_k, Y_k, then
// Z <- H_0 H_1 ... H_{n-3} Z, by the whole CTA.  Warp w takes columns w,
// w + 8, ... of [X Y] and keeps one column in registers (lane l holds rows
// l + 32 r, r < BR).  G = false: the reflectors are staged in shared memory
// (bsm, n^2 + n doubles); G = true: read from global memory (L2).
template <int BR, bool G>
__device__ void bt_back_body(const BItem& it, double* bsm) {
    const int n = it.n, nev = it.nev, t = threadIdx.x, lane = t & 31, warp = t >> 5;
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

// The persistent launch: CTAs take matrices from *next over order[] (largest
// first) until the list is exhausted; each matrix goes through the whole route
// in one CTA.  MINB = CTAs per SM the registers are budgeted for.
template <int MINB>
__global__ void __launch_bounds__(BT, MINB)
bt_persistent_kernel(const BItem* __restrict__ items, const int* __restrict__ order, int count,
                     int* __restrict__ next, int smem_n, int maxit) {
    extern __shared__ double bsm[];
    __shared__ int s_q;
    const int t = threadIdx.x;
    for (;;) {
        __syncthreads();  // the previous matrix is finished with shared memory and s_q
        if (t == 0) s_q = atomicAdd(next, 1);
        __syncthreads();
        const int q = s_q;
        if (q >= count) break;
        const BItem it = items[order[q]];
        const int n = it.n, nev = it.nev;
        const bool in_smem = n <= smem_n;
        if (in_smem) {
            double* S = bsm;
            double* v = S + (size_t)n * (n + 1);
            bt_reduce_body(it, S, n + 1, v, v + n, v + 2 * n);
        } else {
            bt_reduce_body(it, it.S, n, bsm, bsm + n, bsm + 2 * n);
        }
        // every wanted eigenvalue of this matrix (Sturm bisection), then
        // inverse iteration per cluster leader
        // (counts on the zero-diagonal form: ceil(n/2) steps; nev <= n/2)
        for (int k = t; k < nev; k += BT)
            it.lambda[k] = tri::bisect_one_bd((n + 1) / 2, k, it.a2e, it.b2e, it.sc->g, it.sc->pivmin);
        __syncthreads();
        if (it.vectors) {
            const double ctol = fmin(1e-3, 10.0 / ((double)n * sqrt((double)n)));
            for (int k = t; k < nev; k += BT)
                tri::invit_cluster(n, nev, it.alpha, it.lambda, it.sc->g, ctol, maxit, it.bf, it.Qi, it.fail, k);
        }
        __syncthreads();
        if (t == 0 && it.info) *it.info = (*it.fail < nev) ? SKEW_INFO_INVIT_BASE + *it.fail : 0;
        if (it.vectors && nev > 0) {
            if (in_smem) bt_back_body<(BATCH_SMALL_MAX + 31) / 32, false>(it, bsm);
            else if (n <= BATCH_SMALL_MAX) bt_back_body<(BATCH_SMALL_MAX + 31) / 32, true>(it, bsm);
            else if (n <= 256) bt_back_body<8, true>(it, bsm);
            else if (n <= 512) bt_back_body<16, true>(it, bsm);
            else bt_back_body<32, true>(it, bsm);
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
        // global working copy: used whenever the launch keeps this order out
        // of shared memory (the threshold is a launch parameter, 0..160)
        it.S = cv.take<double>(n * n);
        it.V = cv.take<double>(n * n);
        it.tau = cv.take<double>(n);
        it.alpha = cv.take<double>(n);
        it.a2 = cv.take<double>(n);
        it.a2e = cv.take<double>(n / 2 + 1);
        it.b2e = cv.take<double>(n / 2 + 1);
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

}  // namespace

size_t batched_small_ws(int count, const BatchProblem* pr) {
    Carve cv(nullptr, ~size_t(0));
    carve_small(cv, count, pr, nullptr);
    cv.take<int>(1);  // work counter of the persistent launch
    return cv.off + 256;
}

namespace {

// Largest order kept in shared memory for a given shared-memory budget per CTA.
int smem_n_for(size_t budget) {
    int n = 2;
    while (n < BATCH_SMALL_MAX && smem_reduce(n + 1) <= budget) n++;
    return n;
}

template <int MINB>
int prepare_persistent(int smem_n, int nmax, int count, BatchLaunch* out) {
    const size_t dyn_global = sizeof(double) * (2 * (size_t)nmax + 32);
    const size_t dyn = smem_n >= 2 ? std::max(smem_reduce(smem_n), dyn_global) : dyn_global;
    auto kern = bt_persistent_kernel<MINB>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
        return SKEW_ERR_LAUNCH;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, BT, dyn) != cudaSuccess || occ < 1)
        return SKEW_ERR_LAUNCH;
    const int per_sm = occ < MINB ? occ : MINB;
    int grid = per_sm * device_sms();
    if (grid > count) grid = count;
    out->ctas = MINB;
    out->grid = grid;
    out->dyn = dyn;
    out->smem_n = smem_n;
    return 0;
}

}  // namespace

skew_batched_config& batched_default_config() {
    static skew_batched_config c{2, 112, {0, 0}};
    return c;
}

int batched_config_check(const skew_batched_config& c) {
    if (c.ctas_per_sm < 1 || c.ctas_per_sm > 4) return -1;
    if (c.smem_max_n < 0 || c.smem_max_n > BATCH_SMALL_MAX) return -2;
    return 0;
}

// Launch parameters of the persistent kernel for a configuration (sets the
// kernel's shared-memory attribute; no stream work).
int batched_prepare(const BatchPlanDev& d, const skew_batched_config& cfg, BatchLaunch* out) {
    if (batched_config_check(cfg)) return SKEW_ERR_UNSUPPORTED;
    // the shared-memory threshold cannot exceed what the per-SM budget allows
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const size_t budget = (size_t)smem_sm / (size_t)cfg.ctas_per_sm - 2048;
    int smem_n = cfg.smem_max_n;
    if (smem_n >= 2) smem_n = std::min(smem_n, smem_n_for(budget));
    const int cnt = d.count > 0 ? d.count : 1;
    switch (cfg.ctas_per_sm) {
    case 1: return prepare_persistent<1>(smem_n, d.nmax, cnt, out);
    case 2: return prepare_persistent<2>(smem_n, d.nmax, cnt, out);
    case 3: return prepare_persistent<3>(smem_n, d.nmax, cnt, out);
    default: return prepare_persistent<4>(smem_n, d.nmax, cnt, out);
    }
}

// Stream work only: clear the work counter, launch (capturable).
int batched_exec(cudaStream_t st, const BatchPlanDev& d, const BatchLaunch& L, int maxit) {
    if (d.count <= 0) return 0;
    if (cudaMemsetAsync(d.next, 0, sizeof(int), st) != cudaSuccess) return SKEW_ERR_CUDA;
    const BItem* items = static_cast<const BItem*>(d.items);
    switch (L.ctas) {
    case 1: bt_persistent_kernel<1><<<L.grid, BT, L.dyn, st>>>(items, d.order, d.count, d.next, L.smem_n, maxit); break;
    case 2: bt_persistent_kernel<2><<<L.grid, BT, L.dyn, st>>>(items, d.order, d.count, d.next, L.smem_n, maxit); break;
    case 3: bt_persistent_kernel<3><<<L.grid, BT, L.dyn, st>>>(items, d.order, d.count, d.next, L.smem_n, maxit); break;
    default: bt_persistent_kernel<4><<<L.grid, BT, L.dyn, st>>>(items, d.order, d.count, d.next, L.smem_n, maxit);
    }
    count_launch();
    return cuda_ok(cudaGetLastError());
}

int batched_launch(cudaStream_t st, const BatchPlanDev& d, const skew_batched_config& cfg, int maxit) {
    if (d.count <= 0) return 0;
    BatchLaunch L{};
    if (const int rc = batched_prepare(d, cfg, &L)) return rc;
    return batched_exec(st, d, L, maxit);
}

// Places the item table in the workspace and uploads it (synchronously with
// respect to the host buffers: pageable copies).
int batched_upload(cudaStream_t st, int count, const BatchProblem* pr, void* ws, size_t ws_bytes, BatchPlanDev* out) {
    if (count <= 0) return 0;
    for (int b = 0; b < count; b++)
        if (pr[b].n < 2 || pr[b].n > BATCH_MAX) return SKEW_ERR_UNSUPPORTED;
    Carve cv(ws, ws_bytes);
    BCarve bc{};
    carve_small(cv, count, pr, &bc);
    int* d_next = cv.take<int>(1);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    // longest processing time first: largest order first
    bc.order.resize((size_t)count);
    for (int b = 0; b < count; b++) bc.order[(size_t)b] = b;
    std::stable_sort(bc.order.begin(), bc.order.end(), [&](int x, int y) { return pr[x].n > pr[y].n; });
    if (const cudaError_t e = cudaMemcpyAsync(bc.d_items, bc.items.data(), sizeof(BItem) * (size_t)count,
                                              cudaMemcpyHostToDevice, st))
        return cuda_fail(e);
    if (const cudaError_t e = cudaMemcpyAsync(bc.d_order, bc.order.data(), sizeof(int) * (size_t)count,
                                              cudaMemcpyHostToDevice, st))
        return cuda_fail(e);
    out->items = bc.d_items;
    out->order = bc.d_order;
    out->next = d_next;
    out->count = count;
    out->nmax = 2;
    for (int b = 0; b < count; b++) out->nmax = pr[b].n > out->nmax ? pr[b].n : out->nmax;
    return 0;
}

int batched_small(cudaStream_t st, int count, const BatchProblem* pr, void* ws, size_t ws_bytes, int maxit) {
    if (count <= 0) return 0;
    BatchPlanDev d{};
    if (const int rc = batched_upload(st, count, pr, ws, ws_bytes, &d)) return rc;
    return batched_launch(st, d, batched_default_config(), maxit);
}

}  // namespace sk
