// skeweig.cu -- C ABI of the skew-symmetric eigensolver: argument checks,
// workspace carve-up and the stage sequence of Algorithm 1 (two-step form) on
// one stream.
#include <atomic>
#include <cstdint>
#include <mutex>
#include <vector>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace sk {
namespace {

__global__ void copy_lower_kernel(int n, const double* __restrict__ A, int lda, double* __restrict__ W, int ldw,
                                  int check, int* status) {
    size_t total = (size_t)n * n;
    bool bad = false;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        double v = 0.0;
        if (i > j) {
            v = A[(size_t)j * lda + i];
            if (check && !isfinite(v)) bad = true;
        }
        W[(size_t)j * ldw + i] = v;
    }
    if (bad) sk_set_error(status, SKEW_ERR_NONFINITE);
}

__global__ void split_z_kernel(int n, int nev, const double* __restrict__ Z, int ldzw, double* __restrict__ Zre,
                               double* __restrict__ Zim, int ldz) {
    size_t total = (size_t)n * nev;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        Zre[(size_t)j * ldz + i] = Z[(size_t)j * ldzw + i];
        Zim[(size_t)j * ldz + i] = Z[(size_t)(j + nev) * ldzw + i];
    }
}

__global__ void store_status_kernel(const int* status, int* d_info) {
    if (threadIdx.x == 0) *d_info = *status;
}

__global__ void zero_int_kernel(int* p) {
    if (threadIdx.x == 0) *p = 0;
}

// d_info = the first nonzero of status[0] (driver) and status[1] (skew solve)
__global__ void bse_status_kernel(const int* status, int* d_info) {
    if (threadIdx.x == 0) *d_info = status[0] ? status[0] : status[1];
}

inline int grid_for(size_t total) {
    size_t g = (total + 255) / 256;
    return (int)(g > 16384 ? 16384 : (g == 0 ? 1 : g));
}

struct Plan {
    int n, nev, b, P, K, nsw;
    bool vectors, mixed;
    int planes;       // split-BF16 planes of the mixed form (0 in the FP64 form)
    int reduce_prec;  // band reduction: 0 FP64, 2/3 split planes, REDUCE_F64ACC digit slices
    int qband_prec;   // mixed Q_band: 2/3 split planes or REDUCE_F64ACC digit slices
    int reduce_slices, qband_slices;  // digit slices of the REDUCE_F64ACC products
    bool qtrd_f32;    // mixed Q_trd in FP32 arithmetic (else FP64)
    bool qtrd_tc;     // the FP32-level Q_trd on the tensor cores (else SIMT)
    bool qtrd_df;     // Q_trd in double-float on the FP32 pipe (FP64 data)
    size_t ldab;
    // carved pointers
    double *W, *Tfac, *AB, *Vtrd, *tautrd, *alpha, *Qi, *Z;
    float *Z32, *V32, *tau32;  // FP32 Q_trd: Z and the chase's reflectors (sweep stride padded to 64)
    int* status;
    void *ws_reduce, *ws_chase, *ws_tri, *ws_qband, *ws_refine, *ws_qtc;
    size_t sz_reduce, sz_chase, sz_tri, sz_qband, sz_refine, sz_qtc;
    bool refine;  // mixed form with a complete basis (n even, nev = n/2)
};

// One carve-up routine serves both sizing (base == nullptr) and placement.
bool carve_plan(Plan& p, Carve& cv) {
    const size_t n = (size_t)p.n, b = (size_t)p.b;
    const size_t nn = n ? n : 1;
    p.status = cv.take<int>(16);
    p.W = cv.take<double>(nn * nn);
    p.Tfac = cv.take<double>((size_t)(p.P ? p.P : 1) * b * b);
    p.ldab = 2 * b + 1;
    p.AB = cv.take<double>(p.ldab * nn);
    const size_t nsw = (size_t)(p.nsw > 0 ? p.nsw : 1), K = (size_t)(p.K > 0 ? p.K : 1);
    p.Vtrd = cv.take<double>(K * nsw * b);
    p.tautrd = cv.take<double>(K * nsw);
    p.alpha = cv.take<double>(nn);
    const size_t ne = (size_t)(p.nev ? p.nev : 1);
    p.Qi = p.vectors ? cv.take<double>(nn * ne) : nullptr;
    p.Z = p.vectors ? cv.take<double>(nn * 2 * ne) : nullptr;
    p.Z32 = (p.vectors && p.qtrd_f32) ? cv.take<float>(nn * 2 * ne) : nullptr;
    const size_t nsw64 = (nsw + 63) / 64 * 64;
    p.V32 = (p.vectors && p.qtrd_f32) ? cv.take<float>(K * nsw64 * b) : nullptr;
    p.tau32 = (p.vectors && p.qtrd_f32) ? cv.take<float>(K * nsw64) : nullptr;
    p.sz_reduce = band_reduce_ws(p.n, p.b, p.reduce_prec);
    p.ws_reduce = cv.take<char>(p.sz_reduce);
    p.sz_chase = chase_ws(p.n, p.b);
    p.ws_chase = cv.take<char>(p.sz_chase);
    p.sz_tri = tridiag_ws(p.n, p.nev);
    p.ws_tri = cv.take<char>(p.sz_tri);
    p.sz_qband = p.vectors ? (p.mixed ? qband_mixed_ws(p.n, p.b, 2 * p.nev, p.qband_prec)
                                      : qband_ws(p.n, p.b, 2 * p.nev))
                           : 0;
    p.ws_qband = p.vectors ? cv.take<char>(p.sz_qband) : nullptr;
    p.sz_refine = p.refine ? refine_ws(p.n) : 0;
    p.ws_refine = p.refine ? cv.take<char>(p.sz_refine) : nullptr;
    p.sz_qtc = p.qtrd_tc ? qtrd_tc_ws(p.n) : 0;
    p.ws_qtc = p.qtrd_tc ? cv.take<char>(p.sz_qtc) : nullptr;
    return cv.ok;
}

Plan make_plan(int n, int nev, const skew_opts* o, bool vectors) {
    Plan p{};
    p.n = n;
    p.nev = nev;
    p.b = (o && o->band > 0) ? o->band : 64;
    p.P = num_panels(n, p.b);
    p.K = chase_steps(n, p.b);
    p.nsw = n - 2;
    p.vectors = vectors;
    p.mixed = o && (o->mode == SKEW_MODE_MIXED_BF16X3 || o->mode == SKEW_MODE_MIXED_BF16X6 ||
                    o->mode == SKEW_MODE_MIXED_REFINED);
    p.planes = !p.mixed ? 0 : (o->mode == SKEW_MODE_MIXED_BF16X3 ? 2 : 3);
    // the reduction's contractions in the refined mode are FP64-accurate
    p.reduce_prec = !p.mixed ? 0 : (o->mode == SKEW_MODE_MIXED_REFINED ? REDUCE_F64ACC : p.planes);
    p.refine = p.mixed && vectors && n % 2 == 0 && n >= 2 && nev == n / 2 && !(o->fault & SKEW_FAULT_NO_REFINE);
    // back-transforms: split products and FP32 Q_trd in the split modes; the
    // refined mode takes Q_band as FP64-accurate digit-slice products (the
    // refinement starts from vectors about 100x more orthogonal and saves an
    // iteration) and Q_trd in FP32, or in double-float (FP64-accurate) when
    // there is no complete basis to refine (nev < n/2, odd n)
    const bool refined_mode = p.mixed && o->mode == SKEW_MODE_MIXED_REFINED;
    p.qband_prec = !p.mixed ? 0 : (refined_mode ? REDUCE_F64ACC : p.planes);
    p.qtrd_f32 = p.mixed && vectors && !(refined_mode && !p.refine);
    if (o && vectors && (o->qtrd == SKEW_QTRD_FP32 || o->qtrd == SKEW_QTRD_TC)) p.qtrd_f32 = true;
    if (o && o->qtrd == SKEW_QTRD_FP64) p.qtrd_f32 = false;
    // FP32-level Q_trd on the tensor cores only when asked for: measured at
    // n = 16384 it is slower than the SIMT FP32 kernel (542 vs 436 ms) and
    // starts the refinement from a 24x larger orthogonality error
    p.qtrd_tc = p.qtrd_f32 && o && o->qtrd == SKEW_QTRD_TC;
    // without refinement the refined mode needs an FP64-accurate Q_trd: the
    // double-float kernel gives it on the FP32 pipe (the FP64 kernel on
    // request)
    if (o && vectors && o->qtrd == SKEW_QTRD_DF) {
        p.qtrd_df = true;
        p.qtrd_f32 = p.qtrd_tc = false;
    }
    if (vectors && refined_mode && !p.refine && (!o || o->qtrd == SKEW_QTRD_AUTO)) p.qtrd_df = true;
    // With a complete basis the refinement removes the first-order error, so
    // the products before it need only keep the starting vectors at the level
    // of the FP32 Q_trd: 6 digit slices (about 2^-42) for the reduction, 5
    // (2^-35) for Q_band; measured at n = 16384 (BSE), the refinement starts
    // from the same orthogonality (2.7e-4) and takes the same 3 iterations as
    // with 8.  Without refinement they stay FP64-accurate.
    p.reduce_slices = p.refine ? 6 : 8;
    p.qband_slices = p.refine ? 5 : 8;
    return p;
}

size_t plan_bytes(int n, int nev, const skew_opts* o, bool vectors) {
    Plan p = make_plan(n, nev, o, vectors);
    Carve cv(nullptr, ~size_t(0));
    carve_plan(p, cv);
    return cv.off + 256;
}

__global__ void f64_to_f32_kernel(size_t count, const double* __restrict__ x, float* __restrict__ y) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        y[e] = (float)x[e];
}
__global__ void f32_to_f64_kernel(size_t count, const float* __restrict__ x, double* __restrict__ y) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        y[e] = (double)x[e];
}

int check_args(int n, const void* A, int lda, int nev, const void* lambda, const void* Zre, const void* Zim) {
    if (n < 0) return -1;
    if (n > 0 && !A) return -2;
    if (lda < (n > 1 ? n : 1)) return -3;
    if (nev < 0 || nev > n / 2) return -4;
    if (nev > 0 && !lambda) return -5;
    if ((Zre == nullptr) != (Zim == nullptr)) return -6;
    return 0;
}

// Optional per-stage CUDA events recorded on the solve stream.
struct StageEvents {
    cudaEvent_t ev[SKEW_NSTAGES + 1];
};

int run_solve(cudaStream_t st, int n, const double* A, int lda, int nev, double* lambda, double* Zre, double* Zim,
              int ldz, const skew_opts* o, void* ws, size_t ws_bytes, int* d_info, StageEvents* prof = nullptr) {
    auto mark = [&](int i) {
        if (prof) cudaEventRecord(prof->ev[i], st);
    };
    const bool vectors = (Zre != nullptr);
    Plan p = make_plan(n, nev, o, vectors);
    if (p.b != 64) return SKEW_ERR_UNSUPPORTED;
    if (o && o->mode != SKEW_MODE_FP64 && !p.mixed) return SKEW_ERR_UNSUPPORTED;
    {
        Carve cv(ws, ws_bytes);
        if (!carve_plan(p, cv)) return SKEW_ERR_WORKSPACE;
    }
    const int maxit = (o && (o->fault & SKEW_FAULT_INVIT_NOCONV)) ? 0 : 5;
    const unsigned spin_cap = (o && (o->fault & SKEW_FAULT_TINY_WAIT)) ? SK_TINY_SPIN_CAP : 0;
    refine_stats_discard();
    last_refine_info() = RefineInfo{};  // iterations = 0 unless this solve refines

    mark(0);
    {
        KtScope kt(st, KT_OTHER);
        zero_int_kernel<<<1, 32, 0, st>>>(p.status);
        copy_lower_kernel<<<grid_for((size_t)n * n), 256, 0, st>>>(n, A, lda, p.W, n, o ? o->check_finite : 0,
                                                                   p.status);
    }
    count_launch(2);
    mark(1);
    int rc = band_reduce(st, n, p.W, n, p.b, p.Tfac, p.ws_reduce, p.sz_reduce, p.status, p.reduce_prec,
                         p.reduce_slices, spin_cap);
    if (rc) return rc;
    mark(2);
    if (band_pack(st, n, p.b, p.W, n, p.AB, (int)p.ldab) != cudaSuccess) return SKEW_ERR_CUDA;
    mark(3);
    if (p.tau32) {
        // FP32 reflector copies for Q_trd: the taus of steps a sweep does not
        // have stay zero (the FP64 copies are not needed then)
        const size_t nsw64 = ((size_t)p.nsw + 63) / 64 * 64;
        if (const cudaError_t e = cudaMemsetAsync(p.tau32, 0, sizeof(float) * (size_t)p.K * nsw64, st))
            return cuda_fail(e);
        rc = chase(st, n, p.b, p.AB, (int)p.ldab, p.alpha, nullptr, nullptr, p.ws_chase, p.sz_chase, p.status,
                   spin_cap, p.V32, p.tau32);
    } else {
        rc = chase(st, n, p.b, p.AB, (int)p.ldab, p.alpha, p.Vtrd, p.tautrd, p.ws_chase, p.sz_chase, p.status,
                   spin_cap);
    }
    if (rc) return rc;
    mark(4);
    // with refinement the eigenvalues are recomputed from the Rayleigh
    // quotients: the double-float brackets suffice to start from
    rc = tridiag_eig(st, n, p.alpha, nev, lambda, vectors ? p.Qi : nullptr, p.ws_tri, p.sz_tri, p.status, maxit,
                     !p.refine, !(o && o->tridiag == SKEW_TRIDIAG_FULL));
    if (rc) return rc;
    mark(5);
    if (vectors) {
        // Algorithm 1 step 3 (D map) fused with the interleaved -> column-major
        // move; Z = [X | Y] is n x 2 nev with leading dimension n.
        KtScope kt(st, KT_OTHER);
        if (interleaved_to_colmajor(st, n, nev, p.Qi, p.Z, p.Z + (size_t)n * nev, n, true) != cudaSuccess)
            return SKEW_ERR_CUDA;
    }
    mark(6);
    if (vectors && p.qtrd_df) {
        if (apply_qtrd_df(st, n, p.b, p.Vtrd, p.tautrd, p.Z, n, 2 * nev, p.status) != cudaSuccess)
            return SKEW_ERR_CUDA;
    } else if (vectors && !p.qtrd_f32) {
        if (apply_qtrd(st, n, p.b, p.Vtrd, p.tautrd, p.Z, n, 2 * nev) != cudaSuccess) return SKEW_ERR_CUDA;
    } else if (vectors) {
        // mixed form: Q_trd in FP32 arithmetic (the chase's FP32 reflector copies)
        const size_t cnt = (size_t)n * 2 * nev;
        {
            KtScope kt(st, KT_OTHER);
            f64_to_f32_kernel<<<grid_for(cnt), 256, 0, st>>>(cnt, p.Z, p.Z32);
        }
        count_launch();
        if (p.qtrd_tc) {
            rc = apply_qtrd_tc(st, n, p.V32, p.tau32, p.Z32, n, 2 * nev, p.ws_qtc, p.sz_qtc, p.status);
            if (rc) return rc;
        } else if (apply_qtrd_f32(st, n, p.b, p.V32, p.tau32, p.Z32, n, 2 * nev, p.status) != cudaSuccess) {
            return SKEW_ERR_CUDA;
        }
        {
            KtScope kt(st, KT_OTHER);
            f32_to_f64_kernel<<<grid_for(cnt), 256, 0, st>>>(cnt, p.Z32, p.Z);
        }
        count_launch();
    }
    mark(7);
    if (vectors) {
        rc = p.mixed ? apply_qband_mixed(st, n, p.b, p.W, n, p.Tfac, p.Z, n, 2 * nev, p.ws_qband, p.sz_qband, p.status,
                                         p.qband_prec, p.qband_slices)
                     : apply_qband(st, n, p.b, p.W, n, p.Tfac, p.Z, n, 2 * nev, p.ws_qband, p.sz_qband);
        if (rc) return rc;
    }
    mark(8);
    if (p.refine) {
        const int iters = (o && o->refine_iters > 0) ? (o->refine_iters < 8 ? o->refine_iters : 8) : 8;
        const double rho = (o && o->refine_rho > 0) ? (double)o->refine_rho : 1024.0;
        rc = refine(st, n, A, lda, lambda, p.Z, iters, p.ws_refine, p.sz_refine, p.status, &last_refine_info(), rho);
        if (rc) return rc;
    }
    mark(9);
    if (vectors) {
        KtScope kt(st, KT_OTHER);
        split_z_kernel<<<grid_for((size_t)n * nev), 256, 0, st>>>(n, nev, p.Z, n, Zre, Zim, ldz);
        count_launch();
    }
    if (d_info) {
        store_status_kernel<<<1, 32, 0, st>>>(p.status, d_info);
        count_launch();
    }
    mark(10);
    return cuda_ok(cudaGetLastError());
}

std::atomic<long long> g_launches{0};

}  // namespace

void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
RefineInfo& last_refine_info() {
    static RefineInfo info{};
    return info;
}
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {
struct KtRec {
    cudaEvent_t a, b;
    int kind;
    double flops;
};
struct KTimer {
    bool on = false;
    size_t used = 0;
    std::vector<KtRec> recs;  // events are created on first use and reused
    // per-kind totals of the records folded so far (kt_fold)
    double ms[KT_KINDS] = {}, fl[KT_KINDS] = {};
    long long cnt[KT_KINDS] = {};
    long long dropped = 0;  // launches not recorded because the pool was full
    // timeline of the records folded last: kind, start and end (ms after the
    // first of them)
    std::vector<int> tl_kind;
    std::vector<double> tl_a, tl_b;
    void clear() {
        used = 0;
        for (int k = 0; k < KT_KINDS; k++) ms[k] = fl[k] = 0.0, cnt[k] = 0;
        dropped = 0;
        tl_kind.clear();
        tl_a.clear();
        tl_b.clear();
    }
};
KTimer& ktimer() {
    static KTimer t;
    return t;
}
constexpr size_t KT_CAP = 16384;

// Waits for the outstanding records, adds them to the per-kind totals, keeps
// their timeline and frees the pool.  Returns 0 or SKEW_ERR_CUDA.
int kt_fold() {
    KTimer& t = ktimer();
    if (t.used == 0) return 0;
    t.tl_kind.clear();
    t.tl_a.clear();
    t.tl_b.clear();
    const cudaEvent_t t0 = t.recs[0].a;
    for (size_t i = 0; i < t.used; i++) {
        const KtRec& r = t.recs[i];
        if (cudaEventSynchronize(r.b) != cudaSuccess) return SKEW_ERR_CUDA;
        float e = 0.f, a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&e, r.a, r.b) != cudaSuccess) return SKEW_ERR_CUDA;
        if (cudaEventElapsedTime(&a, t0, r.a) != cudaSuccess) return SKEW_ERR_CUDA;
        if (cudaEventElapsedTime(&b, t0, r.b) != cudaSuccess) return SKEW_ERR_CUDA;
        if (r.kind >= 0 && r.kind < KT_KINDS) {
            t.ms[r.kind] += e;
            t.fl[r.kind] += r.flops;
            t.cnt[r.kind]++;
        }
        t.tl_kind.push_back(r.kind);
        t.tl_a.push_back(a);
        t.tl_b.push_back(b);
    }
    t.used = 0;
    return 0;
}
}  // namespace

int g_kt_ozaki_kind = KT_OZAKI;

namespace {
std::atomic<const char*> g_last_cuda_error{"none"};
}
int cuda_fail(cudaError_t e) {
    if (e != cudaSuccess) g_last_cuda_error.store(cudaGetErrorName(e), std::memory_order_relaxed);
    return SKEW_ERR_CUDA;
}

bool kt_enabled() { return ktimer().on; }

int kt_begin(cudaStream_t st) {
    KTimer& t = ktimer();
    if (!t.on) return -1;
    if (t.used == t.recs.size()) {
        if (t.recs.size() >= KT_CAP) {
            t.dropped++;
            return -1;
        }
        KtRec r{};
        if (cudaEventCreate(&r.a) != cudaSuccess) return -1;
        if (cudaEventCreate(&r.b) != cudaSuccess) {
            cudaEventDestroy(r.a);
            return -1;
        }
        t.recs.push_back(r);
    }
    const int slot = (int)t.used;
    if (cudaEventRecord(t.recs[slot].a, st) != cudaSuccess) return -1;
    t.used++;
    return slot;
}

void kt_end(cudaStream_t st, int slot, int kind, double flops) {
    if (slot < 0) return;
    KTimer& t = ktimer();
    t.recs[slot].kind = kind;
    t.recs[slot].flops = flops;
    if (cudaEventRecord(t.recs[slot].b, st) != cudaSuccess) t.recs[slot].kind = -1;
}

}  // namespace sk

using namespace sk;

namespace {

// Library-owned stream-ordered memory pools, one per device, created on first
// use.  Their release threshold is unlimited: a workspace freed by a completed
// call stays reserved for the next call on that device, so repeated solves do
// not map tens of GB of fresh pages each time.  skew_release_memory() returns
// the reserved memory.
constexpr int MAX_POOL_DEVICES = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[MAX_POOL_DEVICES] = {};

int stream_device(cudaStream_t st, int* dev) {
    if (st) {
        if (cudaStreamGetDevice(st, dev) == cudaSuccess) return 0;
        cudaGetLastError();
    }
    return cudaGetDevice(dev) == cudaSuccess ? 0 : -1;
}

cudaMemPool_t lib_pool(int dev) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}

// Stream-ordered workspace for the allocating entry points: the device's
// library pool (the default pool if it cannot be had).  SKEW_FAULT_NOMEM in
// opts makes it fail without allocating (tests of the error path).
int lib_alloc(void** ptr, size_t bytes, cudaStream_t st, const skew_opts* o) {
    *ptr = nullptr;
    if (o && (o->fault & SKEW_FAULT_NOMEM)) return SKEW_ERR_NOMEM;
    int dev = -1;
    cudaMemPool_t pool = nullptr;
    if (stream_device(st, &dev) == 0 && dev >= 0 && dev < MAX_POOL_DEVICES) pool = lib_pool(dev);
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(ptr, bytes, pool, st) : cudaMallocAsync(ptr, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return SKEW_ERR_NOMEM;
    }
    return 0;
}

}  // namespace

extern "C" {

void skew_release_memory(void) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    for (int d = 0; d < MAX_POOL_DEVICES; d++)
        if (g_pools[d]) cudaMemPoolTrimTo(g_pools[d], 0);
}

void skew_opts_default(skew_opts* opts) {
    if (!opts) return;
    std::memset(opts, 0, sizeof(*opts));
    opts->mode = SKEW_MODE_FP64;
    opts->band = 64;
}

const char* skew_eig_strerror(int code) {
    if (code == 0) return "success";
    if (code < 0 && code > -100) return "invalid argument (-k: argument k)";
    if (code >= SKEW_INFO_INVIT_BASE && code < SKEW_ERR_CUDA) return "inverse iteration did not converge (1000 + j)";
    switch (code) {
    case SKEW_ERR_CUDA: return "CUDA runtime call failed";
    case SKEW_ERR_NOMEM: return "device allocation failed";
    case SKEW_ERR_DEVICE_TIMEOUT: return "device-side wait exceeded its cap";
    case SKEW_ERR_UNSUPPORTED: return "mode or size not supported on this GPU";
    case SKEW_ERR_NONFINITE: return "input holds NaN or Inf";
    case SKEW_ERR_WORKSPACE: return "workspace too small";
    case SKEW_ERR_LAUNCH: return "cooperative launch does not fit on this GPU";
    case SKEW_ERR_NOT_DEFINITE: return "the Bethe-Salpeter matrix is not definite (Cholesky of J H failed)";
    default: return "unknown status code";
    }
}

size_t skew_eig_workspace_size(int n, int nev, const skew_opts* opts) {
    if (n < 0 || nev < 0) return 0;
    return plan_bytes(n, nev, opts, true);
}

size_t skew_eig_workspace_size_ex(int n, int nev, const skew_opts* opts, int vectors) {
    if (n < 0 || nev < 0) return 0;
    return plan_bytes(n, nev, opts, vectors != 0);
}

int skew_eig_ex(int n, const double* A, int lda, int nev, double* lambda, double* Z_re, double* Z_im, int ldz,
                const skew_opts* opts, void* workspace, size_t ws_bytes, int* d_info, void* stream) {
    int rc = check_args(n, A, lda, nev, lambda, Z_re, Z_im);
    if (rc) return rc;
    if (Z_re && ldz < (n > 1 ? n : 1)) return -8;
    if (!workspace && n > 0) return -10;
    if (opts && opts->mode == SKEW_MODE_MIXED_INT8) return SKEW_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0 || nev == 0) {
        if (d_info) {
            zero_int_kernel<<<1, 32, 0, st>>>(d_info);
            count_launch();
            if (cudaGetLastError() != cudaSuccess) return SKEW_ERR_CUDA;
        }
        return 0;
    }
    return run_solve(st, n, A, lda, nev, lambda, Z_re, Z_im, ldz, opts, workspace, ws_bytes, d_info);
}

int skew_eig(int n, const double* A, int lda, int nev, double* lambda, double* Z_re, double* Z_im, void* stream) {
    int rc = check_args(n, A, lda, nev, lambda, Z_re, Z_im);
    if (rc) return rc;
    if (n == 0 || nev == 0) return 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool vectors = Z_re != nullptr;
    size_t bytes = plan_bytes(n, nev, nullptr, vectors);
    void* ws = nullptr;
    if (const int arc = lib_alloc(&ws, bytes, st, nullptr)) return arc;
    // the last 256 bytes of the allocation (slack of plan_bytes) hold d_info
    int* d_info = reinterpret_cast<int*>(static_cast<char*>(ws) + bytes - 256);
    rc = run_solve(st, n, A, lda, nev, lambda, Z_re, Z_im, n, nullptr, ws, bytes - 256, d_info);
    int info = 0;
    if (rc == 0) {
        if (cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = SKEW_ERR_CUDA;
    }
    cudaFreeAsync(ws, st);
    if (const cudaError_t e = cudaStreamSynchronize(st)) return cuda_fail(e);
    return rc ? rc : info;
}

}  // extern "C"

namespace {

// Argument check of a batch: -1 count, then the argument number of the
// first invalid per-matrix entry (2 n, 3 A, 4 lda, 5 nev, 6 lambda, 7 Z).
int batch_check(int count, const int* n, const double* const* A, const int* lda, const int* nev,
                double* const* lambda, double* const* Zre, double* const* Zim, const skew_opts* opts) {
    if (count < 0) return -1;
    if (count == 0) return 0;
    if (!n) return -2;
    if (!A) return -3;
    if (!lda) return -4;
    if (!nev) return -5;
    if (!lambda) return -6;
    if ((Zre == nullptr) != (Zim == nullptr)) return -7;
    for (int b = 0; b < count; b++) {
        const int rc = check_args(n[b], A[b], lda[b], nev[b], lambda[b], Zre ? Zre[b] : nullptr,
                                  Zim ? Zim[b] : nullptr);
        if (rc) return rc - 1;  // -1 .. -6 -> -2 .. -7
    }
    if (opts && opts->mode == SKEW_MODE_MIXED_INT8) return SKEW_ERR_UNSUPPORTED;
    return 0;
}

struct BatchPlan {
    std::vector<BatchProblem> small;
    std::vector<int> large;
    size_t small_bytes, large_bytes;
};

BatchPlan plan_batch(int count, const int* n, const double* const* A, const int* lda, const int* nev,
                     double* const* lambda, double* const* Zre, double* const* Zim, const skew_opts* opts,
                     int* d_info) {
    BatchPlan bp{};
    bp.large_bytes = 0;
    for (int b = 0; b < count; b++) {
        const bool vec = Zre && Zre[b];
        if (n[b] < 2 || nev[b] == 0) continue;
        if (n[b] <= BATCH_MAX) {
            BatchProblem q{};
            q.n = n[b];
            q.nev = nev[b];
            q.lda = lda[b];
            q.A = A ? A[b] : nullptr;
            q.lambda = lambda ? lambda[b] : nullptr;
            q.Zre = vec ? Zre[b] : nullptr;
            q.Zim = vec ? Zim[b] : nullptr;
            q.info = d_info ? d_info + b : nullptr;
            bp.small.push_back(q);
        } else {
            bp.large.push_back(b);
            const size_t by = plan_bytes(n[b], nev[b], opts, vec);
            bp.large_bytes = by > bp.large_bytes ? by : bp.large_bytes;
        }
    }
    bp.small_bytes = bp.small.empty() ? 0 : batched_small_ws((int)bp.small.size(), bp.small.data());
    return bp;
}

}  // namespace

extern "C" {

size_t skew_eig_batched_workspace_size(int count, const int* n, const int* nev, const skew_opts* opts) {
    if (count <= 0 || !n || !nev) return 256;
    // sizes only: pointers are not looked at; every matrix is taken with vectors
    std::vector<double*> fake((size_t)count, reinterpret_cast<double*>(16));
    std::vector<int> lda((size_t)count);
    for (int b = 0; b < count; b++) lda[(size_t)b] = n[b] > 1 ? n[b] : 1;
    BatchPlan bp = plan_batch(count, n, fake.data(), lda.data(), nev, fake.data(), fake.data(), fake.data(), opts,
                              nullptr);
    return align_up(bp.small_bytes) + align_up(bp.large_bytes) + 256;
}

int skew_eig_batched_ex(int count, const int* n, const double* const* A, const int* lda, const int* nev,
                        double* const* lambda, double* const* Z_re, double* const* Z_im, const skew_opts* opts,
                        void* workspace, size_t ws_bytes, int* d_info, void* stream) {
    int rc = batch_check(count, n, A, lda, nev, lambda, Z_re, Z_im, opts);
    if (rc) return rc;
    if (count == 0) return 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (d_info) {
        if (const cudaError_t e = cudaMemsetAsync(d_info, 0, sizeof(int) * (size_t)count, st)) return cuda_fail(e);
    }
    BatchPlan bp = plan_batch(count, n, A, lda, nev, lambda, Z_re, Z_im, opts, d_info);
    const size_t need = align_up(bp.small_bytes) + align_up(bp.large_bytes);
    if ((bp.small_bytes || bp.large_bytes) && (!workspace || ws_bytes < need)) return SKEW_ERR_WORKSPACE;
    char* base = static_cast<char*>(workspace);
    if (!bp.small.empty()) {
        rc = batched_small(st, (int)bp.small.size(), bp.small.data(), base, bp.small_bytes, 5);
        if (rc) return rc;
    }
    char* lws = base + align_up(bp.small_bytes);
    for (int b : bp.large) {
        const bool vec = Z_re && Z_re[b];
        rc = run_solve(st, n[b], A[b], lda[b], nev[b], lambda[b], vec ? Z_re[b] : nullptr, vec ? Z_im[b] : nullptr,
                       n[b], opts, lws, bp.large_bytes, d_info ? d_info + b : nullptr);
        if (rc) return rc;
    }
    return cuda_ok(cudaGetLastError());
}

}  // extern "C"

struct skew_batched_plan {
    BatchPlanDev d;
    BatchLaunch launch;
    skew_batched_config cfg;
    int count;
    int* d_info;
};

extern "C" {

int skew_batched_set_config(const skew_batched_config* cfg) {
    if (!cfg) return -1;
    if (batched_config_check(*cfg)) return -1;
    batched_default_config() = *cfg;
    return 0;
}

void skew_batched_get_config(skew_batched_config* cfg) {
    if (cfg) *cfg = batched_default_config();
}

int skew_batched_plan_create(int count, const int* n, const double* const* A, const int* lda, const int* nev,
                             double* const* lambda, double* const* Z_re, double* const* Z_im,
                             const skew_batched_config* cfg, void* workspace, size_t ws_bytes, int* d_info,
                             void* stream, skew_batched_plan** plan) {
    if (!plan) return -14;
    *plan = nullptr;
    int rc = batch_check(count, n, A, lda, nev, lambda, Z_re, Z_im, nullptr);
    if (rc) return rc;
    const skew_batched_config c = cfg ? *cfg : batched_default_config();
    if (batched_config_check(c)) return -9;
    for (int b = 0; b < count; b++)
        if (n[b] > BATCH_MAX) return SKEW_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BatchPlan bp = plan_batch(count, n, A, lda, nev, lambda, Z_re, Z_im, nullptr, d_info);
    if (bp.small_bytes && (!workspace || ws_bytes < bp.small_bytes)) return SKEW_ERR_WORKSPACE;
    skew_batched_plan* p = new skew_batched_plan{};
    p->count = count;
    p->d_info = d_info;
    p->cfg = c;
    if (!bp.small.empty()) {
        rc = batched_upload(st, (int)bp.small.size(), bp.small.data(), workspace, ws_bytes, &p->d);
        if (!rc) rc = batched_prepare(p->d, c, &p->launch);
    }
    if (!rc) {
        if (const cudaError_t e = cudaStreamSynchronize(st)) rc = cuda_fail(e);
    }
    if (rc) {
        delete p;
        return rc;
    }
    *plan = p;
    return 0;
}

int skew_batched_plan_exec(skew_batched_plan* p, void* stream) {
    if (!p) return -1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p->d_info && p->count > 0) {
        if (const cudaError_t e = cudaMemsetAsync(p->d_info, 0, sizeof(int) * (size_t)p->count, st))
            return cuda_fail(e);
    }
    return batched_exec(st, p->d, p->launch, 5);
}

void skew_batched_plan_get_config(const skew_batched_plan* p, skew_batched_config* cfg) {
    if (p && cfg) *cfg = p->cfg;
}

void skew_batched_plan_destroy(skew_batched_plan* p) { delete p; }

int skew_batched_plan_tune(skew_batched_plan* p, skew_batched_config* best, int* cand_ctas, int* cand_smem,
                           float* cand_ms, int cap, void* stream) {
    if (!p) return -1;
    if (cap < 0) return -6;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p->d.count <= 0) {
        if (best) *best = p->cfg;
        return 0;
    }
    static const int kSmem[] = {0, 48, 64, 80, 96, 112, 128, 160};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SKEW_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SKEW_ERR_CUDA;
    }
    int ncand = 0, rc = 0;
    float best_ms = 0.f;
    skew_batched_config best_cfg = p->cfg;
    BatchLaunch best_launch = p->launch;
    int last_smem = -1, last_ctas = -1;
    for (int ctas = 1; ctas <= 4 && !rc; ctas++) {
        for (int si = 0; si < (int)(sizeof(kSmem) / sizeof(kSmem[0])) && !rc; si++) {
            const skew_batched_config c{ctas, kSmem[si], {0, 0}};
            BatchLaunch L{};
            if (batched_prepare(p->d, c, &L)) continue;
            // thresholds the shared-memory budget caps to the same value time the same launch
            if (L.ctas == last_ctas && L.smem_n == last_smem) continue;
            last_ctas = L.ctas;
            last_smem = L.smem_n;
            float ms = 1e30f;
            for (int rep = 0; rep < 3 && !rc; rep++) {
                if (cudaEventRecord(e0, st) != cudaSuccess) rc = SKEW_ERR_CUDA;
                if (!rc) rc = batched_exec(st, p->d, L, 5);
                if (!rc && cudaEventRecord(e1, st) != cudaSuccess) rc = SKEW_ERR_CUDA;
                if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = SKEW_ERR_CUDA;
                float t = 0.f;
                if (!rc && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = SKEW_ERR_CUDA;
                if (!rc && rep > 0 && t < ms) ms = t;  // the first run warms up
            }
            if (rc) break;
            if (ncand < cap) {
                if (cand_ctas) cand_ctas[ncand] = ctas;
                if (cand_smem) cand_smem[ncand] = L.smem_n;
                if (cand_ms) cand_ms[ncand] = ms;
            }
            if (ncand == 0 || ms < best_ms) {
                best_ms = ms;
                best_cfg = skew_batched_config{ctas, L.smem_n, {0, 0}};
                best_launch = L;
            }
            ncand++;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    // keep the fastest (its kernel attribute is set again for the launch)
    if (batched_prepare(p->d, best_cfg, &best_launch)) return SKEW_ERR_LAUNCH;
    p->cfg = best_cfg;
    p->launch = best_launch;
    if (best) *best = best_cfg;
    return ncand;
}

int skew_eig_batched(int count, const int* n, const double* const* A, const int* lda, const int* nev,
                     double* const* lambda, double* const* Z_re, double* const* Z_im, const skew_opts* opts,
                     void* stream) {
    int rc = batch_check(count, n, A, lda, nev, lambda, Z_re, Z_im, opts);
    if (rc) return rc;
    if (count == 0) return 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BatchPlan bp = plan_batch(count, n, A, lda, nev, lambda, Z_re, Z_im, opts, nullptr);
    const size_t need = align_up(bp.small_bytes) + align_up(bp.large_bytes);
    if (need == 0) return 0;
    void* ws = nullptr;
    if (const int arc = lib_alloc(&ws, need, st, opts)) return arc;
    rc = skew_eig_batched_ex(count, n, A, lda, nev, lambda, Z_re, Z_im, opts, ws, need, nullptr, stream);
    cudaFreeAsync(ws, st);
    return rc;
}

int skew_eig_host(int n, const double* A, int lda, int nev, double* lambda, double* Z_re, double* Z_im,
                  const skew_opts* opts, void* stream) {
    int rc = check_args(n, A, lda, nev, lambda, Z_re, Z_im);
    if (rc) return rc;
    if (n == 0 || nev == 0) return 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool vectors = Z_re != nullptr;
    const size_t nn = (size_t)n;
    if (opts && opts->mode == SKEW_MODE_MIXED_INT8) return SKEW_ERR_UNSUPPORTED;
    size_t bytes = plan_bytes(n, nev, opts, vectors);
    size_t io = align_up(sizeof(double) * nn * n) + align_up(sizeof(double) * nev) +
                (vectors ? 2 * align_up(sizeof(double) * nn * nev) : 0) + 256;
    char* base = nullptr;
    if (const int arc = lib_alloc((void**)&base, bytes + io, st, opts)) return arc;
    double* dA = reinterpret_cast<double*>(base + bytes);
    double* dl = reinterpret_cast<double*>(base + bytes + align_up(sizeof(double) * nn * n));
    double* dzr = vectors ? reinterpret_cast<double*>(reinterpret_cast<char*>(dl) + align_up(sizeof(double) * nev)) : nullptr;
    double* dzi = vectors ? reinterpret_cast<double*>(reinterpret_cast<char*>(dzr) + align_up(sizeof(double) * nn * nev)) : nullptr;
    int* d_info = reinterpret_cast<int*>(base + bytes - 256);
    int info = 0;
    rc = 0;
    // one linear copy when the columns are contiguous, a pitched one otherwise
    const cudaError_t ce =
        (lda == n) ? cudaMemcpyAsync(dA, A, sizeof(double) * nn * nn, cudaMemcpyHostToDevice, st)
                   : cudaMemcpy2DAsync(dA, sizeof(double) * nn, A, sizeof(double) * (size_t)lda, sizeof(double) * nn,
                                       nn, cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) rc = SKEW_ERR_CUDA;
    if (!rc) rc = run_solve(st, n, dA, n, nev, dl, dzr, dzi, n, opts, base, bytes - 256, d_info);
    if (!rc) {
        if (cudaMemcpyAsync(lambda, dl, sizeof(double) * nev, cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = SKEW_ERR_CUDA;
        if (vectors) {
            if (cudaMemcpyAsync(Z_re, dzr, sizeof(double) * nn * nev, cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = SKEW_ERR_CUDA;
            if (cudaMemcpyAsync(Z_im, dzi, sizeof(double) * nn * nev, cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = SKEW_ERR_CUDA;
        }
        if (cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = SKEW_ERR_CUDA;
    }
    cudaFreeAsync(base, st);
    if (const cudaError_t e = cudaStreamSynchronize(st)) return cuda_fail(e);
    return rc ? rc : info;
}

int skew_eig_profile(int n, const double* A, int lda, int nev, double* lambda, double* Z_re, double* Z_im, int ldz,
                     const skew_opts* opts, void* workspace, size_t ws_bytes, float* stage_ms, void* stream) {
    int rc = check_args(n, A, lda, nev, lambda, Z_re, Z_im);
    if (rc) return rc;
    if (Z_re && ldz < (n > 1 ? n : 1)) return -8;
    if (!workspace && n > 0) return -10;
    if (!stage_ms) return -12;
    if (opts && opts->mode == SKEW_MODE_MIXED_INT8) return SKEW_ERR_UNSUPPORTED;
    for (int i = 0; i < SKEW_NSTAGES; i++) stage_ms[i] = 0.0f;
    if (n == 0 || nev == 0) return 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    StageEvents ev;
    for (int i = 0; i <= SKEW_NSTAGES; i++)
        if (cudaEventCreate(&ev.ev[i]) != cudaSuccess) return SKEW_ERR_CUDA;
    int* d_info = nullptr;
    // status word: the caller workspace's carve starts with it (see carve_plan)
    rc = run_solve(st, n, A, lda, nev, lambda, Z_re, Z_im, ldz, opts, workspace, ws_bytes, nullptr, &ev);
    int info = 0;
    if (rc == 0) {
        d_info = static_cast<int*>(workspace);
        if (cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = SKEW_ERR_CUDA;
    }
    if (const cudaError_t e = cudaStreamSynchronize(st)) rc = cuda_fail(e);
    if (rc == 0)
        for (int i = 0; i < SKEW_NSTAGES; i++) cudaEventElapsedTime(&stage_ms[i], ev.ev[i], ev.ev[i + 1]);
    for (int i = 0; i <= SKEW_NSTAGES; i++) cudaEventDestroy(ev.ev[i]);
    // kernel timing: the solve is complete, so its records can be folded into
    // the per-kind totals (the pool then never fills across repeated solves)
    if (rc == 0 && ktimer().on && kt_fold() != 0) rc = SKEW_ERR_CUDA;
    return rc ? rc : info;
}

namespace {
struct BseWs {
    double *M, *JL, *K, *NP;
    int* status;
    void* solve;
    size_t solve_bytes;
};
bool carve_bse(Carve& cv, int h, int nev, const skew_opts* o, BseWs* w) {
    const size_t N = 2 * (size_t)h;
    w->status = cv.take<int>(16);
    w->M = cv.take<double>(N * N);
    w->JL = cv.take<double>(N * N);  // J L, later the eigenvectors z of K (N x 2 nev)
    w->K = cv.take<double>(N * N);
    w->NP = cv.take<double>(N * 64);
    w->solve_bytes = plan_bytes((int)N, nev, o, true);
    w->solve = cv.take<char>(w->solve_bytes);
    return cv.ok;
}
}  // namespace

size_t skew_bse_workspace_size(int h, int nev, const skew_opts* opts) {
    if (h < 1 || nev < 1) return 0;
    Carve cv(nullptr, ~size_t(0));
    BseWs w{};
    carve_bse(cv, h, nev, opts, &w);
    return cv.off + 256;
}

int skew_bse_solve(int h, const double* A_re, const double* A_im, int lda, const double* B_re, const double* B_im,
                   int ldb, int nev, double* lambda, double* psi_re, double* psi_im, int ldpsi, const skew_opts* opts,
                   void* workspace, size_t ws_bytes, int* d_info, void* stream) {
    if (h < 1) return -1;
    if (!A_re || !A_im) return -2;
    if (lda < h) return -4;
    if (!B_re || !B_im) return -5;
    if (ldb < h) return -7;
    if (nev < 1 || nev > h) return -8;
    if (!lambda) return -9;
    if (!psi_re || !psi_im) return -10;
    if (ldpsi < 2 * h) return -12;
    if (!workspace) return -14;
    if (!d_info) return -16;
    if (opts && opts->mode == SKEW_MODE_MIXED_INT8) return SKEW_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Carve cv(workspace, ws_bytes);
    BseWs w{};
    if (!carve_bse(cv, h, nev, opts, &w)) return SKEW_ERR_WORKSPACE;
    const int N = 2 * h;
    zero_int_kernel<<<1, 32, 0, st>>>(w.status);
    count_launch();
    // 1. M = J H; 2. M = L L^T
    if (const cudaError_t e = bse_build_m(st, h, A_re, A_im, lda, B_re, B_im, ldb, w.M, N)) return cuda_fail(e);
    if (const cudaError_t e = cholesky_lower(st, N, w.M, N, w.NP, w.status)) return cuda_fail(e);
    // 3. K = L^T (J L), then the skew solve (its lower triangle is read)
    if (const cudaError_t e = bse_jl(st, h, w.M, N, w.JL, N)) return cuda_fail(e);
    if (const cudaError_t e = gemm(st, true, false, N, N, N, 1.0, w.M, N, w.JL, N, 0.0, w.K, N))
        return cuda_fail(e);
    double* Zr = w.JL;
    double* Zi = w.JL + (size_t)N * nev;
    int rc = run_solve(st, N, w.K, N, nev, lambda, Zr, Zi, N, opts, w.solve, w.solve_bytes, w.status + 1);
    if (rc) return rc;
    // 4. x = L^-T z (real and imaginary parts), psi = Q x sqrt(lambda)
    if (const cudaError_t e = trsm_lower_t(st, N, w.M, N, Zr, N, 2 * nev)) return cuda_fail(e);
    if (const cudaError_t e = bse_psi(st, h, nev, Zr, Zi, N, lambda, psi_re, psi_im, ldpsi)) return cuda_fail(e);
    // status: the Cholesky's, else the skew solve's
    bse_status_kernel<<<1, 32, 0, st>>>(w.status, d_info);
    count_launch();
    return cuda_ok(cudaGetLastError());
}

size_t skew_refine_ws(int n) { return refine_ws(n) + align_up(sizeof(double) * (size_t)n * n) + 256; }

int skew_refine(int n, const double* A, int lda, double* lambda, double* Z_re, double* Z_im, int ldz, int iters,
                void* ws, size_t ws_bytes, int* d_status, void* stream) {
    if (n < 2 || n % 2) return -1;
    if (!A) return -2;
    if (lda < n) return -3;
    if (!lambda) return -4;
    if (!Z_re || !Z_im) return -5;
    if (ldz < n) return -7;
    if (iters < 1) return -8;
    const int m = n / 2;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Carve cv(ws, ws_bytes);
    double* M = cv.take<double>((size_t)n * n);
    size_t rb = refine_ws(n);
    void* rws = cv.take<char>(rb);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    if (cudaMemcpy2DAsync(M, sizeof(double) * n, Z_re, sizeof(double) * ldz, sizeof(double) * n, m,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpy2DAsync(M + (size_t)n * m, sizeof(double) * n, Z_im, sizeof(double) * ldz, sizeof(double) * n, m,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SKEW_ERR_CUDA;
    int rc = refine(st, n, A, lda, lambda, M, iters, rws, rb, d_status, &last_refine_info());
    if (rc) return rc;
    if (cudaMemcpy2DAsync(Z_re, sizeof(double) * ldz, M, sizeof(double) * n, sizeof(double) * n, m,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpy2DAsync(Z_im, sizeof(double) * ldz, M + (size_t)n * m, sizeof(double) * n, sizeof(double) * n, m,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SKEW_ERR_CUDA;
    return 0;
}

size_t skew_metrics_ws(int n, int nev, int ncols) { return metrics_ws(n, nev, ncols > 0 ? ncols : 1); }

int skew_eig_metrics(int n, const double* A, int lda, int nev, const double* lambda, const double* Z_re,
                     const double* Z_im, int ldz, const int* cols, int ncols, double* out3, void* ws, size_t ws_bytes,
                     void* stream) {
    if (n < 1) return -1;
    if (!A) return -2;
    if (lda < n) return -3;
    if (nev < 1 || nev > n) return -4;
    if (!lambda || !Z_re || !Z_im) return -5;
    if (ldz < n) return -8;
    if (ncols < 1 || (!cols && ncols != nev) || ncols > nev) return -10;
    if (!out3) return -11;
    return metrics(static_cast<cudaStream_t>(stream), n, A, lda, nev, lambda, Z_re, Z_im, ldz, cols, ncols, out3, ws,
                   ws_bytes);
}

long long skew_launch_count(void) { return launch_count(); }

const char* skew_last_cuda_error(void) { return g_last_cuda_error.load(std::memory_order_relaxed); }

int skew_kernel_timing(int enable) {
    KTimer& t = ktimer();
    t.on = enable != 0;
    t.clear();
    return 0;
}

int skew_kernel_timing_read(int kind, double* ms, double* flops, long long* launches) {
    if (kind < 0 || kind >= KT_KINDS) return -1;
    KTimer& t = ktimer();
    if (kt_fold() != 0) return SKEW_ERR_CUDA;
    if (ms) *ms = t.ms[kind];
    if (flops) *flops = t.fl[kind];
    if (launches) *launches = t.cnt[kind];
    return t.dropped ? -2 : 0;
}

long long skew_kernel_timing_dropped(void) { return ktimer().dropped; }

int skew_kernel_timeline(int cap, int* kinds, double* start_ms, double* end_ms) {
    if (cap < 0) return -1;
    KTimer& t = ktimer();
    if (kt_fold() != 0) return SKEW_ERR_CUDA;
    const size_t have = t.tl_kind.size();
    const int cnt = (int)(have < (size_t)cap ? have : (size_t)cap);
    for (int i = 0; i < cnt; i++) {
        if (kinds) kinds[i] = t.tl_kind[i];
        if (start_ms) start_ms[i] = t.tl_a[i];
        if (end_ms) end_ms[i] = t.tl_b[i];
    }
    return cnt;
}

int skew_refine_stats(double* emax, int* nclose, int cap) {
    refine_stats_flush();
    const RefineInfo& r = last_refine_info();
    for (int i = 0; i < cap && i < 8; i++) {
        if (emax) emax[i] = r.emax[i];
        if (nclose) nclose[i] = r.nclose[i];
    }
    return r.iterations;
}

int skew_refine_trace(double* rnorm, long long* where, int cap) {
    refine_stats_flush();
    const RefineInfo& r = last_refine_info();
    for (int i = 0; i < cap && i < 8; i++) {
        if (rnorm) rnorm[i] = r.rnorm[i];
        if (where) where[i] = r.where[i];
    }
    return r.iterations;
}

int skew_refine_slices(int* slices, int* uslices, int cap) {
    refine_stats_flush();
    const RefineInfo& r = last_refine_info();
    for (int i = 0; i < cap && i < 8; i++) {
        if (slices) slices[i] = r.slices[i];
        if (uslices) uslices[i] = r.uslices[i];
    }
    return r.iterations;
}

// ---------------------------------------------------------------- stages
size_t skew_band_reduce_ws(int n, int b) { return band_reduce_ws(n, b); }

int skew_band_reduce(int n, double* W, int ldw, int b, double* Tfac, void* ws, size_t ws_bytes, int* d_status,
                     void* stream) {
    if (n < 0) return -1;
    if (ldw < (n > 1 ? n : 1)) return -3;
    if (b <= 0 || b % 64) return -4;
    return band_reduce(static_cast<cudaStream_t>(stream), n, W, ldw, b, Tfac, ws, ws_bytes, d_status);
}

int skew_band_pack(int n, int b, const double* W, int ldw, double* AB, int ldab, void* stream) {
    if (n < 0) return -1;
    if (b <= 0) return -2;
    if (ldab < 2 * b + 1) return -6;
    return band_pack(static_cast<cudaStream_t>(stream), n, b, W, ldw, AB, ldab) == cudaSuccess ? 0 : SKEW_ERR_CUDA;
}

int skew_chase_steps(int n, int b) { return chase_steps(n, b); }
size_t skew_chase_ws(int n, int b) { return chase_ws(n, b); }

int skew_band_to_tridiag(int n, int b, double* AB, int ldab, double* alpha, double* Vtrd, double* tautrd, void* ws,
                         size_t ws_bytes, int* d_status, void* stream) {
    if (n < 0) return -1;
    if (b != 64) return -2;
    if (ldab < 2 * b + 1) return -4;
    return chase(static_cast<cudaStream_t>(stream), n, b, AB, ldab, alpha, Vtrd, tautrd, ws, ws_bytes, d_status, 0);
}

size_t skew_tridiag_ws(int n, int nev) {
    return tridiag_ws(n, nev) + align_up(sizeof(double) * (size_t)(n > 0 ? n : 1) * (nev > 0 ? nev : 1)) + 256;
}

int skew_tridiag_eig(int n, const double* alpha, int nev, double* lambda, double* Q, int ldq, void* ws,
                     size_t ws_bytes, int* d_status, void* stream) {
    if (n < 1) return -1;
    if (nev < 1 || nev > n) return -3;
    if (Q && ldq < n) return -6;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Carve cv(ws, ws_bytes);
    double* Qi = Q ? cv.take<double>((size_t)n * nev) : nullptr;
    size_t rest = tridiag_ws(n, nev);
    void* tws = cv.take<char>(rest);
    if (!cv.ok) return SKEW_ERR_WORKSPACE;
    int rc = tridiag_eig(st, n, alpha, nev, lambda, Qi, tws, rest, d_status, 5);
    if (rc) return rc;
    if (Q && interleaved_to_colmajor(st, n, nev, Qi, Q, nullptr, ldq, false) != cudaSuccess) return SKEW_ERR_CUDA;
    return 0;
}

int skew_dmap(int n, int k, const double* Q, int ldq, double* X, double* Y, int ldz, void* stream) {
    if (n < 0) return -1;
    if (k < 0) return -2;
    return dmap_colmajor(static_cast<cudaStream_t>(stream), n, k, Q, ldq, X, Y, ldz) == cudaSuccess ? 0 : SKEW_ERR_CUDA;
}

int skew_apply_qtrd(int n, int b, const double* Vtrd, const double* tautrd, double* Z, int ldz, int k, void* stream) {
    if (n < 0) return -1;
    if (b != 64) return -2;
    return apply_qtrd(static_cast<cudaStream_t>(stream), n, b, Vtrd, tautrd, Z, ldz, k) == cudaSuccess ? 0
                                                                                                      : SKEW_ERR_CUDA;
}

size_t skew_apply_qtrd_f32_ws(int n, int tensor) { return tensor ? qtrd_tc_ws(n) : 256; }

int skew_apply_qtrd_f32(int n, int b, const float* V32, const float* tau32, float* Z, int ldz, int k, int tensor,
                        void* ws, size_t ws_bytes, int* d_status, void* stream) {
    if (n < 0) return -1;
    if (b != 64) return -2;
    if (n >= 3 && k > 0 && (!V32 || !tau32)) return -3;
    if (ldz < (n > 1 ? n : 1)) return -6;
    if (k < 0) return -7;
    if (tensor != 0 && tensor != 1) return -8;
    if (!d_status) return -11;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (tensor) return apply_qtrd_tc(st, n, V32, tau32, Z, ldz, k, ws, ws_bytes, d_status);
    return apply_qtrd_f32(st, n, b, V32, tau32, Z, ldz, k, d_status) == cudaSuccess ? 0 : SKEW_ERR_CUDA;
}

int skew_apply_qtrd_df(int n, int b, const double* Vtrd, const double* tautrd, double* Z, int ldz, int k,
                       int* d_status, void* stream) {
    if (n < 0) return -1;
    if (b != 64) return -2;
    if (n >= 3 && k > 0 && (!Vtrd || !tautrd)) return -3;
    if (ldz < (n > 1 ? n : 1)) return -6;
    if (k < 0) return -7;
    if (!d_status) return -8;
    return apply_qtrd_df(static_cast<cudaStream_t>(stream), n, b, Vtrd, tautrd, Z, ldz, k, d_status) == cudaSuccess
               ? 0
               : SKEW_ERR_CUDA;
}

size_t skew_qband_ws(int n, int b, int k) { return qband_ws(n, b, k); }

int skew_apply_qband(int n, int b, const double* W, int ldw, const double* Tfac, double* Z, int ldz, int k, void* ws,
                     size_t ws_bytes, void* stream) {
    if (n < 0) return -1;
    if (b <= 0 || b % 64) return -2;
    return apply_qband(static_cast<cudaStream_t>(stream), n, b, W, ldw, Tfac, Z, ldz, k, ws, ws_bytes);
}

}  // extern "C"
