// internal.h -- host-side launchers shared between the translation units of
// the skew-symmetric eigensolver library.  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/skeweig.h"

namespace sk {

// ---- gemm_f64.cu -----------------------------------------------------------
// C[M x N] = alpha * op(A) op(B) + beta * C, column-major FP64.
// op(A) = A (ta = false) or A^T (ta = true); likewise op(B).
// splitk > 1 (or 0: chosen from the tile count) splits the K range over
// CTAs.  With part (part_elems doubles, at least M N for a split to happen)
// each range writes its partial product there and a second launch adds them
// in range order, so the result is the same on every run; the split count is
// limited to part_elems / (M N).  Without part the ranges accumulate into C
// with FP64 atomics (beta applied first), whose order varies.
cudaError_t gemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, double alpha,
                 const double* A, int lda, const double* B, int ldb, double beta,
                 double* C, int ldc, int splitk = 0, double* part = nullptr, size_t part_elems = 0);

// P[m x nb] = S V where S = L - L^T is the skew matrix whose strict lower
// triangle is stored in W (ld ldw); V is m x nb (ld ldv).  Split K as for
// gemm (ordered with part, atomics without); P is overwritten.
cudaError_t skew_symm(cudaStream_t st, int m, int nb, const double* W, int ldw,
                      const double* V, int ldv, double* P, int ldp, int splitk = 0,
                      double* part = nullptr, size_t part_elems = 0);

// Lower 64 x 64 tiles (diagonal tiles complete) of C[m x m] +=
// X[m x k] Y[m x k]^T.  Used for the skew rank-2k update with
// X = [V W], Y = [W -V] (zero_diag: the diagonal set to 0, exact for a skew
// result) and for the Cholesky's symmetric trailing update (zero_diag false).
cudaError_t gemm_lower_tiles(cudaStream_t st, int m, int k, const double* X, int ldx,
                             const double* Y, int ldy, double* C, int ldc, bool zero_diag = true);

// ---- band_reduce.cu --------------------------------------------------------
// planes > 0: the skew SYMM and the rank-2k update run as split-BF16 tensor-core
// GEMMs with that many planes per operand (2: BF16x3, 3: BF16x6); planes ==
// REDUCE_F64ACC: as FP64-accurate digit-slice tensor-core products.
constexpr int REDUCE_F64ACC = 8;
size_t band_reduce_ws(int n, int b, int planes = 0);
// slices: digit slices of the REDUCE_F64ACC products (8: FP64-accurate);
// spin_cap: polls of the panel QR's grid barrier before it gives up with
// SKEW_ERR_DEVICE_TIMEOUT (0: the default cap)
int band_reduce(cudaStream_t st, int n, double* W, int ldw, int b, double* Tfac,
                void* ws, size_t ws_bytes, int* d_status, int planes = 0, int slices = 8,
                unsigned spin_cap = 0);
cudaError_t band_pack(cudaStream_t st, int n, int b, const double* W, int ldw,
                      double* AB, int ldab);
// Explicit V (m x b, ld ldv) of panel p from the reduced W.
cudaError_t panel_v(cudaStream_t st, int n, int b, int p, const double* W, int ldw,
                    double* V, int ldv);
int num_panels(int n, int b);

// ---- chase.cu ---------------------------------------------------------------
int chase_steps(int n, int b);
size_t chase_ws(int n, int b);
// Vtrd / tautrd (may be null): the reflectors in FP64, slot k nsw + s.  V32 /
// tau32 (may be null): FP32 copies with the sweep stride padded to a multiple
// of 64 (slot k nsw64 + s); slots of steps a sweep does not have are not
// written.  spin_cap: polls of a wait on the previous sweep's progress before
// it gives up with SKEW_ERR_DEVICE_TIMEOUT (0: the default cap).
int chase(cudaStream_t st, int n, int b, double* AB, int ldab, double* alpha,
          double* Vtrd, double* tautrd, void* ws, size_t ws_bytes, int* d_status,
          unsigned spin_cap, float* V32 = nullptr, float* tau32 = nullptr);

// ---- tridiag.cu -------------------------------------------------------------
size_t tridiag_ws(int n, int nev);
// Eigenvalues (descending) and eigenvectors of tridiag(alpha, 0, alpha).
// Vectors go to Qi in interleaved layout Qi[i * nev + k].
// fp64 = false: eigenvalues to about 2^-42 ||S|| from double-float counts
// only (a caller that refines them afterwards); otherwise finished in FP64.
// bidiag: the FP64 bisection finish counts on the zero-diagonal form (B B^T
// of the perfect-shuffled bidiagonal, half-length recurrences; nev <= n/2).
int tridiag_eig(cudaStream_t st, int n, const double* alpha, int nev, double* lambda,
                double* Qi, void* ws, size_t ws_bytes, int* d_status, int maxit, bool fp64 = true,
                bool bidiag = true);
// Interleaved Qi -> column-major X (and Y) with optional D map.
cudaError_t interleaved_to_colmajor(cudaStream_t st, int n, int nev, const double* Qi,
                                    double* X, double* Y, int ldz, bool dmap);
cudaError_t dmap_colmajor(cudaStream_t st, int n, int k, const double* Q, int ldq,
                          double* X, double* Y, int ldz);

// ---- backtransform.cu -------------------------------------------------------
cudaError_t apply_qtrd(cudaStream_t st, int n, int b, const double* Vtrd,
                       const double* tautrd, double* Z, int ldz, int k);
// FP32 Q_trd from the chase's FP32 reflectors (stride nsw64, taus of absent
// steps zero).
cudaError_t apply_qtrd_f32(cudaStream_t st, int n, int b, const float* V32, const float* tau32, float* Z, int ldz,
                           int k, int* status);
// ---- qtrd_df.cu (Q_trd in double-float on the FP32 pipe) -----------------
// Z (FP64, n x k, ld ldz) <- Q_trd Z from the chase's FP64 reflectors (layout
// of apply_qtrd), about 2^-46 accurate per operation; status receives
// SKEW_ERR_DEVICE_TIMEOUT if a copy never lands.
cudaError_t apply_qtrd_df(cudaStream_t st, int n, int b, const double* Vtrd, const double* tautrd, double* Z,
                          int ldz, int k, int* status);
// ---- qtrd_tc.cu (Q_trd on the tensor cores) ------------------------------
// Z (FP32, n x k, ld ldz) <- Q_trd Z from the chase's FP32 reflectors (slot
// k nsw64 + s): each 64-sweep block in compact WY form, applied by tcgen05
// BF16x6 products with the window in TMEM.  Workspace: the blocks' operand
// images, qtrd_tc_ws(n) bytes.
size_t qtrd_tc_ws(int n);
int apply_qtrd_tc(cudaStream_t st, int n, const float* V32, const float* tau32, float* Z, int ldz, int k,
                  void* ws, size_t ws_bytes, int* status);
size_t qband_ws(int n, int b, int k);
size_t qband_mixed_ws(int n, int b, int k, int planes);
int apply_qband_mixed(cudaStream_t st, int n, int b, const double* W, int ldw, const double* Tfac, double* Z, int ldz,
                      int k, void* ws, size_t ws_bytes, int* status, int planes, int slices = 8);
int apply_qband(cudaStream_t st, int n, int b, const double* W, int ldw,
                const double* Tfac, double* Z, int ldz, int k, void* ws, size_t ws_bytes);

// ---- umma_gemm.cu (tcgen05 BF16x3) ------------------------------------------
// C = alpha * split3(A) split3(B)^T + beta * C (FP64 C, column-major, ldc) with
// A[i,k] = A[i*a_rs + k*a_ks] (or the skew matrix of a lower triangle stored
// column-major with ld a_ks when a_skew), B[j,k] = B[j*b_rs + k*b_ks];
// lower: only the lower 128-tiles of C (M == N), C += alpha D, zero diagonal.
// nplanes = 2: BF16x3 (hi*hi + lo*hi + hi*lo); nplanes = 3: BF16x6 (the six
// products of order <= 2 of hi, mid, lo).
size_t split_gemm_ws(int M, int N, int K, int nplanes = 3);
int split_gemm(cudaStream_t st, int M, int N, int K, double alpha, const double* A, long long a_rs, long long a_ks,
               int a_skew, const double* B, long long b_rs, long long b_ks, double beta, double* C, long long ldc,
               int lower, void* ws, size_t ws_bytes, int* status, int nplanes = 3);

// ---- ozaki_gemm.cu (FP64-accurate product from exact BF16 digit slices) -------
// C = alpha * (sa A)(sb B)^T + beta * C, A[i,k] = A[i*a_rs + k*a_ks],
// B[j,k] = B[j*b_rs + k*b_ks], C column-major.
size_t ozaki_gemm_ws(int M, int N, int K);
// An operand cut into its 8 digit slices (planes of Rp x Kp BF16, row-major)
// with per-row exponents; reusable across products.
struct OzOperand {
    __nv_bfloat16* d;
    int* e;
    int rows, K;
    long long Rp, Kp;
    // a view into a larger split (oz_view): row r of the view is row roff + r
    // of the split (d and e already advanced by roff), element k of a row is
    // element koff + k (koff a multiple of 64)
    int roff, koff;
};
// Rows r0 .. r0+rows-1 and elements k0 .. k0+K-1 of a split operand, without
// copying (k0 a multiple of 64; rows and K within the operand).
OzOperand oz_view(const OzOperand& o, int r0, int k0, int rows, int K);
size_t ozaki_operand_ws(int rows, int K);
// skip (device flag, may be null): nonzero at run time -> the launches do nothing.
int ozaki_split(cudaStream_t st, int rows, int K, const double* src, long long rs, long long ks, double sgn, int skew,
                void* ws, size_t ws_bytes, OzOperand* op, const int* skip = nullptr);
// ksplit > 1: K is cut into up to that many ranges (one CTA per tile and
// range) and the partial tiles, ranges x N x M doubles in part (capacity
// part_elems doubles: fewer ranges are taken when they would not fit), are
// summed in order.
int ozaki_gemm_pre(cudaStream_t st, const OzOperand& A, const OzOperand& B, double alpha, double beta, double* C,
                   long long ldc, int* status, int slices = 8, int lower = 0, int ksplit = 1,
                   double* part = nullptr, size_t part_elems = 0, const int* skip = nullptr,
                   const int* s_dyn = nullptr);
// skip: device flag, nonzero at run time -> the launch does nothing; s_dyn:
// device slice count (1 .. slices) read by the kernel in place of slices
// (the launch shape and the work recorded for kernel timing use slices).
// a_skew: A is the skew matrix of the strict lower triangle stored column-major
// with leading dimension a_ks (a_rs unused).  slices (1..8): digit slices kept,
// accuracy about 2^-7 slices relative to |a_r|max |b_c|max per term.  lower:
// only 128 x 64 tiles that reach the diagonal or lie below it are written.
int ozaki_gemm(cudaStream_t st, int M, int N, int K, double alpha, const double* A, long long a_rs, long long a_ks,
               double sa, const double* B, long long b_rs, long long b_ks, double sb, double beta, double* C,
               long long ldc, void* ws, size_t ws_bytes, int* status, int a_skew = 0, int slices = 8,
               int lower = 0);

// ---- refine.cu (FP64 eigenpair refinement, mixed form) ---------------------------
struct RefineInfo {
    int iterations;
    double emax[8];   // largest |E_ij| over separated pairs, per iteration
    int nclose[8];    // pairs not separated (E_ij = R_ij / 2), per iteration
    double rnorm[8];  // ||R||_F over the Z^H Z block before each update
    long long where[8];  // location of the largest correction: i | j << 20 | block << 40
    int slices[8];       // digit slices of the Gram and projection products
    int uslices[8];      // digit slices of the update product
};
size_t refine_ws(int n);
// M = [X Y] (n x n, ld n) and lambda (n/2) refined in place; n even.
// rho: separation factor of the first-order correction (pairs whose
// correction would exceed 1/rho go to Rayleigh-Ritz clusters)
int refine(cudaStream_t st, int n, const double* A, int lda, double* lambda, double* M, int maxit, void* ws,
           size_t ws_bytes, int* status, RefineInfo* info, double rho = 1024.0);
RefineInfo& last_refine_info();
// Statistics of a refinement that ran without host round trips reach
// last_refine_info() through a pinned buffer: refine_stats_flush() copies
// them in (the caller has synchronised the solve's stream first);
// refine_stats_discard() drops a copy still pending (a new solve started).
void refine_stats_flush();
void refine_stats_discard();

// ---- batched.cu (many small independent solves) ------------------------------
// Largest order of the one-CTA shared-memory path, and of the batched path
// (one CTA per matrix, working matrix in global memory above the former).
constexpr int BATCH_SMALL_MAX = 160;
constexpr int BATCH_MAX = 1024;
struct BatchProblem {
    int n, nev, lda;
    const double* A;
    double *lambda, *Zre, *Zim;  // Z: n x nev, leading dimension n; Zre == null: values only
    int* info;                   // device status word of this matrix (may be null)
};
size_t batched_small_ws(int count, const BatchProblem* probs);
// every n in [2, BATCH_MAX]; FP64 throughout; one persistent launch with the
// process-wide default configuration
int batched_small(cudaStream_t st, int count, const BatchProblem* probs, void* ws, size_t ws_bytes, int maxit);
// The uploaded item table of a batch (device pointers into the workspace).
struct BatchPlanDev {
    const void* items;  // per-matrix descriptors (batched.cu's layout)
    const int* order;   // matrices largest first
    int* next;          // work counter of the persistent launch
    int count, nmax;
};
struct BatchLaunch {
    int ctas, grid;
    size_t dyn;
    int smem_n;
};
int batched_upload(cudaStream_t st, int count, const BatchProblem* probs, void* ws, size_t ws_bytes,
                   BatchPlanDev* out);
int batched_prepare(const BatchPlanDev& d, const skew_batched_config& cfg, BatchLaunch* out);
int batched_exec(cudaStream_t st, const BatchPlanDev& d, const BatchLaunch& L, int maxit);
int batched_launch(cudaStream_t st, const BatchPlanDev& d, const skew_batched_config& cfg, int maxit);
skew_batched_config& batched_default_config();
int batched_config_check(const skew_batched_config& c);

// ---- bse.cu (the Bethe-Salpeter driver's steps around the skew solver) ------
cudaError_t bse_build_m(cudaStream_t st, int h, const double* Ar, const double* Ai, int lda, const double* Br,
                        const double* Bi, int ldb, double* M, int ldm);
cudaError_t cholesky_lower(cudaStream_t st, int N, double* M, int ld, double* NP, int* status);
cudaError_t bse_jl(cudaStream_t st, int h, double* L, int ld, double* JL, int ldj);
cudaError_t trsm_lower_t(cudaStream_t st, int N, const double* L, int ld, double* X, int ldx, int ncols);
cudaError_t bse_psi(cudaStream_t st, int h, int nev, const double* Xr, const double* Xi, int ldx,
                    const double* lambda, double* Pr, double* Pi, int ldp);

// ---- metrics.cu -------------------------------------------------------------
size_t metrics_ws(int n, int nev, int s);
int metrics(cudaStream_t st, int n, const double* A, int lda, int nev, const double* lambda, const double* X,
            const double* Y, int ldz, const int* cols, int s, double* out3, void* ws, size_t ws_bytes);

// ---- misc -------------------------------------------------------------------
// Host-side count of kernel launches issued by this library (diagnostics).
void count_launch(int k = 1);
long long launch_count();
// Records the name of a failed CUDA call (for skew_last_cuda_error) and
// returns SKEW_ERR_CUDA; cuda_ok(e) is cuda_fail(e) unless e == cudaSuccess.
int cuda_fail(cudaError_t e);
inline int cuda_ok(cudaError_t e) { return e == cudaSuccess ? 0 : cuda_fail(e); }
// Kernel timing (diagnostics): when switched on, kt_begin / kt_end bracket a
// launch with CUDA events on its stream and record its algorithmic flops.
enum {
    KT_OZAKI = 0,         // digit-slice products outside the refinement
    KT_SPLIT = 1,         // BF16 plane products (split modes)
    KT_OZAKI_REFINE = 2,  // digit-slice products of the refinement
    KT_SLICE_SPLIT = 3,   // operand splitters (digit slices, BF16 planes)
    KT_PANEL_QR = 4,      // cooperative panel QR
    KT_GEMM_F64 = 5,      // FP64 GEMM-type kernels (SYMM, rank-2k, W build, T factors, FP64 Q_band)
    KT_CHASE = 6,         // bulge chase
    KT_BISECT = 7,        // bisection
    KT_INVIT = 8,         // inverse iteration
    KT_QTRD = 9,          // Q_trd back-transform
    KT_REFINE_AUX = 10,   // O(n^2) kernels of the refinement
    KT_OTHER = 11,        // copies, conversions, D map, output
    KT_KINDS = 12
};
// kind recorded for ozaki_gemm launches (the refinement sets KT_OZAKI_REFINE
// for its n x n x n products while it runs)
extern int g_kt_ozaki_kind;
int kt_begin(cudaStream_t st);
void kt_end(cudaStream_t st, int slot, int kind, double flops);
bool kt_enabled();
// Brackets the launches issued in its lifetime as one timed record of `kind`.
struct KtScope {
    cudaStream_t st;
    int slot, kind;
    double flops;
    KtScope(cudaStream_t s, int k, double f = 0.0) : st(s), slot(kt_begin(s)), kind(k), flops(f) {}
    ~KtScope() { kt_end(st, slot, kind, flops); }
    KtScope(const KtScope&) = delete;
    KtScope& operator=(const KtScope&) = delete;
};
// elements (r, c) of an M x N result with c <= r (the lower triangle)
inline double lower_count(double M, double N) {
    return N <= M ? N * (N + 1) / 2 + (M - N) * N : M * (M + 1) / 2;
}
int device_sms();
inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Bump allocator over a caller workspace.
struct Carve {
    char* base;
    size_t cap, off = 0;
    bool ok = true;
    Carve(void* b, size_t c) : base(static_cast<char*>(b)), cap(c) {}
    template <typename T>
    T* take(size_t count) {
        size_t bytes = align_up(count * sizeof(T));
        if (off + bytes > cap) { ok = false; return nullptr; }
        T* p = reinterpret_cast<T*>(base + off);
        off += bytes;
        return p;
    }
};

}  // namespace sk
