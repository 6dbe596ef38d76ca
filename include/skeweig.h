/*
 * skeweig.h -- C ABI of a single-GPU (GB300, sm_103a) dense eigensolver for
 * real skew-symmetric matrices, following the two-step method of Penke,
 * Marek, Vorwerk, Draxl and Benner ("High Performance Solution of
 * Skew-symmetric Eigenvalue Problems with Applications in Solving the
 * Bethe-Salpeter Eigenvalue Problem", Parallel Computing).
 *
 * Problem (Sec. 1 and Algorithm 1): A = -A^T in R^{n x n}.  Its eigenvalues
 * are +-i*lambda_j (Sec. 2.1: they come in pairs and the eigenvectors of the
 * pair are complex conjugates, so half the spectrum suffices, Sec. 4.1 "50%").
 * The solver returns the nev <= floor(n/2) largest lambda_j >= 0, descending,
 * and eigenvectors Z = Z_re + i Z_im with
 *     A Z[:, j] = i * lambda[j] * Z[:, j],   Z^H Z = I.
 * conj(Z[:, j]) is the eigenvector of -i*lambda[j].
 *
 * Route (all on the device, Algorithm 1 in its two-step form, Sec. 2.1/2.3.2):
 *   full-to-band (blocked Householder panels, compact WY Q = I - V T V^T,
 *   Eq. 7; skew trailing update A <- A + V W^T - W V^T, Eqs. 8-10 with
 *   U1 = -U2), band-to-tridiagonal bulge chase (Sec. 2.3.2, skew SYR2/SYMV),
 *   the Lemma-1 link tridiag(alpha, 0, alpha) = -i D^H T D, bisection and
 *   inverse iteration on that symmetric tridiagonal (Sec. 3), back
 *   transformation by D (Algorithm 1 step 3) on real and imaginary parts
 *   separately (Sec. 2.3), then by Q_trd and Q_band (Sec. 2.1, step 3 a/b).
 *
 * Conventions for every entry point unless stated otherwise:
 *   - Matrices are column-major FP64: element (i, j) at ptr[i + j*ld].
 *   - Pointers are DEVICE pointers owned by the caller (the *_host entry is
 *     the exception).  Only the strict lower triangle of A is read; A is
 *     treated as L - L^T and is never written.
 *   - stream is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Work is stream-ordered.
 *   - Return codes: 0 success; -k argument k invalid; 1000 + j inverse
 *     iteration did not converge for eigenpair j (results still written);
 *     SKEW_ERR_* below.
 *   - Diagnostics (refinement statistics, launch count, kernel timing) are
 *     process-wide records of the most recent call.  Calls from several
 *     host threads at once are not tested; their records would mix.
 */
#ifndef SKEWEIG_H
#define SKEWEIG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SKEW_OK 0
#define SKEW_INFO_INVIT_BASE 1000      /* 1000 + j: eigenvector j did not converge */
#define SKEW_ERR_CUDA 2001             /* a CUDA runtime call failed */
#define SKEW_ERR_NOMEM 2002            /* device allocation failed */
#define SKEW_ERR_DEVICE_TIMEOUT 2003   /* a capped device-side wait gave up */
#define SKEW_ERR_UNSUPPORTED 2004      /* mode/size not supported on this GPU */
#define SKEW_ERR_NONFINITE 2005        /* A holds NaN or Inf (check_finite) */
#define SKEW_ERR_WORKSPACE 2006        /* caller workspace too small */
#define SKEW_ERR_LAUNCH 2007           /* cooperative launch could not fit */
#define SKEW_ERR_NOT_DEFINITE 2008     /* skew_bse_solve: M = J H is not positive definite */

typedef enum {
    SKEW_MODE_FP64 = 0,            /* every step in FP64 */
    SKEW_MODE_MIXED_BF16X3 = 1,    /* dense contractions (skew SYMM, rank-2k update,
                                      Q_band) as BF16x3 splits on tcgen05, Q_trd in
                                      FP32; reflectors, chase and tridiagonal solve
                                      in FP64; then, when n is even and nev = n/2,
                                      FP64 eigenpair refinement (Ogita-Aishima
                                      through -iA) with FP64-accurate tensor-core
                                      products (skew_gemm_f64acc) */
    SKEW_MODE_MIXED_INT8 = 2,      /* INT8 Ozaki splits: tcgen05 kind::i8 is not
                                      available on sm_103a -> SKEW_ERR_UNSUPPORTED */
    SKEW_MODE_MIXED_BF16X6 = 3,    /* as BF16X3 with three BF16 planes per operand
                                      (hi, mid, lo) and the six products of order
                                      <= 2: about FP32 accuracy */
    SKEW_MODE_MIXED_REFINED = 4    /* the reduction's contractions (skew SYMM,
                                      rank-2k update) and Q_band as BF16 digit-
                                      slice products on tcgen05 (6 and 5 slices:
                                      errors about 2^-42 and 2^-35), Q_trd in
                                      FP32, then the FP64 refinement with
                                      FP64-accurate products (n even, nev = n/2).
                                      Without such a complete basis (nev < n/2,
                                      odd n) nothing is refined: all products
                                      keep 8 slices (FP64-accurate) and Q_trd
                                      runs in double-float (SKEW_QTRD_DF) */
} skew_mode;

/* Fault hooks (host-side injection for tests; never fault the GPU). */
#define SKEW_FAULT_NOMEM 1         /* entry points that allocate (skew_eig_host,
                                      skew_eig_batched) fail as if the pool had no
                                      memory: SKEW_ERR_NOMEM, nothing launched */
#define SKEW_FAULT_INVIT_NOCONV 2  /* give inverse iteration zero iterations */
#define SKEW_FAULT_TINY_WAIT 4     /* the solve's waits between CTAs (panel-QR
                                      grid barrier, bulge-chase progress flags)
                                      give up after a few polls: a wait that is
                                      not satisfied at once ends the kernel with
                                      SKEW_ERR_DEVICE_TIMEOUT in the status */
#define SKEW_FAULT_NO_REFINE 8     /* mixed modes: skip the FP64 refinement */

typedef struct {
    int mode;          /* skew_mode; default SKEW_MODE_FP64 */
    int band;          /* panel width = band width b; 0 -> 64.  The kernels are
                          built for b = 64: any other value returns
                          SKEW_ERR_UNSUPPORTED */
    int check_finite;  /* 1: scan A for NaN/Inf first (SKEW_ERR_NONFINITE) */
    int fault;         /* SKEW_FAULT_* bits, tests only; 0 in production */
    int refine_iters;  /* mixed modes: maximum refinement iterations (1..8); 0 -> 8 */
    int refine_rho;    /* mixed modes: neighbouring eigenvalues whose first-order
                          correction would rotate by more than 1/refine_rho are
                          refined together by Rayleigh-Ritz (clusters of up to 16);
                          0 -> 1024 */
    int qtrd;          /* arithmetic of the Q_trd back-transform: SKEW_QTRD_* */
    int tridiag;       /* Sturm counts of the FP64 bisection: SKEW_TRIDIAG_* */
} skew_opts;

/* skew_opts.tridiag.  SKEW_TRIDIAG_AUTO (0): the FP64 bisection finish counts
 * on the zero-diagonal form of tridiag(alpha, 0, alpha) (Sec. 2.2, remark
 * after Algorithm 1): shuffled even-first it is [[0, B], [B^T, 0]] with B
 * bidiagonal, its eigenvalues >= 0 are the square roots of those of B B^T, and
 * the count of B B^T at x^2 (stationary qd transform) takes ceil(n/2) steps
 * instead of n.  SKEW_TRIDIAG_FULL (1): the Sturm count of S itself. */
#define SKEW_TRIDIAG_AUTO 0
#define SKEW_TRIDIAG_FULL 1

/* skew_opts.qtrd: SKEW_QTRD_AUTO (0) takes the mode's choice (FP64 in the FP64
 * form; FP32 SIMT when the mixed modes refine; double-float when the refined
 * mode cannot refine (nev < n/2, odd n) and FP64 in the split modes then);
 * the others force FP32 SIMT, FP64 SIMT, the tensor-core form (compact WY
 * blocks of 64 sweeps, BF16x6 tcgen05 products with FP32 accumulation,
 * FP32-level accuracy) or double-float (every value a pair of FP32 numbers,
 * exact two-product and two-sum on the FP32 pipe: about 2^-46 per operation,
 * FP64-level accuracy for the bounds at several times the FP64 pipe's rate). */
#define SKEW_QTRD_AUTO 0
#define SKEW_QTRD_FP32 1
#define SKEW_QTRD_FP64 2
#define SKEW_QTRD_TC 3
#define SKEW_QTRD_DF 4

/* Default options (FP64 mode, b = 64). */
void skew_opts_default(skew_opts* opts);

/* Human-readable text for a return code. Never NULL. */
const char* skew_eig_strerror(int code);

/* Name of the CUDA error behind the most recent SKEW_ERR_CUDA return of this
 * process (e.g. "cudaErrorLaunchOutOfResources"), or "none".  Static string;
 * never NULL. */
const char* skew_last_cuda_error(void);

/*
 * Memory of the allocating entry points (skew_eig, skew_eig_host,
 * skew_eig_batched): stream-ordered allocations from a library-owned memory
 * pool of the stream's device, created on first use, whose freed memory stays
 * reserved for the next call (repeated solves of one size allocate nothing
 * new).  skew_release_memory() returns the memory held by completed calls to
 * the system.  The *_ex entry points take caller workspace and never allocate.
 */
void skew_release_memory(void);

/*
 * Full solve, device buffers.  Eigenvalues lambda[0..nev-1] (descending,
 * >= 0) and, unless Z_re == Z_im == NULL, Z_re / Z_im (n x nev, leading
 * dimension n).  Takes its workspace from the library pool on `stream`,
 * synchronises `stream` at the end and returns the numerical status.
 * Arguments: 1 n >= 0, 2 A (n x n, ld lda), 3 lda >= max(1, n),
 * 4 0 <= nev <= n/2, 5 lambda (NULL only if nev == 0), 6/7 Z_re/Z_im (both
 * NULL or both set), 8 stream.
 */
int skew_eig(int n, const double* A, int lda, int nev, double* lambda,
             double* Z_re, double* Z_im, void* stream);

/* Bytes of device workspace skew_eig_ex needs for (n, nev, opts), with
 * eigenvectors; the _ex form takes vectors = 0 for an eigenvalues-only solve
 * (Z_re == Z_im == NULL), which needs far less. */
size_t skew_eig_workspace_size(int n, int nev, const skew_opts* opts);
size_t skew_eig_workspace_size_ex(int n, int nev, const skew_opts* opts, int vectors);

/*
 * Asynchronous full solve with caller workspace (>= skew_eig_workspace_size
 * bytes, 256-byte aligned).  ldz >= max(1, n) is the leading dimension of
 * Z_re / Z_im.  The numerical status is written to *d_info (device int) in
 * stream order; the return value only reports argument and launch errors.
 * The call neither allocates nor synchronises, and its launches can be
 * captured in a CUDA graph and replayed: the refinement of the mixed modes
 * takes its decisions (stop, digit slices of the update) on the device and
 * launches its full iteration budget, whose launches after the stop return at
 * once.  With kernel timing on (skew_kernel_timing) the refinement reads its
 * decisions on the host instead, synchronising `stream` once per iteration.
 * Arguments are numbered as in skew_eig with 8 ldz, 9 opts (NULL = default),
 * 10 workspace, 11 ws_bytes, 12 d_info, 13 stream.
 */
int skew_eig_ex(int n, const double* A, int lda, int nev, double* lambda,
                double* Z_re, double* Z_im, int ldz, const skew_opts* opts,
                void* workspace, size_t ws_bytes, int* d_info, void* stream);

/*
 * Full solve from HOST buffers (A, lambda, Z_re, Z_im in host memory, ideally
 * pinned).  Copies A in, solves with `opts` (NULL = default), copies results
 * out; synchronises `stream`.  Argument numbering as skew_eig with 8 opts,
 * 9 stream.
 */
int skew_eig_host(int n, const double* A, int lda, int nev, double* lambda,
                  double* Z_re, double* Z_im, const skew_opts* opts, void* stream);

/*
 * Batched solve: `count` independent problems, each as in skew_eig (matrix b:
 * order n[b], device A[b] with leading dimension lda[b], nev[b] eigenpairs
 * into device lambda[b], Z_re[b], Z_im[b] of leading dimension n[b]).  The
 * size arrays and the pointer arrays are host arrays; Z_re == Z_im == NULL
 * (the arrays) or Z_re[b] == Z_im[b] == NULL (one matrix) asks for
 * eigenvalues only.  Orders 2..1024 are solved together in one persistent
 * launch (see skew_batched_config below: each CTA takes whole matrices,
 * largest first, and runs unblocked Householder tridiagonalisation with the
 * matrix in shared or global memory, bisection, inverse iteration and the
 * back-transform), always in FP64; larger orders run the two-step solve of
 * skew_eig_ex one after another in `opts`' mode.  Not in the paper (it solves one matrix per run).
 * Asynchronous on `stream`.  skew_eig_batched takes its workspace from the
 * library pool (stream-ordered, freed on the stream) and reports no per-matrix
 * status; skew_eig_batched_ex takes a caller workspace of at least
 * skew_eig_batched_workspace_size(count, n, nev, opts) bytes and a device
 * array d_info[count] (may be NULL) that receives 0 or 1000 + j per matrix.
 * Returns 0, -1 (count < 0), -k for the first invalid per-matrix argument
 * (2 n, 3 A, 4 lda, 5 nev, 6 lambda, 7 Z), SKEW_ERR_WORKSPACE, SKEW_ERR_NOMEM,
 * SKEW_ERR_UNSUPPORTED (INT8 mode) or SKEW_ERR_CUDA.
 */
size_t skew_eig_batched_workspace_size(int count, const int* n, const int* nev, const skew_opts* opts);
int skew_eig_batched(int count, const int* n, const double* const* A, const int* lda, const int* nev,
                     double* const* lambda, double* const* Z_re, double* const* Z_im,
                     const skew_opts* opts, void* stream);
int skew_eig_batched_ex(int count, const int* n, const double* const* A, const int* lda,
                        const int* nev, double* const* lambda, double* const* Z_re,
                        double* const* Z_im, const skew_opts* opts, void* workspace,
                        size_t ws_bytes, int* d_info, void* stream);

/*
 * Batched solve as a plan: one persistent launch for the whole batch.
 * Not in the paper (it solves one matrix per run; each matrix here follows
 * Algorithm 1 in its one-step form: unblocked Householder tridiagonalisation,
 * Lemma-1 link, bisection and inverse iteration, D map and back
 * transformation, FP64 throughout).
 *
 * skew_batched_config sets the launch: ctas_per_sm (1..4) CTAs of 256 threads
 * per SM take matrices from a device work counter, largest first; orders up to
 * smem_max_n (0..160; capped by the shared memory of ctas_per_sm CTAs per SM)
 * keep the working matrix in shared memory, larger ones in global memory.
 * skew_batched_set_config / get_config hold the process-wide default used by
 * skew_eig_batched(_ex) and by plans created with cfg == NULL (initially
 * ctas_per_sm = 2, smem_max_n = 112).
 *
 * skew_batched_plan_create checks the batch (arguments as skew_eig_batched_ex:
 * 2 n, 3 A, 4 lda, 5 nev, 6 lambda, 7 Z; every order must be <= 1024, else
 * SKEW_ERR_UNSUPPORTED), lays the per-matrix descriptors out in the caller's
 * workspace (at least skew_eig_batched_workspace_size bytes), uploads them on
 * `stream` and synchronises it, and fixes the launch parameters.  The device
 * buffers named in the call must stay valid while the plan is used.
 * skew_batched_plan_exec then only clears d_info (may be NULL; per matrix 0 or
 * 1000 + j) and the work counter and launches the persistent kernel: no host
 * synchronisation and no allocation, so the call can be captured into a CUDA
 * graph and replayed.  skew_batched_plan_tune times every candidate
 * configuration on the plan's batch (one warm-up and two timed runs each, CUDA
 * events on `stream`), keeps the fastest in the plan and returns it; cand_*
 * (may be NULL) receive up to cap candidates and their times in ms; returns
 * the number of candidates timed or a negative / SKEW_ERR_* code.
 */
typedef struct {
    int ctas_per_sm;
    int smem_max_n;
    int reserved[2];
} skew_batched_config;
typedef struct skew_batched_plan skew_batched_plan;
int skew_batched_set_config(const skew_batched_config* cfg);
void skew_batched_get_config(skew_batched_config* cfg);
int skew_batched_plan_create(int count, const int* n, const double* const* A, const int* lda, const int* nev,
                             double* const* lambda, double* const* Z_re, double* const* Z_im,
                             const skew_batched_config* cfg, void* workspace, size_t ws_bytes, int* d_info,
                             void* stream, skew_batched_plan** plan);
int skew_batched_plan_exec(skew_batched_plan* plan, void* stream);
int skew_batched_plan_tune(skew_batched_plan* plan, skew_batched_config* best, int* cand_ctas,
                           int* cand_smem, float* cand_ms, int cap, void* stream);
void skew_batched_plan_get_config(const skew_batched_plan* plan, skew_batched_config* cfg);
void skew_batched_plan_destroy(skew_batched_plan* plan);

/*
 * The Bethe-Salpeter eigenproblem around the skew solver (Sec. 3, Theorem 1,
 * the four steps of the structure-preserving method):
 *   H_BS = [[A, B], [-conj(B), -conj(A)]],  A = A^H, B = B^T (h x h complex),
 * definite (Omega = [[A, B], [conj(B), conj(A)]] positive definite).  Step 1
 * forms M = J H = [[Re(A+B), Im(A-B)], [-Im(A+B), Re(A-B)]] (2h x 2h, real
 * symmetric positive definite, Eq. SymmetricM), step 2 its Cholesky factor
 * M = L L^T, step 3 solves the skew-symmetric eigenproblem of K = L^T J L
 * (J = [[0, I], [-I, 0]]) with skew_eig_ex in opts' mode, step 4 transforms
 * back: x = L^-T z and psi = Q x with the unitary Q = [[I, -iI], [I, iI]] /
 * sqrt(2) of Theorem 1.  Returns the nev largest positive eigenvalues of H_BS
 * (descending) in lambda and psi = psi_re + i psi_im (2h x nev, ld ldpsi)
 * with H_BS psi = psi diag(lambda) and psi^H S psi = I, S = diag(I, -I).
 * All matrices are device, column-major FP64; A and B are given as real and
 * imaginary parts (ld lda / ldb; A is read whole, B whole).  Asynchronous on
 * `stream`; the numerical status goes to *d_info: 0, SKEW_ERR_NOT_DEFINITE
 * (a Cholesky pivot not positive), 1000 + j (inverse iteration), or
 * SKEW_ERR_*.  Workspace: skew_bse_workspace_size(h, nev, opts) bytes.
 * Arguments: 1 h >= 1, 2-3 A_re / A_im, 4 lda >= h, 5-6 B_re / B_im,
 * 7 ldb >= h, 8 1 <= nev <= h, 9 lambda, 10-11 psi_re / psi_im,
 * 12 ldpsi >= 2h, 14 workspace, 16 d_info.
 */
size_t skew_bse_workspace_size(int h, int nev, const skew_opts* opts);
int skew_bse_solve(int h, const double* A_re, const double* A_im, int lda, const double* B_re,
                   const double* B_im, int ldb, int nev, double* lambda, double* psi_re, double* psi_im,
                   int ldpsi, const skew_opts* opts, void* workspace, size_t ws_bytes, int* d_info,
                   void* stream);

/* Stages timed by skew_eig_profile (Algorithm 1, two-step form):
 * 0 ingest (copy of the strict lower triangle), 1 full-to-band reduction,
 * 2 band pack, 3 bulge chase, 4 tridiagonal solve (bisection + inverse
 * iteration), 5 D map, 6 Q_trd back-transform, 7 Q_band back-transform,
 * 8 FP64 refinement (mixed modes), 9 output copy. */
#define SKEW_NSTAGES 10

/*
 * skew_eig_ex plus CUDA events between the stages above, recorded on
 * `stream`; synchronises `stream`, writes the stage durations in milliseconds
 * to the HOST array stage_ms[SKEW_NSTAGES] and returns the numerical status
 * (0, 1000 + j or SKEW_ERR_*).  Arguments as skew_eig_ex; 12 stage_ms.
 */
int skew_eig_profile(int n, const double* A, int lda, int nev, double* lambda,
                     double* Z_re, double* Z_im, int ldz, const skew_opts* opts,
                     void* workspace, size_t ws_bytes, float* stage_ms, void* stream);

/*
 * Accuracy of a computed decomposition (Algorithm 1 "Ensure"), on the device,
 * restricted to the columns cols[0..ncols-1] of Z (cols == NULL: all nev
 * columns, ncols == nev; cols is a DEVICE int array):
 *   out3[0] = ||A Z_S - Z_S diag(i lambda_S)||_F
 *   out3[1] = ||Z_S^H Z - I_S||_F   (I_S: the columns S of the identity)
 *   out3[2] = ||A||_F
 * out3 is a HOST array; the call synchronises `stream`.  Workspace of at
 * least skew_metrics_ws(n, nev, ncols) bytes.
 */
size_t skew_metrics_ws(int n, int nev, int ncols);
int skew_eig_metrics(int n, const double* A, int lda, int nev, const double* lambda,
                     const double* Z_re, const double* Z_im, int ldz, const int* cols,
                     int ncols, double* out3, void* ws, size_t ws_bytes, void* stream);

/*
 * Mixed-precision dense contraction on the tensor cores (tcgen05, BF16
 * inputs, FP32 accumulation in TMEM), the primitive of the mixed form:
 *   C = alpha * A B^T + beta * C            (lower == 0)
 *   C[lower 128-tiles] += alpha * A B^T, diagonal set to 0   (lower == 1, M == N)
 * with every FP64 operand split into hi = bf16(x), lo = bf16(x - hi) and the
 * product taken as hi*hi + lo*hi + hi*lo (relative error about 2^-16 per
 * product plus K * 2^-24 from the FP32 sums).  Not in the paper.
 * A is M x K with element (i, k) at A[i*a_rs + k*a_ks], B is N x K with
 * (j, k) at B[j*b_rs + k*b_ks] (device, FP64); C is column-major FP64, ld
 * ldc.  Workspace >= skew_gemm_bf16x3_ws(M, N, K) bytes (the BF16 planes).
 * planes = 3 splits into hi, mid, lo and keeps the six products of order
 * <= 2 (BF16x6, about 2^-24 relative).
 * Arguments: 1 M, 2 N, 3 K >= 1, 13 ldc >= M, 14 lower, 15 planes (2 or 3).
 */
size_t skew_gemm_bf16x3_ws(int M, int N, int K);
int skew_gemm_bf16x3(int M, int N, int K, double alpha, const double* A,
                     long long a_rs, long long a_ks, const double* B, long long b_rs,
                     long long b_ks, double beta, double* C, int ldc, int lower,
                     int planes, void* ws, size_t ws_bytes, int* d_status, void* stream);

/*
 * FP64-accurate product on the BF16 tensor cores, the primitive of the
 * eigenpair refinement of the mixed form:  C = alpha * A B^T + beta * C.
 * Each row of A and of B is scaled by a power of two and cut into 8 digit
 * slices of 7 bits (integers BF16 holds exactly); slice products of equal
 * order are summed in FP32 over K groups of 512 (exactly for the six leading
 * orders) and folded in double-float (about 48 bits), so the error is a few
 * units of 2^-48 times the row-max products, independent of cancellation.
 * Not in the paper.
 * Layouts and argument numbering as skew_gemm_bf16x3 (no lower mode).
 * skew_gemm_f64acc_ex adds: slices (1..8; the products of slice pairs of
 * order < slices are kept, error about 2^-7 slices of the row-max products,
 * -14 otherwise) and lower (1: only the 128 x 64 output tiles that reach or
 * lie below the diagonal are written, the others are left untouched; -15
 * otherwise).  Workspace: skew_gemm_f64acc_ws(M, N, K).
 */
size_t skew_gemm_f64acc_ws(int M, int N, int K);
int skew_gemm_f64acc(int M, int N, int K, double alpha, const double* A,
                     long long a_rs, long long a_ks, const double* B, long long b_rs,
                     long long b_ks, double beta, double* C, int ldc,
                     void* ws, size_t ws_bytes, int* d_status, void* stream);
int skew_gemm_f64acc_ex(int M, int N, int K, double alpha, const double* A,
                     long long a_rs, long long a_ks, const double* B, long long b_rs,
                     long long b_ks, double beta, double* C, int ldc, int slices, int lower,
                     void* ws, size_t ws_bytes, int* d_status, void* stream);

/*
 * FP64 eigenpair refinement on its own (the last stage of the mixed modes):
 * given approximate lambda (n/2) and Z_re / Z_im (n x n/2, ld ldz, device)
 * of skew A (n even), run at most `iters` Ogita-Aishima iterations through
 * H = -iA with FP64-accurate tensor-core products and overwrite them.
 * Asynchronous (the convergence test runs on the device; see skew_eig_ex).
 * Workspace >= skew_refine_ws(n) bytes.  Not in the paper.
 * Arguments: 1 n (even, >= 2), 2 A, 3 lda, 4 lambda, 5/6 Z_re/Z_im, 7 ldz,
 * 8 iters >= 1.
 */
size_t skew_refine_ws(int n);
int skew_refine(int n, const double* A, int lda, double* lambda, double* Z_re,
                double* Z_im, int ldz, int iters, void* ws, size_t ws_bytes,
                int* d_status, void* stream);

/* Statistics of the most recent refinement in this process (diagnostics;
 * read them after synchronising the stream of that solve, whose record
 * arrives in stream order): returns the number of iterations; emax[i] =
 * largest first-order correction
 * |E_jk| of iteration i, nclose[i] = pairs not separated enough for it
 * (up to cap entries each, either pointer may be NULL). */
int skew_refine_stats(double* emax, int* nclose, int cap);
/* Same run: rnorm[i] = ||I - Z^H Z||_F seen by iteration i before its update,
 * where[i] = location of the largest correction (row | column << 20 |
 * block << 40, block 0 = Z^H Z part, 1 = conjugate part). */
int skew_refine_trace(double* rnorm, long long* where, int cap);
/* Same run: digit slices (1..8; 8 = FP64-accurate) of iteration i's Gram and
 * projection products (slices[i]) and of its update product (uslices[i]). */
int skew_refine_slices(int* slices, int* uslices, int cap);

/* Number of CUDA kernels this library has launched in this process
 * (diagnostics; counts host-side launch calls). */
long long skew_launch_count(void);

/* Kernel timing (diagnostics).  skew_kernel_timing(1) clears the record and
 * from then on brackets the library's launches (one record per launch or per
 * group of launches of one kind) with CUDA events on the stream they go to
 * (two event records each); skew_kernel_timing(0) stops.  Records wait in a
 * pool of 16384 until they are folded into per-kind totals: at the end of
 * every skew_eig_profile call (its solve is then complete) and by each of the
 * read functions below.  A launch that finds the pool full is not recorded and
 * counted as dropped (skew_kernel_timing_dropped).  Not thread-safe: one
 * solving thread per process while it is on.
 * skew_kernel_timing_read folds the outstanding records (waiting for their
 * events) and returns, summed over the records of one kind since timing was
 * switched on, the event-measured time (*ms), the algorithmic flops (*flops;
 * for the two product kinds: 2 M N K per kept slice or plane product over the
 * outputs the launch writes, 0 for the others) and the record count.  Returns
 * 0, -1 for an unknown kind, -2 when records were dropped (the totals miss
 * them), or SKEW_ERR_CUDA. */
#define SKEW_KERNEL_OZAKI 0        /* ozaki_gemm_kernel outside the refinement (reduction, Q_band) */
#define SKEW_KERNEL_SPLIT 1        /* BF16x3 / BF16x6 split product (umma_gemm_kernel) */
#define SKEW_KERNEL_OZAKI_REFINE 2 /* ozaki_gemm_kernel inside the refinement (n x n x n) */
#define SKEW_KERNEL_SLICE_SPLIT 3  /* operand splitters (digit slices, BF16 planes) */
#define SKEW_KERNEL_PANEL_QR 4     /* cooperative panel QR */
#define SKEW_KERNEL_GEMM_F64 5     /* FP64 GEMM-type kernels (SYMM, rank-2k, W build, T, FP64 Q_band) */
#define SKEW_KERNEL_CHASE 6        /* bulge chase */
#define SKEW_KERNEL_BISECT 7       /* bisection */
#define SKEW_KERNEL_INVIT 8        /* inverse iteration */
#define SKEW_KERNEL_QTRD 9         /* Q_trd back-transform */
#define SKEW_KERNEL_REFINE_AUX 10  /* O(n^2) kernels of the refinement */
#define SKEW_KERNEL_OTHER 11       /* copies, conversions, D map, output */
#define SKEW_KERNEL_KINDS 12
int skew_kernel_timing(int enable);
int skew_kernel_timing_read(int kind, double* ms, double* flops, long long* launches);
long long skew_kernel_timing_dropped(void);
/* Timeline of the records folded last (after a skew_eig_profile call: the
 * records of that solve): for the first min(cap, records) records in launch
 * order, kinds[i] (SKEW_KERNEL_*), and the start and end of record i in
 * milliseconds after the start of record 0 (events of different streams, as
 * the side stream of the band reduction, interleave).  Folds the outstanding
 * records first.  Any output pointer may be NULL.  Returns the number of
 * records written, -1 for cap < 0, or SKEW_ERR_CUDA. */
int skew_kernel_timeline(int cap, int* kinds, double* start_ms, double* end_ms);

/* ------------------------------------------------------------------------
 * Stage entry points (the steps of Algorithm 1 one at a time; used by the
 * per-stage parity tests).  Each takes a caller workspace of at least the
 * size its *_ws function returns, and a device status word *d_status (int,
 * set to a nonzero SKEW_ERR_* / 1000+j code on a device-side failure; the
 * caller zeroes it).
 * --------------------------------------------------------------------- */

/* Full-to-band reduction (Sec. 2.3.2, Eqs. 7-10), in place on W (n x n, ld
 * ldw).  On entry W's strict lower triangle holds A.  On exit, for panel
 * p = 0..P-1 (P = max(0, floor((n-2)/b))): the lower triangles of the
 * diagonal b x b blocks and the upper triangles of the blocks
 * W[(p+1)b:(p+2)b, pb:(p+1)b] hold the band (lower bandwidth b); the
 * Householder vectors v (unit leading entry implicit) of panel p are stored
 * below that, column pb+i holding v_i in rows (p+1)b+i+1 .. n-1 (Sec. 2.1:
 * vectors stored in place of the eliminated columns).  Tfac (P x b x b,
 * column-major b x b per panel) receives the upper-triangular T of
 * Q_p = I - V_p T_p V_p^T.  b is a multiple of 64. */
size_t skew_band_reduce_ws(int n, int b);
int skew_band_reduce(int n, double* W, int ldw, int b, double* Tfac,
                     void* ws, size_t ws_bytes, int* d_status, void* stream);

/* Copy the band out of a reduced W into lower band storage AB ((2b+1) x n,
 * ld ldab >= 2b+1): AB[d + c*ldab] = band(c+d, c), d = 0..b; rows b+1..2b
 * (room for the bulge) are zeroed. */
int skew_band_pack(int n, int b, const double* W, int ldw, double* AB, int ldab,
                   void* stream);

/* Band-to-tridiagonal bulge chase (Sec. 2.3.2).  AB as produced by
 * skew_band_pack, overwritten.  Output alpha[0..n-2] with T[c, c+1] =
 * alpha[c] (the Lemma-1 link input) and the chase reflectors: sweep s,
 * step k has v (length b, v[0] = 1, zero-padded) at Vtrd[(k*(n-2) + s)*b]
 * and tau at tautrd[k*(n-2) + s], k < skew_chase_steps(n, b). */
int skew_chase_steps(int n, int b);
size_t skew_chase_ws(int n, int b);
int skew_band_to_tridiag(int n, int b, double* AB, int ldab, double* alpha,
                         double* Vtrd, double* tautrd, void* ws, size_t ws_bytes,
                         int* d_status, void* stream);

/* Symmetric tridiagonal solve for S = tridiag(alpha, 0, alpha) (Lemma 1,
 * Sec. 3: bisection + inverse iteration): the nev largest eigenvalues
 * (descending) into lambda and, if Q != NULL, eigenvectors into Q (n x nev,
 * ld ldq) with each vector's largest-modulus entry positive.  Here
 * 1 <= nev <= n. */
size_t skew_tridiag_ws(int n, int nev);
int skew_tridiag_eig(int n, const double* alpha, int nev, double* lambda,
                     double* Q, int ldq, void* ws, size_t ws_bytes,
                     int* d_status, void* stream);

/*
 * skew_tridiag_eig without any device allocation: the same computation and
 * results, with the scratch memory in a static device array of
 * SKEW_NOALLOC_SCRATCH_BYTES (6 MiB) that every device loading the library
 * holds until the process exits.  For callers that may not allocate device
 * memory (their application owns every allocation, or cudaMalloc's device
 * synchronisation is not allowed); the paper has no counterpart.
 * Limit: the call fits when skew_tridiag_ws(n, nev) <= SKEW_NOALLOC_SCRATCH_BYTES
 * (with Q; about 41 * n * nev bytes for nev >= 64, e.g. n = 512, nev = 256);
 * larger sizes return SKEW_ERR_WORKSPACE.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress) and caches it; make
 * that first call before any stream capture.  The address belongs to the
 * current device: `stream` must be a stream of the current device (or NULL),
 * otherwise SKEW_ERR_UNSUPPORTED.  All calls share the array, which keeps the
 * previous call's contents: calls that overlap on the GPU race, so serialise
 * them.  Arguments 1 n >= 1, 2 alpha (device, n-1; may be NULL when n = 1),
 * 3 1 <= nev <= n, 4 lambda (device, nev), 5 Q (device or NULL), 6 ldq >= n,
 * 7 d_status (device int, zeroed by the caller), 8 stream.
 */
#define SKEW_NOALLOC_SCRATCH_BYTES (6u << 20)
int skew_tridiag_eig_noalloc(int n, const double* alpha, int nev, double* lambda,
                             double* Q, int ldq, int* d_status, void* stream);

/* Algorithm 1 step 3: X + iY = D Q, D = diag(i^r), r = 0..n-1. */
int skew_dmap(int n, int k, const double* Q, int ldq, double* X, double* Y,
              int ldz, void* stream);

/* Z <- Q_trd Z (Sec. 2.1 step 3a) for the chase reflectors above; Z is
 * n x k, ld ldz. */
int skew_apply_qtrd(int n, int b, const double* Vtrd, const double* tautrd,
                    double* Z, int ldz, int k, void* stream);

/* Z <- Q_trd Z in FP32 (Sec. 2.1 step 3a; the FP32-level form of the mixed
 * modes) from FP32 reflectors: V32 holds v (64 floats, v[0] = 1, zero padded)
 * of sweep s, step k at slot k * nsw64 + s and tau32 its tau at the same slot
 * (nsw64 = n - 2 rounded up to a multiple of 64; the taus of steps a sweep does
 * not have are zero).  Z is FP32, n x k, ld ldz.  tensor = 0: reflector by
 * reflector on the FP32 pipe; tensor = 1: 64-sweep blocks in compact WY form
 * (Eq. 7) applied by tcgen05 BF16x6 products, workspace
 * skew_apply_qtrd_f32_ws(n, 1) bytes (the blocks' operands).  d_status is a
 * device int set on a device-side failure.  Arguments 1 n, 2 b (64),
 * 3 V32/tau32, 6 ldz, 7 k, 8 tensor (0 or 1), 11 d_status. */
size_t skew_apply_qtrd_f32_ws(int n, int tensor);
int skew_apply_qtrd_f32(int n, int b, const float* V32, const float* tau32, float* Z, int ldz, int k,
                        int tensor, void* ws, size_t ws_bytes, int* d_status, void* stream);

/* Z <- Q_trd Z (Sec. 2.1 step 3a) in double-float arithmetic on the FP32 pipe
 * (SKEW_QTRD_DF) from the FP64 reflectors of skew_band_to_tridiag (layout of
 * skew_apply_qtrd); Z is FP64, n x k, ld ldz.  d_status is a device int set
 * on a device-side failure (SKEW_ERR_DEVICE_TIMEOUT).  Arguments 1 n, 2 b (64),
 * 3 Vtrd/tautrd, 6 ldz, 7 k, 8 d_status. */
int skew_apply_qtrd_df(int n, int b, const double* Vtrd, const double* tautrd, double* Z, int ldz, int k,
                       int* d_status, void* stream);

/* Z <- Q_band Z (Sec. 2.1 step 3b) for a W / Tfac pair produced by
 * skew_band_reduce; Z is n x k, ld ldz. */
size_t skew_qband_ws(int n, int b, int k);
int skew_apply_qband(int n, int b, const double* W, int ldw, const double* Tfac,
                     double* Z, int ldz, int k, void* ws, size_t ws_bytes,
                     void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SKEWEIG_H */
