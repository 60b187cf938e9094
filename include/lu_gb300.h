/*
 * lu_gb300.h -- C ABI of a GB300 (sm_103a) library for blocked right-looking
 * LU factorization with partial pivoting and depth-1 static look-ahead, after
 * "Programming Parallel Dense Matrix Factorizations with Look-Ahead and
 * OpenMP" (arXiv 1804.07017).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are column-major: element (i, j) of a matrix with leading
 *    dimension ld lives at ptr[i + j*ld].  ld >= max(1, rows).
 *  - Every matrix, vector and pivot pointer is a DEVICE pointer owned by the
 *    caller, unless an argument says "host".  The library never frees or
 *    retains caller memory beyond the call.
 *  - Pivots follow LAPACK getrf: ipiv[j] (int32, 1-based) is the row that was
 *    interchanged with row j+1 at elimination step j (sequential interchanges,
 *    not a permutation vector).  The factors are stored in LAPACK layout:
 *    P A = L U, unit-lower L strictly below the diagonal, U on and above it.
 *  - Workspace (exchange slots, counters, pivot plans, low-precision operand
 *    copies, residual vectors) is owned by the handle, allocated on first use
 *    with cudaMalloc, grown when a larger problem arrives and freed by
 *    lu_destroy.
 *  - Calls named *_ex are asynchronous on the handle's stream (lu_set_stream)
 *    and report device-side outcomes through a caller-provided device int32
 *    `info`.  The plain calls (lu_factor, lu_solve) use a process-wide default
 *    handle on the legacy default stream and synchronise before returning.
 *
 * Return codes: 0 success; -i the i-th argument is invalid; the runtime errors
 * below; for factorizations a positive value i means U(i,i) is exactly zero
 * (the factorization is still completed, as in LAPACK getrf).
 * No call aborts, traps or throws across this boundary.
 */
#ifndef LU_GB300_H
#define LU_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LU_SUCCESS 0
#define LU_ERR_CUDA (-101)        /* a CUDA runtime/driver call failed (see lu_last_error) */
#define LU_ERR_NOMEM (-102)       /* workspace allocation failed */
#define LU_ERR_TIMEOUT (-103)     /* a bounded device-side wait expired; results are invalid */
#define LU_ERR_UNSUPPORTED (-104) /* the requested size/type/precision is not supported */
#define LU_ERR_HANDLE (-105)      /* null or destroyed handle */
#define LU_ERR_IO (-106)          /* a tuning-table file could not be read, parsed or written */
#define LU_WARN_NOT_CONVERGED (0x40000000) /* lu_gesv_mixed: tol not reached in max_iter */

typedef struct lu_context *lu_handle;

/* Arithmetic type of a factorization / of the matrix storage. */
typedef enum { LU_F64 = 0, LU_F32 = 1 } lu_dtype;

/* Operand precision of the tensor-core trailing update in the mixed-precision
 * path (panels, triangular solves and the stored factors stay FP32; the
 * products accumulate in FP32). */
typedef enum {
    LU_TU_BF16 = 0, /* bf16 operands, tcgen05.mma kind::f16 */
    LU_TU_FP16 = 1, /* fp16 operands, tcgen05.mma kind::f16 */
    LU_TU_FP8 = 2,  /* e4m3 operands with power-of-two block scales (one per row of L21,
                       one per column of U12), kind::f8f6f4; nb a multiple of 128 */
    LU_TU_F32 = 3,  /* FP32 on the CUDA cores (no tensor cores; a reference point) */
    LU_TU_BF16X3 = 4, /* split bf16: each FP32 operand as hi + lo bf16, three products
                         (hi*hi + hi*lo + lo*hi) accumulated in FP32, kind::f16 */
    LU_FULL_F64 = 5, /* lu_gesv_mixed only: FP64 factors and FP64 correction solves
                        (the plain FP64 path, refined the same way) */
    LU_TU_BF16X6 = 6 /* split bf16 in three parts, the six products of weight >= 2^-16
                        (the full FP32 significand), kind::f16 */
} lu_prec;

/* Options of a blocked factorization (Sec. 3-4 of the paper). */
typedef struct {
    int nb;        /* algorithmic block size b (panel width), 1..1024; 0 = the value
                      lu_tune_nb measured for this factorization kind and n on
                      this device, or 256 when none was measured */
    int lookahead; /* 0: no look-ahead, the PF(k); TU(k) loop of Listing 3.
                      1: depth-1 static look-ahead of Listing 5: PU(k+1) (the
                         left part of TU_k plus PF_{k+1}) runs concurrently with
                         TU_right(k).
                      2: depth 2 (Sec. 4 notes that deeper look-ahead follows
                         the same pattern): the high-priority stream also applies
                         TU_k to panel k+2, so PF_{k+1} waits only for TU_k on its
                         own columns and never for TU_right(k-1); the right update
                         starts after panel k+2 */
    int steal;     /* 1: the CTAs freed by PU(k+1) join TU_right(k) (the GPU
                      analogue of the malleable BLAS of Sec. 4.2); 0: they do not */
    int leaf;      /* column width handled by one panel-factorization leaf
                      kernel inside the recursive panel (0 = automatic) */
    int pf_ctas;   /* maximum CTAs of a panel-factorization leaf, also capping the
                      thread-block cluster of a cluster leaf (0 = automatic: the
                      largest cluster that fits) */
    int tu_reserve; /* with look-ahead: SMs the right trailing update leaves to the
                      panel path (and that rejoin it as stealing CTAs once the
                      panel is done); 0 = automatic (the tuned value, else a
                      sixth of the SMs) */
    int nsched;    /* > 0: per-step block sizes (the GPU form of the paper's
                      early termination, Sec. 4.2: b adjusted from step to step);
                      step k eliminates sched[k] columns, the last entry repeats,
                      the final step takes what remains; 0 = the fixed nb */
    const int32_t *sched; /* host array of nsched block sizes, each 1..1024 (the
                      tensor-core update needs multiples of 64, FP8 of 128; other
                      widths run that step's update on the CUDA cores); read
                      during the call only */
    int rtm;       /* 1: instead of the static look-ahead, the runtime-task
                      schedule the paper compares against (Sec. 3.3, Listing 4):
                      every PF(k), every block-column update TU(k, j) and the
                      interchanges of panel k on the columns left of it are
                      tasks of one dependency DAG, replayed as a CUDA graph whose
                      executor starts each task when its inputs are ready (any
                      look-ahead depth); PF(k) and TU(k, k+1) run at high
                      priority.  FP64/FP32 factorizations on the CUDA cores
                      (lu_factor_ex, lu_potrf_ex); 0 = static look-ahead */
    int pf_sms;    /* > 0, with look-ahead: an SM partition of at least this many
                      SMs (rounded up to the device's granularity, 8 on GB300)
                      reserved for the panel-factorization leaves, and the right
                      trailing update confined to the other SMs (two green
                      contexts: process-local, no device setting changes); the
                      factors are bit-identical to pf_sms = 0.  If the device or
                      driver cannot partition, the call runs without a partition.
                      A repeated mixed factorization is then not replayed as a
                      graph.  0 = no partition */
} lu_opts;

/* Fills *opts with the defaults (nb = 256, lookahead = 1, steal = 1, automatic
 * rest, no schedule). */
void lu_default_opts(lu_opts *opts);

/* Handle lifetime.  lu_create returns 0 or LU_ERR_CUDA/LU_ERR_NOMEM. */
int lu_create(lu_handle *handle);
int lu_destroy(lu_handle handle);
/* Sets the CUDA stream (a cudaStream_t passed as void*, NULL = legacy default)
 * on which the handle's asynchronous calls are ordered. */
int lu_set_stream(lu_handle handle, void *stream);

/* Total number of kernels this library has launched in this process (all
 * handles).  Monotone; used to count launches inside a timed region. */
int64_t lu_launch_count(void);
/* Text of the last CUDA error seen by the library (static storage). */
const char *lu_last_error(void);

/* Kernel classes of the built-in launch profiler. */
enum {
    LU_K_PANEL = 0,     /* panel-factorization leaf (RL1) */
    LU_K_LASWP = 1,     /* interchange plans and row interchanges */
    LU_K_TRSM = 2,      /* RL2 */
    LU_K_GEMM = 3,      /* RL3 on the CUDA cores */
    LU_K_TC_UPDATE = 4, /* RL3 on the tensor cores */
    LU_K_PACK = 5,      /* operand rounding / packing for the tensor cores */
    LU_K_SOLVE = 6,     /* triangular solves and row permutations of a solve */
    LU_K_RESIDUAL = 7,  /* FP64 residuals, norms, conversions of the refinement */
    LU_K_OTHER = 8,
    LU_K_BATCHED = 9,   /* the persistent batched factorization + solve */
    LU_K_COUNT = 10
};
/* lu_profile_enable(mask): from now on every kernel launch of a class whose bit
 * (1 << class) is set in mask is bracketed by two CUDA events recorded on its
 * own stream (mask 0 = off, -1 = all).  lu_profile_read synchronises the device
 * and returns, for one class, the number of launches since the last reset, the
 * sum of their event-to-event durations (ms) and of their algorithmic bytes
 * and flops (host pointers, any may be NULL).  lu_profile_reset clears. */
int lu_profile_enable(int mask);
/* lu_profile_stride(every): with every = s > 1 only one launch in s of each
 * profiled class (the 1st, the (s+1)th, ...) carries events, so that a profile
 * taken inside a timed region perturbs it less; launches and durations read
 * back are those of the sampled launches.  every <= 1 samples all (default). */
int lu_profile_stride(int every);
int lu_profile_reset(void);
int lu_profile_read(int kclass, int64_t *launches, double *ms, double *bytes, double *flops);

/*
 * lu_factor -- P A = L U of an n x n FP64 matrix, in place (LU_blk, RL1-RL3,
 * Sec. 3; depth-1 look-ahead, Sec. 4).
 *   n     order of A, n >= 0 (n = 0 is a no-op)
 *   A     device, n x n column-major, leading dimension lda; overwritten by L\U
 *   lda   >= max(1, n)
 *   ipiv  device int32[n]; receives the pivots (LAPACK convention)
 *   nb    block size b, 1..1024, or 0 for the tuned value (see lu_tune_nb)
 * Synchronises the legacy default stream.  Returns 0, i > 0 (first exactly
 * zero U(i,i)), -i for an invalid argument, or a runtime error code.
 */
int lu_factor(int64_t n, double *A, int64_t lda, int32_t *ipiv, int nb);

/*
 * lu_solve -- X = A^{-1} B from the output of lu_factor (the getrs that pairs
 * with getrf: apply the interchanges, solve with unit-lower L, then with U).
 *   LU, ipiv  device, as returned by lu_factor with lda = n
 *   B         device, n x nrhs, leading dimension n; overwritten by X
 * Synchronises.  Returns 0, -i, or a runtime error code.
 */
int lu_solve(int64_t n, int64_t nrhs, const double *LU, const int32_t *ipiv, double *B);

/*
 * lu_factor_ex -- as lu_factor, for FP64 or FP32 storage and arithmetic,
 * with explicit options, asynchronous on the handle's stream.
 *   info  device int32[1]; receives 0, the first zero pivot i > 0, or
 *         LU_ERR_TIMEOUT if a bounded device wait expired.
 * Returns 0 (enqueued), -i, or a runtime error code.
 */
int lu_factor_ex(lu_handle handle, lu_dtype dtype, int64_t n, void *A, int64_t lda,
                 int32_t *ipiv, const lu_opts *opts, int32_t *info);

/*
 * lu_solve_ex -- X = A^{-1} B from lu_factor_ex output (same dtype);
 * asynchronous.  B is n x nrhs with leading dimension ldb, overwritten by X.
 */
int lu_solve_ex(lu_handle handle, lu_dtype dtype, int64_t n, int64_t nrhs, const void *LU,
                int64_t lda, const int32_t *ipiv, void *B, int64_t ldb);

/* ----------------------------------------------------------------------------
 * The individual steps of one iteration of LU_blk, exposed for testing and
 * for callers that build their own schedules.  All asynchronous on the
 * handle's stream; dtype selects FP64 or FP32.
 * ------------------------------------------------------------------------- */

/*
 * lu_panel_factor_ex -- RL1: [A11; A21] := LU_unb([A11; A21]) for an m x w
 * panel (m >= w), with partial pivoting over the panel's rows.
 *   A        device, top-left element of the panel, leading dimension lda
 *   ipiv     device int32[w]; ipiv[j] = 1-based row (relative to the panel's
 *            first row) interchanged with row j+1
 *   info     device int32[1]; set to j+1 for the first exactly zero pivot if
 *            it was 0, or to LU_ERR_TIMEOUT
 * The interchanges are applied across the panel's w columns only.
 */
int lu_panel_factor_ex(lu_handle handle, lu_dtype dtype, int64_t m, int64_t w, void *A,
                       int64_t lda, int32_t *ipiv, const lu_opts *opts, int32_t *info);

/*
 * lu_laswp_ex -- apply the interchanges ipiv[k1], ..., ipiv[k2-1] (1-based
 * row numbers of A, applied in that order: row k+1 <-> row ipiv[k]) to
 * columns 0 .. ncols-1 of A (the laswp of the getrf decomposition, Sec. 3.4).
 */
int lu_laswp_ex(lu_handle handle, lu_dtype dtype, int64_t ncols, void *A, int64_t lda,
                int64_t k1, int64_t k2, const int32_t *ipiv);

/*
 * lu_trsm_ex -- RL2: B := trilu(L)^{-1} B with L an m x m unit-lower matrix
 * (its diagonal and upper part are not read) and B m x n.
 */
int lu_trsm_ex(lu_handle handle, lu_dtype dtype, int64_t m, int64_t n, const void *L,
               int64_t ldl, void *B, int64_t ldb);

/*
 * lu_gemm_update_ex -- RL3: C := C - A B with A m x k, B k x n, C m x n, all
 * in the storage dtype, on the CUDA cores (FP64 or FP32 fused multiply-add).
 */
int lu_gemm_update_ex(lu_handle handle, lu_dtype dtype, int64_t m, int64_t n, int64_t k,
                      const void *A, int64_t lda, const void *B, int64_t ldb, void *C,
                      int64_t ldc);

/*
 * lu_gemm_update_tc_ex -- RL3, C := C - A B on the tensor cores: A (m x k) and
 * B (k x n) are FP32 and are rounded to the operand type of `prec` (round to
 * nearest even; LU_TU_BF16, LU_TU_FP16, LU_TU_BF16X3 or LU_TU_BF16X6; with LU_TU_FP8 each row of A and
 * each column of B is scaled by a power of two 2^e, e the smallest integer with max|block| / 2^e <= 448,
 * before rounding to e4m3), the products accumulate in FP32, the scales are applied to the FP32
 * accumulator, and C (FP32, m x n) is updated in place.  k must be a multiple of 64 (128 for FP8).
 *   info  device int32[1]; 0, or LU_ERR_TIMEOUT if a bounded wait expired.
 */
int lu_gemm_update_tc_ex(lu_handle handle, lu_prec prec, int64_t m, int64_t n, int64_t k, const float *A,
                         int64_t lda, const float *B, int64_t ldb, float *C, int64_t ldc, int32_t *info);

/*
 * lu_panel_factor_noalloc -- the panel factorization of lu_panel_factor_ex for
 * callers that cannot allocate device memory: code running where cudaMalloc
 * is unavailable or not allowed (a host callback, an allocator's own code
 * path, a latency-critical loop that preallocated everything, a process whose
 * device memory pool belongs to someone else).  The paper has no counterpart;
 * it is an interface convenience.
 *   dtype, m, w, A, lda, ipiv, opts, info   as in lu_panel_factor_ex
 *   stream   cudaStream_t (as void*, NULL = legacy default) the work is queued on
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call.  The
 * scratch it needs (synchronisation counters, the panel leaf's exchange slots
 * and one interchange plan) is a statically sized __device__ array inside the
 * library, lu_noalloc_scratch_bytes() bytes (about 155 KB), held by every GPU
 * that loads the library until the process exits.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress, with that device
 * current): make it before any stream capture.  Every call on a device shares
 * the array and finds the previous call's contents in it (the counters are
 * cleared at the start of each call), so calls that overlap on the GPU race:
 * serialise them.  Returns -i for an invalid argument, LU_ERR_UNSUPPORTED when
 * w > 1024 (the plan the array holds covers at most 1024 interchanges) or the
 * panel does not fit the leaf kernels, LU_ERR_CUDA, or 0 when enqueued.
 */
int lu_panel_factor_noalloc(lu_dtype dtype, int64_t m, int64_t w, void *A, int64_t lda, int32_t *ipiv,
                            const lu_opts *opts, int32_t *info, void *stream);
/* Size in bytes of the static scratch array used by lu_panel_factor_noalloc. */
size_t lu_noalloc_scratch_bytes(void);

/*
 * lu_peak_fma -- measurement utility, not a step of the method (the paper
 * measures on a multicore CPU and names no GPU peak): launches `blocks` CTAs of
 * `threads` threads (32..256, a multiple of 32), each thread running
 * lu_peak_fma_chains() independent fused multiply-add chains for `iters`
 * iterations in FP64 (dtype LU_F64) or FP32 (LU_F32), and writes one value per
 * thread to `sink` (device buffer of blocks * threads elements of that type,
 * caller-owned).  The work is 2 * chains * iters * blocks * threads flops; the
 * caller times the launch with CUDA events on `stream` and so obtains the
 * CUDA cores' FMA throughput, the denominator of the kernels that run there.
 * Asynchronous.  Returns -i for an invalid argument, LU_ERR_CUDA, or 0.
 */
int lu_peak_fma(lu_dtype dtype, int blocks, int threads, int64_t iters, void *sink, void *stream);
int lu_peak_fma_chains(void);

/*
 * lu_selftest_wait_timeout -- diagnostic of the failure path shared by every
 * kernel that synchronises CTAs through global memory: launches a grid barrier
 * that can never complete, whose bounded wait gives up after limit_ns
 * nanoseconds (1 .. 2e9) of device time; *status (device int32) receives
 * LU_ERR_TIMEOUT when the path works.  Asynchronous; leaves the device usable.
 */
int lu_selftest_wait_timeout(lu_handle handle, int64_t limit_ns, int32_t *status);

/* ----------------------------------------------------------------------------
 * Mixed precision (not in the paper, whose experiments are FP64 only): FP32
 * panels, triangular solves and factors, a tensor-core trailing update, and
 * FP64 iterative refinement of A x = b.
 * ------------------------------------------------------------------------- */

/*
 * lu_factor_mixed_ex -- blocked FP32 LU of an n x n FP32 matrix with the same
 * look-ahead schedule as lu_factor_ex, whose trailing update (RL3) runs on the
 * tensor cores with operands rounded to `prec` (LU_TU_BF16 / LU_TU_FP16) and
 * FP32 accumulation; LU_TU_F32 keeps it on the CUDA cores.  When nb is not a
 * multiple of 64 the update falls back to FP32 on the CUDA cores.  LU_TU_BF16X3
 * and LU_TU_BF16X6 run the same kernel on split operands with a 3x / 6x longer K.
 * Asynchronous; info as in lu_factor_ex.  The launch sequence depends only on
 * the arguments (pointers, sizes, options, handle stream): the second call with
 * the same arguments captures it as a CUDA graph and later ones replay it (the
 * data in those buffers may change freely between calls; while the launch
 * profiler is enabled every call runs the launches directly).
 */
int lu_factor_mixed_ex(lu_handle handle, lu_prec prec, int64_t n, float *A, int64_t lda, int32_t *ipiv,
                       const lu_opts *opts, int32_t *info);

/*
 * lu_gesv_mixed -- solve A X = B for an n x n FP64 matrix A and n x nrhs FP64
 * B: copy A to FP32, factor it with lu_factor_mixed_ex, solve in FP32 (with
 * prec = LU_FULL_F64: copy, factor and solve in FP64 instead), then
 * refine in FP64: r = B - A X with the original A, stop when the normwise
 * backward error eta = max_c ||r_c|| / (||A|| ||x_c|| + ||b_c||) (inf-norms)
 * is <= 0.9 tol (the margin covers the rounding of the FP64 residual itself),
 * or after max_iter corrections.
 *   A, B      device FP64, not modified
 *   X         device FP64 n x nrhs (ldx), receives the solution (the iterate
 *             with the smallest eta if tol was not reached)
 *   tol       stopping threshold (1e-14 in the experiments), >= 0
 *   max_iter  maximum number of corrections (30 in the experiments), >= 0
 *   opts      factorization options (NULL = defaults)
 *   iters     host; number of corrections applied to reach the returned X
 *   bwd_err   host; eta of the returned X
 * Synchronous (the host reads eta once per iteration).  Returns 0,
 * LU_WARN_NOT_CONVERGED, i > 0 if U(i,i) of the FP32 factors is exactly zero,
 * -i, or a runtime error code.
 */
int lu_gesv_mixed(lu_handle handle, lu_prec prec, int64_t n, int64_t nrhs, const double *A, int64_t lda,
                  const double *B, int64_t ldb, double *X, int64_t ldx, double tol, int max_iter,
                  const lu_opts *opts, int *iters, double *bwd_err);

/* ----------------------------------------------------------------------------
 * Batched (not in the paper): many independent small systems in one launch.
 * ------------------------------------------------------------------------- */

/*
 * lu_gesv_batched -- for each i < batch, P_i A_i = L_i U_i in place (LU_blk,
 * RL1-RL3, with 32-column panels) and, if B is not NULL, B_i := A_i^{-1} B_i.
 * One persistent launch: matrices are taken largest first from an atomic
 * counter by CTAs that each factor (and solve) one matrix at a time.
 *   dtype    LU_F64 or LU_F32 (all matrices the same type)
 *   n        device int32[batch], orders, 0 <= n_i <= 512
 *   A        device array of batch device pointers, column-major A_i
 *   lda      device int64[batch], lda_i >= max(1, n_i)
 *   ipiv     device array of batch device pointers to int32[n_i]
 *   nrhs     device int32[batch], 0 <= nrhs_i <= 8 (ignored when B is NULL)
 *   B        NULL, or device array of batch device pointers to n_i x nrhs_i
 *   ldb      device int64[batch] (ignored when B is NULL)
 *   info     device int32[batch]: 0; i > 0 = first exactly zero pivot (the
 *            system is then not solved); -4 bad lda_i; -9 bad ldb_i;
 *            LU_ERR_UNSUPPORTED for n_i or nrhs_i out of range
 * Asynchronous on the handle's stream; the launch can be captured in a CUDA
 * graph (its order/counter workspace is allocated on the first call).
 * Returns 0 (enqueued), -i for an invalid host argument, or a runtime error.
 */
int lu_gesv_batched(lu_handle handle, lu_dtype dtype, int batch, const int32_t *n, void *const *A,
                    const int64_t *lda, int32_t *const *ipiv, const int32_t *nrhs, void *const *B,
                    const int64_t *ldb, int32_t *info);
/* lu_factor_batched -- lu_gesv_batched without right-hand sides. */
int lu_factor_batched(lu_handle handle, lu_dtype dtype, int batch, const int32_t *n, void *const *A,
                      const int64_t *lda, int32_t *const *ipiv, int32_t *info);
/*
 * lu_solve_batched -- for each i < batch, B_i := (P_i^T L_i U_i)^{-1} B_i with
 * the factors and interchanges that lu_factor_batched (or lu_gesv_batched) left
 * in LU_i and ipiv_i (getrs: interchanges, unit-lower solve, upper solve).
 * Arguments as lu_gesv_batched; B must not be NULL (-9 otherwise).  The factors
 * are not checked for zero pivots: a singular U_i gives non-finite B_i, as in
 * getrs.  info_i: 0, or -4 / -9 / LU_ERR_UNSUPPORTED as above.
 */
int lu_solve_batched(lu_handle handle, lu_dtype dtype, int batch, const int32_t *n, void *const *LU,
                     const int64_t *lda, int32_t *const *ipiv, const int32_t *nrhs, void *const *B,
                     const int64_t *ldb, int32_t *info);

/*
 * lu_potrf_ex -- Cholesky factorization A = L L^T of a symmetric positive
 * definite n x n matrix on the same blocked right-looking skeleton with depth-1
 * look-ahead (Sec. 3-4; the paper names Cholesky among the factorizations that
 * fit it).  Elimination without interchanges gives A = L~ U with U = D L~^T for
 * such A; the call returns L = L~ D^{1/2}.
 *   h      handle (its stream orders the work; asynchronous)
 *   dtype  LU_F64 or LU_F32 (CUDA-core arithmetic)
 *   n      order, n >= 0
 *   A      device, n x n column-major with leading dimension lda, BOTH triangles
 *          holding the symmetric matrix.  On exit the lower triangle (diagonal
 *          included) holds L; the strict upper triangle is overwritten (it holds
 *          D L~^T).
 *   lda    >= max(1, n)
 *   opts   nb (0 = tuned, see lu_tune_nb), lookahead; NULL = defaults
 *   info   device int32 (out): 0, or j > 0 when the pivot of step j - 1 was not
 *          positive (the leading j x j minor is not positive definite; L is then
 *          not meaningful), or LU_ERR_TIMEOUT
 * Returns 0, -i for an invalid argument, or a runtime error code.
 */
int lu_potrf_ex(lu_handle h, lu_dtype dtype, int64_t n, void *A, int64_t lda, const lu_opts *opts, int32_t *info);

/*
 * Block-size autotuning.  Sec. 3 leaves the algorithmic block size b to the
 * implementation (the paper's experiments fix b = 192 for their processor).  On
 * the GPU, b trades the number of panel factorizations on the critical path of
 * the look-ahead schedule (Sec. 4) against the width of the trailing updates,
 * so the library measures it.  A process-wide table maps (device name,
 * factorization kind, ceil(log2 n)) to the nb of least measured time;
 * factorizations given nb = 0 take the table's value, else 256.  If the
 * environment variable LU_GB300_TUNE_FILE names a file, the first nb = 0 lookup
 * loads it (lu_tune_load).
 *
 * Factorization kinds: an lu_prec value other than LU_FULL_F64 (the mixed
 * factorization of lu_factor_mixed_ex / lu_gesv_mixed with that update), or
 * one of the two below.
 */
#define LU_TUNE_F64 100 /* FP64 factorization: lu_factor, lu_factor_ex(LU_F64), lu_gesv_mixed(LU_FULL_F64) */
#define LU_TUNE_F32 101 /* FP32 factorization on the CUDA cores: lu_factor_ex(LU_F32) */
/* The batched kernel (lu_gesv_batched and friends), FP64 / FP32: the table's value
 * for these kinds is the tile cut-over of the batched trailing update -- a panel
 * step whose trailing order is below it uses 32 x 32 output tiles, otherwise
 * 64 x 64 (1 = always 64 x 64) -- looked up with n = 512. */
#define LU_TUNE_BATCHED_F64 102
#define LU_TUNE_BATCHED_F32 103
/* Cut-overs used when none was tuned (measured on a GB300 with the 4096-system
 * batch of orders log-uniform in [16, 512]). */
#define LU_BATCHED_CUT_F64 193
#define LU_BATCHED_CUT_F32 97

/*
 * lu_tune_nb -- time the factorization of `kind` on a seeded synthetic n x n
 * matrix with iid U[-1,1) entries, for each candidate nb, and record the fastest.
 *   h           handle; its stream orders the runs, and the call synchronises it
 *   kind        factorization kind (above)
 *   n           order, 1 <= n <= 2^30
 *   candidates  host int[count], count >= 1: the nb values to try.  A value the
 *               factorization rejects (outside 1..1024, not a multiple of 128 for
 *               LU_TU_FP8, or too large for the memory) is skipped.
 *   reps        >= 1 runs per candidate; the least time counts (the first run
 *               of a mixed factorization is eager, the second captures its graph)
 *   opts        look-ahead, stealing, leaf and pf_ctas used for every run
 *               (NULL = defaults; its nb is ignored)
 *   best_nb     host int (out): the candidate of least time, also stored in the table
 *   ms          host float[count] or NULL (out): each candidate's least time in
 *               milliseconds, -1 for a skipped one
 * The scratch matrix (n*n elements of the kind's type) is allocated with
 * cudaMalloc and freed before returning.  Returns 0, -i for an invalid argument,
 * LU_ERR_NOMEM (scratch matrix), LU_ERR_UNSUPPORTED (no candidate ran) or a
 * runtime error of the factorization.
 */
int lu_tune_nb(lu_handle h, int kind, int64_t n, const int *candidates, int count, int reps, const lu_opts *opts,
               int *best_nb, float *ms);

/*
 * lu_tune_batched -- time the batched factorization + solve (lu_gesv_batched)
 * of `dtype` on a synthetic batch with the caller's sizes (host arrays n[batch],
 * orders 0..512, and nrhs[batch], 0..8; entries iid U[-1,1) from a fixed seed)
 * for each candidate tile cut-over cuts[count] (1..513, see
 * LU_TUNE_BATCHED_F64), and store the fastest in the table (n = 512).
 *   reps   >= 1 runs per candidate, the least time counts
 *   best   host int (out): the chosen cut-over
 *   ms     host float[count] or NULL (out): each candidate's least time
 * Every candidate computes the same factors (the tile shape changes no
 * operation).  Scratch matrices are allocated and freed inside.  Returns 0,
 * -i for an invalid argument, LU_ERR_NOMEM or a runtime error.
 */
int lu_tune_batched(lu_handle h, lu_dtype dtype, int batch, const int32_t *n, const int32_t *nrhs, int reps,
                    const int *cuts, int count, int *best, float *ms);

/* The table's nb for (device, kind, ceil(log2 n)), or 0 when there is none.
 * device: host string, or NULL for the current CUDA device's name. */
int lu_tune_get(const char *device, int kind, int64_t n);
/* Stores nb (and its time in ms, informative) for (device, kind, ceil(log2 n)),
 * replacing an entry with the same key (and any plan it held).  Returns 0, -1 (device NULL without a
 * CUDA device, empty, or holding a tab or newline), -2 (kind), -3 (n < 1), -4 (nb). */
int lu_tune_set(const char *device, int kind, int64_t n, int nb, float ms);
/* Empties the table.  Returns 0. */
int lu_tune_clear(void);
/* Writes the table to the host file `path` as text lines
 * "device<TAB>kind<TAB>ceil(log2 n)<TAB>nb<TAB>ms", followed for a tuned plan by
 * "<TAB>reserve<TAB>depth<TAB>schedule" (comma-separated block sizes, "-" for
 * none) and, when the plan has a leaf SM partition, "<TAB>pf_sms".  Returns 0,
 * -1 (NULL path) or LU_ERR_IO. */
int lu_tune_save(const char *path);
/* Merges the lines of such a file into the table (an entry replaces one with the
 * same key).  Every line is validated first; on any malformed line nothing is
 * merged.  Returns 0, -1 (NULL path) or LU_ERR_IO (unreadable or malformed). */
int lu_tune_load(const char *path);

/*
 * lu_potrf_mixed_ex -- Cholesky A = L L^T of a symmetric positive definite FP32
 * matrix (lu_potrf_ex's algorithm: elimination without interchanges on the
 * look-ahead skeleton, only the lower block triangle updated, then L = L~ D^{1/2})
 * with the trailing update A22 -= L21 U12 on the tensor cores in the operand
 * precision prec (LU_TU_BF16X6 keeps FP32-level accuracy; LU_TU_F32 = the CUDA
 * cores, as lu_potrf_ex).  The update takes only the tiles on or below the
 * diagonal panel blocks (n^3/3 flops).  Arguments, layout, info and return codes
 * as lu_potrf_ex; opts.nb must be a multiple of 64 for the tensor cores (other
 * steps fall back to the CUDA cores) and opts.rtm is rejected with
 * LU_ERR_UNSUPPORTED on the tensor-core path.
 */
int lu_potrf_mixed_ex(lu_handle handle, lu_prec prec, int64_t n, float *A, int64_t lda, const lu_opts *opts,
                      int32_t *info);

/*
 * lu_geqrf_ex -- Householder QR of an m x n matrix, A = Q R, on the blocked
 * look-ahead skeleton of Sec. 4 (the paper's second factorization, Sec. 6.3;
 * 4n^3/3 flops when m = n).  Per panel k: PF_k factors the panel column by
 * column (reflector H_j = I - tau_j v_j v_j^T mapping the updated column j onto
 * beta e_j with beta = -sign(a_jj) ||x||, tau_j = 0 when nothing lies below
 * the diagonal), then the compact-WY form Q_k = I - V_k T_k V_k^T; TU_k applies
 * Q_k^T to the columns on the right as C -= V_k (T_k^T (V_k^T C)).  With
 * look-ahead, TU_k on panel k+1 and PF_{k+1} overlap TU_k on the rest.
 *   dtype  LU_F64 or LU_F32; A (device, column-major, lda >= max(1, m)) is
 *          overwritten in LAPACK geqrf layout: R on and above the diagonal, v_j
 *          below it (v_j(j) = 1 implied)
 *   tau    device array of min(m, n) scalars of the same type (out)
 *   opts   nb 1..128 (0 or NULL: 128), lookahead 0 or 1, a schedule of widths
 *          <= 128; other fields ignored
 *   info   device int32 (out): 0, or LU_ERR_TIMEOUT if a bounded wait of the
 *          panel gave up
 * Workspace (the explicit V blocks, T factors, products, split-K partials)
 * belongs to the handle.  Asynchronous on the handle's stream.  Returns 0, -i
 * for an invalid argument, LU_ERR_UNSUPPORTED (nb > 128, depth 2, the task-DAG
 * schedule, or a panel too tall for one co-resident grid: m beyond ~50000 in
 * FP64), LU_ERR_NOMEM or LU_ERR_CUDA.
 */
int lu_geqrf_ex(lu_handle handle, lu_dtype dtype, int64_t m, int64_t n, void *A, int64_t lda, void *tau,
                const lu_opts *opts, int32_t *info);

/*
 * lu_geqrf_mixed_ex -- lu_geqrf_ex for an FP32 matrix with the last of the three
 * products of each update, C -= V_k (T_k^T V_k^T C), on the tensor cores in the
 * operand precision prec (LU_TU_BF16X6 keeps FP32-level accuracy; LU_TU_BF16,
 * LU_TU_FP16, LU_TU_BF16X3 trade accuracy; LU_TU_F32 = the CUDA cores, then the
 * same as lu_geqrf_ex).  V_k is packed once per panel, T_k^T V_k^T C per update;
 * steps whose width is not a multiple of 64 use the CUDA cores.  Arguments,
 * layout, info and return codes as lu_geqrf_ex (-2: prec is LU_TU_FP8 or not a
 * precision code).
 */
int lu_geqrf_mixed_ex(lu_handle handle, lu_prec prec, int64_t m, int64_t n, float *A, int64_t lda, float *tau,
                      const lu_opts *opts, int32_t *info);

/*
 * lu_tune_plan -- tune the whole schedule of the factorization of `kind` at
 * order n on a seeded synthetic matrix (iid U[-1,1)), in four measured stages:
 *   1. the block size b among 128, 192, 256, 320, 384, 512 (multiples of 64,
 *      of 128 for LU_TU_FP8, on the tensor-core kinds);
 *   2. with look-ahead, the SMs the right update leaves to the panel path
 *      (lu_opts.tu_reserve) among 1/12, 1/6, 1/4 and 1/3 of the SMs;
 *   3. with look-ahead, the depth 1 or 2, then an SM partition of 16, 24 or 32
 *      SMs for the panel leaves (lu_opts.pf_sms);
 *   4. a per-step schedule, the GPU form of the paper's early termination
 *      (Sec. 4.2: b adjusted on the fly when PU(k+1) and TU_right(k) are out of
 *      balance): the steps of the factorization at b/2, b and 2b are traced
 *      (lu_step_trace), and walking the columns, each step takes the width whose
 *      traced step at that position added the least critical-path time per
 *      eliminated column; the schedule is kept only if it beats the fixed plan.
 *   h         handle; its stream orders the runs, and the call synchronises it
 *   reps      >= 1 runs per candidate, the least time counts (use 3: a repeated
 *             mixed factorization is captured on its second run, replayed after)
 *   opts      look-ahead on/off, stealing, leaf and pf_ctas for every run (NULL =
 *             defaults); its nb, tu_reserve and schedule are ignored
 *   best      host (out): the chosen options; best->sched points into `sched`
 *   sched     host int32[cap] (out) for the schedule; a schedule longer than cap
 *             is not chosen
 *   best_ms   host float or NULL (out): the chosen plan's least time (ms)
 *   fixed_ms  host float or NULL (out): the best plan without a schedule (ms)
 * The plan is also stored in the table for (device, kind, ceil(log2 n)), where
 * calls with nb = 0 find it.  The scratch matrix is allocated and freed inside.
 * Returns 0, -i for an invalid argument, LU_ERR_NOMEM, LU_ERR_UNSUPPORTED (no
 * candidate ran) or a runtime error of the factorization.
 */
int lu_tune_plan(lu_handle h, int kind, int64_t n, int reps, const lu_opts *opts, lu_opts *best, int32_t *sched,
                 int cap, float *best_ms, float *fixed_ms);
/* Stores a plan for (device, kind, ceil(log2 n)): nb, reserve (0 = automatic),
 * depth (0 = the caller's), a schedule of nsched block sizes (host array, may
 * be NULL when nsched is 0), the leaf SM partition pf_sms (0 = none) and its
 * time.  Returns 0 or -i for the i-th argument (-7: a width outside 1..1024,
 * or not a multiple of 128 for FP8). */
int lu_tune_plan_set(const char *device, int kind, int64_t n, int nb, int reserve, int depth, const int32_t *sched,
                     int nsched, int pf_sms, float ms);
/* Reads the plan for (device, kind, ceil(log2 n)) into the non-NULL outputs
 * (at most cap schedule entries; *nsched receives the full length).  Returns 1
 * when an entry exists, else 0. */
int lu_tune_plan_get(const char *device, int kind, int64_t n, int *nb, int *reserve, int *depth, int32_t *sched,
                     int cap, int *nsched, int *pf_sms);

/*
 * lu_step_trace -- diagnostic of the look-ahead schedule (Sec. 4): with enable
 * != 0, later factorizations on this handle record CUDA events around every
 * step: on the panel stream from the start of PU(k+1) (TU_k on the next panel
 * and PF_{k+1}) to its end, and on the update stream around TU_right(k).  A
 * traced mixed factorization is not replayed as a graph.  Returns 0.
 * lu_step_trace_read synchronises with the last traced factorization and fills,
 * for its first min(cap, steps) steps, the panel's first column k0, its width
 * kb, span_ms (the time from the step's start to the later of PU(k+1)'s and
 * TU_right(k)'s ends: what the step adds to the critical path), pu_ms and
 * tu_ms (any output may be NULL).  Returns the number of steps, or < 0.
 */
int lu_step_trace(lu_handle h, int enable);
int64_t lu_step_trace_read(lu_handle h, int cap, int64_t *k0, int32_t *kb, float *span_ms, float *pu_ms,
                           float *tu_ms);

#ifdef __cplusplus
}
#endif

#endif /* LU_GB300_H */
