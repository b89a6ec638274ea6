/*
 * gbgemm -- single-precision GEMM for one NVIDIA GB300 GPU (sm_103a).
 *
 * The operation (Section III-A of Tasende, "Generation of the Single
 * Precision BLAS library for the Parallella platform ...", 2016, the problem
 * the BLIS-generated sgemm solves):
 *
 *     C_out = alpha * op(A) * op(B) + beta * C_in
 *
 * with A, B, C in column-major storage with leading dimensions, op(X) = X or
 * X^T, and M, N, K arbitrary.  Element by element, for 0 <= i < m, 0 <= j < n:
 *
 *     C[i + j*ldc] = alpha * sum_{p<k} opA(i,p) * opB(p,j) + beta * C[i + j*ldc]
 *     opA(i,p) = A[i + p*lda] (transa = 'N'/'n')  or  A[p + i*lda] ('T','t','C','c')
 *     opB(p,j) = B[p + j*ldb] (transb = 'N'/'n')  or  B[j + p*ldb] ('T','t','C','c')
 *
 * For real data the conjugate letters equal their plain ones: 'C' (conjugate
 * transpose, BLAS argument letter) behaves as 'T'.  Argument order and
 * conventions follow reference BLAS sgemm: beta == 0 never reads C (NaN in C
 * does not propagate); alpha == 0 or k == 0 never reads A or B; m == 0 or
 * n == 0, or (alpha == 0 or k == 0) with beta == 1, returns without work.
 * Entries of C outside rows 0..m-1 of each column are never written.
 *
 * Two paths compute the same result within the componentwise bound
 *     |C - C_exact|_ij <= 2 * max(k,1) * 2^-24 * (|alpha| sum_p |opA(i,p)||opB(p,j)| + |beta| |C_in,ij|)
 *   GBGEMM_PATH_SIMT        plain FP32 fused multiply-add on the CUDA cores.
 *   GBGEMM_PATH_SPLIT_BF16  each badly scaled operand row (of op(A)) or
 *                           column (of op(B)) -- largest magnitude outside
 *                           [2^-48, 2^48) -- is scaled by a power of two so
 *                           its largest entry lies in [0.5, 1).  For
 *                           k >= 512 every entry x becomes hi + lo (two
 *                           BF16 values, hi = bf16(x), lo = bf16(x - hi))
 *                           and the tensor cores accumulate hi*hi + hi*lo +
 *                           lo*hi in FP32; for k < 512 it becomes hi + mid +
 *                           lo3 (lo3 = bf16(x - hi - mid), the sum is exact)
 *                           and six products are accumulated (hi*hi, hi*mid,
 *                           mid*hi, hi*lo3, mid*mid, lo3*hi).  Either way
 *                           the bound holds for every k.
 *   GBGEMM_PATH_AUTO        SPLIT_BF16 when k >= 128, else SIMT.
 *
 * Memory and streams.  All matrix pointers are DEVICE pointers owned by the
 * caller, who keeps them alive until the work queued on the handle's stream
 * has completed.  Calls are asynchronous on that stream: no call in this
 * header synchronises the host except where stated.  The handle owns a
 * device workspace (split panels and row maxima) that grows on demand with
 * cudaMalloc; gbgemm_reserve_workspace() pre-sizes it so that later calls do
 * not allocate.
 *
 * Errors.  Every call returns GBGEMM_OK (0) or a negative status.  Argument
 * errors of gbgemm_sgemm return minus the 1-based position of the argument
 * in the BLAS argument list (transa = 1 ... ldc = 13), checked in that order
 * (see gbgemm_sgemm).  No call aborts the process.  Device-side failures (a
 * bounded wait that ran out) are recorded in a device status word read by
 * gbgemm_get_device_status().
 */
#ifndef GBGEMM_H
#define GBGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GBGEMM_OK = 0,
  GBGEMM_ERR_NOT_INITIALIZED = -100,  /* null handle or plan */
  GBGEMM_ERR_ALLOC = -101,            /* device or host allocation failed */
  GBGEMM_ERR_CUDA = -102,             /* a CUDA runtime call failed */
  GBGEMM_ERR_UNSUPPORTED_DEVICE = -103, /* split path requested on a device that is not sm_103 */
  GBGEMM_ERR_DEVICE_TIMEOUT = -104,   /* a kernel's bounded wait ran out (see gbgemm_get_device_status) */
  GBGEMM_ERR_BAD_PLAN = -105,         /* plan inputs invalid (bad problem index in *bad_index) */
  GBGEMM_ERR_INVALID_VALUE = -106,    /* other invalid argument (path code, size, pointer) */
  GBGEMM_ERR_SCRATCH_LIMIT = -107     /* problem needs more than GBGEMM_NOALLOC_SCRATCH_BYTES */
} gbgemm_status;

typedef enum {
  GBGEMM_PATH_AUTO = 0,
  GBGEMM_PATH_SIMT = 1,
  GBGEMM_PATH_SPLIT_BF16 = 2
} gbgemm_path;

typedef struct gbgemm_handle gbgemm_handle;

/* Create a handle bound to CUDA device `device` (made current for the call).
 * The handle starts on the legacy default stream (NULL) with path AUTO.
 * Errors: GBGEMM_ERR_INVALID_VALUE (h NULL), GBGEMM_ERR_CUDA (bad device),
 * GBGEMM_ERR_ALLOC. */
int gbgemm_create(gbgemm_handle** h, int device);

/* Destroy a handle and free its workspace.  Synchronises the handle's stream
 * first.  A NULL handle returns GBGEMM_ERR_NOT_INITIALIZED. */
int gbgemm_destroy(gbgemm_handle* h);

/* Set the cudaStream_t (passed as void*) that later calls queue work on. */
int gbgemm_set_stream(gbgemm_handle* h, void* cuda_stream);

/* Force a path (gbgemm_path).  SPLIT_BF16 forced with 16 <= k < 128 holds the
 * error bound (AUTO leaves those sizes to SIMT only because they are faster
 * there); with k < 16 it still runs but the bound is then not guaranteed.
 * Bad code: GBGEMM_ERR_INVALID_VALUE. */
int gbgemm_set_path(gbgemm_handle* h, int path);

/* Path taken by the handle's most recent gbgemm_sgemm (0 when it returned
 * early without launching the product kernels). */
int gbgemm_last_path(gbgemm_handle* h, int* path);

/* Grow the workspace to at least `bytes` now (cudaMalloc; synchronous). */
int gbgemm_reserve_workspace(gbgemm_handle* h, size_t bytes);

/* Workspace bytes the split path needs for one (m, n, k) problem without
 * k slicing: 256 bytes of control words, one counter per 128-row band of
 * op(A) and op(B), the row maxima, and the BF16 panels (twice the panels
 * when k < 512). */
size_t gbgemm_split_workspace_bytes(int64_t m, int64_t n, int64_t k);

/* BLAS-convention sgemm (Section III-A problem statement).
 * transa, transb: 'N','n','T','t','C','c'.  m, n, k >= 0.
 * A: device, stored (transa N ? m x k : k x m) with lda >= max(1, rows).
 * B: device, stored (transb N ? k x n : n x k) with ldb >= max(1, rows).
 * C: device, m x n with ldc >= max(1, m); read only when beta != 0.
 * Argument errors, in this order: transa -1, transb -2, m -3, n -4, k -5,
 * lda -8, ldb -10, ldc -13; then null A (when read) -7, null B -9,
 * null C (m*n > 0) -12.  Then GBGEMM_ERR_NOT_INITIALIZED for a NULL handle.
 * Queues kernels on the handle's stream and returns without waiting. */
int gbgemm_sgemm(gbgemm_handle* h, char transa, char transb, int64_t m, int64_t n, int64_t k,
                 float alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                 float beta, float* C, int64_t ldc);

/* Strided batch of `batch` equal sgemms: problem z (0 <= z < batch) is
 *   C_z := alpha op(A_z) op(B_z) + beta C_z,
 *   A_z = A + z*stride_a, B_z = B + z*stride_b, C_z = C + z*stride_c (elements),
 * each as in gbgemm_sgemm.  The paper's micro-kernel is exactly such a series
 * of fixed-size problems fed by BLIS (Section III-A, III-C); the paper itself
 * has no batched call.  stride_a or stride_b 0 shares one operand among all
 * problems; the results must not overlap (stride_c >= ldc (n - 1) + m when
 * batch > 1).  One packing launch (both operands of every problem) and one
 * persistent GEMM launch serve the whole batch (split path), or one SIMT
 * launch.  The workspace
 * holds about batch x gbgemm_split_workspace_bytes(m, n, k) bytes on the
 * split path.
 * Argument errors, in this order: transa -1, transb -2, m -3, n -4, k -5,
 * lda -8, stride_a -9, ldb -11, stride_b -12, ldc -15, stride_c -16,
 * batch (< 0 or > 65535) -17; then null A (when read) -7, null B -10,
 * null C -14.  Then GBGEMM_ERR_NOT_INITIALIZED for a NULL handle.  batch 0
 * returns at once.  Queues kernels on the handle's stream. */
int gbgemm_sgemm_strided_batched(gbgemm_handle* h, char transa, char transb, int64_t m, int64_t n, int64_t k,
                                 float alpha, const float* A, int64_t lda, int64_t stride_a, const float* B,
                                 int64_t ldb, int64_t stride_b, float beta, float* C, int64_t ldc, int64_t stride_c,
                                 int64_t batch);

/* BLAS-convention sgemv, y := alpha op(A) x + beta y.  The paper's HPL run is
 * limited by Level-2 BLAS on the host (Sections IV-C, V); this is the GPU
 * counterpart, memory-bound (every element of A read once).
 * trans: 'N','n' (op(A) = A, x of length n, y of length m) or 'T','t','C','c'
 * (op(A) = A^T, x of length m, y of length n).  A: device, m x n, lda >=
 * max(1, m).  x, y: device vectors with increments incx, incy != 0 (negative:
 * the vector runs backwards from the end of its storage, as in BLAS).  y is
 * read only when beta != 0.  Sums are formed in a fixed order (run-to-run
 * deterministic); the summed dimension is cut into slices when the other one
 * gives too few blocks, the slices' partial sums (in the handle's workspace)
 * added in order.
 * Argument errors, in this order: trans -1, m -2, n -3, lda -6, incx -8,
 * incy -11; then null A (when read) -5, null x -7, null y (len(y) > 0) -10.
 * Then GBGEMM_ERR_NOT_INITIALIZED for a NULL handle.  Queues kernels on the
 * handle's stream. */
int gbgemm_sgemv(gbgemm_handle* h, char trans, int64_t m, int64_t n, float alpha, const float* A, int64_t lda,
                 const float* x, int64_t incx, float beta, float* y, int64_t incy);

/* LU factorisation with partial pivoting, P A = L U, in FP32 (LAPACK sgetrf
 * for a square matrix): the factorisation the paper's HPL run performs
 * (Section IV-C, Table VII), right-looking and blocked by nb columns, with
 * every trailing update A22 := A22 - L21 U12 done by this library's sgemm
 * (the Linpack-shaped C := C - A B).
 * A: device, n x n column-major, lda >= max(1, n), overwritten by the packed
 * factors (L strictly below the diagonal with a unit diagonal implied, U on
 * and above).  ipiv: device, n ints; ipiv[j] (1-based) is the row exchanged
 * with row j at step j.  The pivot of column j is the row of largest |a_ij|
 * on or below the diagonal, the first such row on ties.  info: device, one
 * int, set to 0, then to j + 1 for the first exactly zero pivot U(j, j) (the
 * factorisation still completes, as in LAPACK).  nb: block width, 1 ..
 * GBGEMM_SGETRF_MAX_NB, or 0 for GBGEMM_SGETRF_DEFAULT_NB below n =
 * GBGEMM_SGETRF_WIDE_N and GBGEMM_SGETRF_MAX_NB from there (the faster of the
 * two measured at N 4608, 8192 and 16384 on GB300).  Each block of nb
 * columns is factored as panels of at most 32 columns (narrower when the
 * panel's rows outgrow the shared memory of a cluster of 16 thread blocks,
 * which holds a panel for its whole factorisation), the exchanges and
 * triangular solves of each panel applied across the block and the block
 * columns updated with k = the panel width; after the block, the whole
 * trailing matrix is updated with k = nb.  The next block is factored on a
 * second stream of the handle while the trailing matrix is updated (the two
 * touch disjoint columns; the handle's stream waits for it).  Columns are
 * scaled by the pivot's reciprocal, as LAPACK's unblocked factorisation and
 * HPL do, so |l_ij| <= 1 holds up to one rounding.
 * Results are bit-identical from run to run.  Queues kernels on the
 * handle's stream (and its look-ahead stream, joined back to it) and returns
 * without synchronising; the per-call tuner is not used for the trailing
 * updates.
 * Argument errors, in this order: n (< 0 or > INT_MAX) -1, null A (n > 0) -2,
 * lda -3, null ipiv (n > 0) -4, null info -5, nb -6.  Then
 * GBGEMM_ERR_NOT_INITIALIZED for a NULL handle, GBGEMM_ERR_ALLOC,
 * GBGEMM_ERR_CUDA, or an error of the trailing sgemm. */
#define GBGEMM_SGETRF_MAX_NB 128
#define GBGEMM_SGETRF_DEFAULT_NB 32
#define GBGEMM_SGETRF_WIDE_N 12288
int gbgemm_sgetrf(gbgemm_handle* h, int64_t n, float* A, int64_t lda, int* ipiv, int* info, int nb);

/* Solve A X = B with the factors of gbgemm_sgetrf (LAPACK sgetrs, no
 * transpose): the row exchanges of ipiv in order, then forward substitution
 * with unit L, then back substitution with U.  LU, ipiv: device, as
 * gbgemm_sgetrf left them.  B: device, n x nrhs column-major, ldb >=
 * max(1, n), overwritten by X.  The solves go by diagonal blocks of 256 rows.
 * With one right-hand side each substitution is one cooperative launch: a
 * block of rows is solved by one CTA as soon as the blocks before it are
 * (flags in the handle's workspace; a wait that runs out after 2 s sets the
 * device status, see gbgemm_get_device_status).  With several, one thread
 * block per right-hand side solves each diagonal block, and the off-diagonal
 * parts go through this library's sgemm.
 * Argument errors, in this order: n (< 0 or > INT_MAX) -1, nrhs (< 0 or >
 * INT_MAX) -2, null LU (n > 0) -3, lda -4, null ipiv (n > 0) -5, null B
 * (n, nrhs > 0) -6, ldb -7.  Then GBGEMM_ERR_NOT_INITIALIZED for a NULL
 * handle, GBGEMM_ERR_CUDA, GBGEMM_ERR_ALLOC.  Queues kernels on the handle's
 * stream. */
int gbgemm_sgetrs(gbgemm_handle* h, int64_t n, int64_t nrhs, const float* LU, int64_t lda, const int* ipiv, float* B,
                  int64_t ldb);

/* Synchronise the handle's stream, then read and clear the device status
 * word: *status = 0 when no kernel reported a failure since the last read,
 * else the first failing kernel's code (GBGEMM_ERR_DEVICE_TIMEOUT).  Returns
 * GBGEMM_ERR_CUDA if the stream reported a CUDA error. */
int gbgemm_get_device_status(gbgemm_handle* h, int* status);

/* Failure-detection check (tests).  Queues on the handle's stream one thread
 * that waits, with the same bounded mbarrier wait every kernel of this
 * library uses, on a barrier that nothing arrives on and no copy is bound
 * to; after timeout_ns (1 ns .. GBGEMM_DEBUG_MAX_WAIT_NS) the wait gives up,
 * GBGEMM_ERR_DEVICE_TIMEOUT is recorded in the device status word (read it
 * with gbgemm_get_device_status) and the kernel returns normally: the CUDA
 * context stays usable.  The paper has no counterpart (its co-processor
 * runs without such checks).  Errors: GBGEMM_ERR_INVALID_VALUE for a
 * timeout out of range, GBGEMM_ERR_CUDA if the launch fails. */
#define GBGEMM_DEBUG_MAX_WAIT_NS 100000000ull
int gbgemm_debug_expire_wait(gbgemm_handle* h, uint64_t timeout_ns);

/* Profiling (benchmark use).  Between begin and end the handle records a
 * pair of CUDA events on its stream around every launch of the split-path
 * GEMM kernel, and counts every kernel the library launches.  While it
 * profiles, the GEMM is launched after the packing completes (not as a
 * programmatic dependent that may start early), so each pair brackets the
 * GEMM kernel alone.
 * gbgemm_profile_end synchronises the stream and returns the summed GEMM
 * kernel time in milliseconds, the number of GEMM launches and the number
 * of kernels launched by the library (memsets not included).  Any output
 * pointer may be NULL. */
int gbgemm_profile_begin(gbgemm_handle* h);
int gbgemm_profile_end(gbgemm_handle* h, double* gemm_ms, int64_t* gemm_launches, int64_t* kernel_launches);

/* FP64 error check on the GPU (tests and benchmarks; the sgemm paths never
 * use FP64).  For the block rows [i0, i1) x columns [j0, j1) of an m x n
 * result it recomputes C64 = alpha * sum_p opA(i,p) opB(p,j) + beta * C_in
 * (Section III-A) with FP64 products and sums in p order, and the
 * acceptance bound
 *   bound_ij = 2 max(k,1) 2^-24 (|alpha| sum_p |opA(i,p)||opB(p,j)| + |beta||C_in,ij|),
 * then returns *max_ratio = max |C_out,ij - C64_ij| / bound_ij (+inf when a
 * zero bound is exceeded or a difference is NaN).  C_in is the C the sgemm
 * started from (caller keeps a copy), C_out its result; both use ldc.  All
 * matrix pointers are device pointers.  Synchronises the handle's stream. */
int gbgemm_check_error(gbgemm_handle* h, char transa, char transb, int64_t m, int64_t n, int64_t k, float alpha,
                       const float* A, int64_t lda, const float* B, int64_t ldb, float beta, const float* C_in,
                       const float* C_out, int64_t ldc, int64_t i0, int64_t i1, int64_t j0, int64_t j1,
                       double* max_ratio);

/* Human-readable name of a status code (static string, never NULL). */
const char* gbgemm_status_string(int status);

/* ---------------------------------------------------------------------- */
/* Grouped sgemm: many independent problems, one captured CUDA graph.
 *
 * The BLIS driver of Section III-A divides one sgemm into small predefined
 * multiplications for its micro-kernel; the grouped call applies the same
 * division across problems: every problem is cut into tiles, the tiles of
 * all problems form one work list per kernel, and persistent thread blocks
 * drain it.  Each problem has the arguments of gbgemm_sgemm and its own
 * configuration (path and tile shape):
 *
 *   GBGEMM_CFG_SIMT_128x128, _64x64, _128x64   FP32 SIMT path, CTA tile shape
 *   GBGEMM_CFG_SPLIT_BN64, _BN128, _BN256      split-BF16 tensor path, 128 x BN
 *                                              tiles (needs k >= 16, alpha != 0:
 *                                              below k = 16 the three-part split
 *                                              can miss the error bound)
 *
 * Plan creation checks every problem (in problem order; *bad_index = the
 * first bad problem and the return value is GBGEMM_ERR_BAD_PLAN), chooses the
 * configurations, allocates the plan's device memory (hi/lo panels, row
 * maxima, descriptors, work lists) and captures the graph on a private
 * stream; it synchronises the device.  Running the plan is one
 * cudaGraphLaunch on the caller's stream and allocates nothing.
 *
 * Ownership: the plan captures the A, B, C pointers given at creation; to
 * run again on new data, write it into the same buffers.  The problems'
 * buffers and the handle must outlive the plan.  Problems must not write
 * overlapping parts of C (undefined otherwise).  Problems with m or n = 0,
 * or with (alpha = 0 or k = 0) and beta = 1, are skipped; (alpha = 0 or
 * k = 0) with another beta scales C on the SIMT path. */
typedef struct {
  char transa, transb;
  int64_t m, n, k;
  float alpha, beta;
  const float* A; int64_t lda;
  const float* B; int64_t ldb;
  float* C; int64_t ldc;
} gbgemm_problem;

typedef enum {
  GBGEMM_CFG_SIMT_128x128 = 0,
  GBGEMM_CFG_SIMT_64x64 = 1,
  GBGEMM_CFG_SIMT_128x64 = 2,
  GBGEMM_CFG_SPLIT_BN64 = 3,
  GBGEMM_CFG_SPLIT_BN128 = 4,
  GBGEMM_CFG_SPLIT_BN256 = 5,
  GBGEMM_NUM_CONFIGS = 6
} gbgemm_config;

/* Every source keeps the default rule's path for a problem (split from
 * k = 16 with alpha != 0, SIMT otherwise); the tuner and the predictor choose
 * the tile shape within that path.  A grouped plan runs many problems in one
 * launch, so the launch overhead that keeps the single call on SIMT below
 * k = 128 does not apply. */
typedef enum {
  GBGEMM_CONFIG_PREDICTED = 0,  /* learned predictor, tuner as fallback */
  GBGEMM_CONFIG_TUNED = 1,      /* exhaustive autotuner (timed on the GPU) */
  GBGEMM_CONFIG_DEFAULT = 2     /* fixed heuristic, no timing */
} gbgemm_config_source;

typedef struct gbgemm_grouped_plan gbgemm_grouped_plan;

/* probs: host array of `count` problems (device matrix pointers).
 * config_source: a gbgemm_config_source.  On success *plan owns the plan. */
int gbgemm_grouped_plan_create(gbgemm_handle* h, const gbgemm_problem* probs, int64_t count, int config_source,
                               gbgemm_grouped_plan** plan, int64_t* bad_index);
/* As gbgemm_grouped_plan_create with the configuration of every problem
 * given (host array of `count` gbgemm_config values).  An illegal
 * configuration for its problem is a bad problem. */
int gbgemm_grouped_plan_create_with_configs(gbgemm_handle* h, const gbgemm_problem* probs, int64_t count,
                                            const int* configs, gbgemm_grouped_plan** plan, int64_t* bad_index);
/* One cudaGraphLaunch on cuda_stream (a cudaStream_t; NULL = legacy default). */
int gbgemm_grouped_plan_run(gbgemm_grouped_plan* plan, void* cuda_stream);
/* Copy the configuration chosen for every problem (count ints; -1 for a
 * skipped problem) into configs (host). */
int gbgemm_grouped_plan_configs(const gbgemm_grouped_plan* plan, int* configs);
/* Plan statistics (host outputs, any may be NULL): problems on the split and
 * SIMT paths, their FLOPs (2mnk), kernels per run, device bytes held. */
int gbgemm_grouped_plan_stats(const gbgemm_grouped_plan* plan, int64_t* n_split, int64_t* n_simt, double* flops_split,
                              double* flops_simt, int* kernels_per_run, size_t* device_bytes);
/* Free the plan (synchronises the device first). */
int gbgemm_grouped_plan_destroy(gbgemm_grouped_plan* plan);
/* ---------------------------------------------------------------------- */
/* Autotuner.  The paper fixes its micro-kernel sizes at compile time
 * (Sections III-C, III-D); here every legal configuration (gbgemm_config) of
 * a problem shape is timed on the GPU -- CUDA events, one warm-up, the median
 * of `reps` runs -- on scratch buffers owned by the handle (same leading
 * dimensions and 16-byte alignment as the problem; the problem's own data is
 * never touched), and the result is cached in the handle under the key
 * (m, n, k, transposes, alignment classes of A, B, C).
 *
 * Two figures per configuration (microseconds, -1 when illegal):
 *   latency  one call on that problem alone;
 *   cost     GPU time per problem inside a grouped batch: a grouped plan of
 *            R copies of the problem (enough to fill every SM twice, at most
 *            256) is replayed and cost = replay time / R.  Used to rank
 *            configurations for grouped plans.
 * gbgemm_autotune synchronises the handle's stream; it must not run during
 * stream capture.  Any output pointer may be NULL. */
int gbgemm_autotune(gbgemm_handle* h, const gbgemm_problem* prob, int reps, float* latency_us, float* cost_us,
                    int* best_by_latency, int* best_by_cost);
/* Cache persistence: a text file, one line per shape key. */
int gbgemm_tuning_save(gbgemm_handle* h, const char* path);
int gbgemm_tuning_load(gbgemm_handle* h, const char* path);
int gbgemm_tuning_clear(gbgemm_handle* h);
/* ---------------------------------------------------------------------- */
/* Schedules of a single call.  The paper fixes the division of one sgemm
 * into micro-kernel work and the order of that work by hand (Sections
 * III-A, III-C: the ir / or ratios, KSUB, the Task / Column / K loops); here
 * a schedule fixes, for one gbgemm_sgemm call, the path, the tile, the order
 * of the tiles and the division of k:
 *   s = 0, 1, 2          SIMT path, CTA tile 128x128, 64x64, 128x64;
 *   s = 3 + 12 b + 4 r + q   split-BF16 path, tile 128 x BN with BN = 64 << b
 *                        (b = 0, 1, 2), tiles visited in groups of R tile
 *                        rows (all tile columns of a group before the next
 *                        group) with R = 1, 4, 16 for r = 0, 1, 2, and k-slicing
 *                        level q = 0..3: the k range cut into S = 1, F/4,
 *                        F/2 or F slices (split-K: the slices' raw
 *                        accumulators summed in slice order by a reduction),
 *                        where F is the slice count that gives about one
 *                        work item per SM (at most 32 slices of at least 4 k
 *                        chunks of 32; F = 1 when the output has more than
 *                        half as many 128 x BN tiles as the GPU has SMs, or
 *                        k < 512), S rounded down so that no slice is empty.
 * 39 schedules; the tile shapes are those of gbgemm_config.  Legal: SIMT
 * schedules always; split schedules when k >= 16 and alpha != 0 (the error
 * bound, as for the grouped configurations); q > 0 when its S is at least 2
 * and differs from level q - 1's.  The fixed heuristic's split-K (one
 * problem, long k, few tiles) is level 3 with BN 256. */
#define GBGEMM_NUM_SCHEDULES 39
/* Decode schedule s (host only, no GPU): path (gbgemm_path value), tile
 * rows and columns, R and the k-slicing level q as above (1 and 0 for SIMT).
 * Bad s: GBGEMM_ERR_INVALID_VALUE.  Any output pointer may be NULL. */
int gbgemm_schedule_info(int s, int* path, int* tile_m, int* tile_n, int* raster, int* kslice_level);
/* Whether schedule s may run problem prob on this handle's GPU (*legal = 0 or 1). */
int gbgemm_schedule_legal(gbgemm_handle* h, const gbgemm_problem* prob, int s, int* legal);
/* The schedule the fixed heuristic (tuning mode 0, path AUTO) gives prob. */
int gbgemm_schedule_default(gbgemm_handle* h, const gbgemm_problem* prob, int* s);
/* Time every legal schedule of prob's shape as one call (latency, CUDA
 * events, one warm-up, median of `reps`; -1 when illegal) on the tuner's
 * scratch buffers; cached in the handle like gbgemm_autotune's results.
 * *best = the lowest latency (ties to the lower index).  Synchronises the
 * handle's stream.  latency_us: host array of GBGEMM_NUM_SCHEDULES, or NULL. */
int gbgemm_autotune_schedules(gbgemm_handle* h, const gbgemm_problem* prob, int reps, float* latency_us, int* best);
/* Schedule of the handle's most recent gbgemm_sgemm that launched the product
 * kernels (-1 before the first). */
int gbgemm_last_schedule(gbgemm_handle* h, int* s);
/* Pin schedule s for the handle's later single calls (s = -1 unpins).  A
 * pinned schedule overrides the tuning mode for every call it is legal for
 * (gbgemm_schedule_legal, and on the handle's path unless that is AUTO);
 * other calls choose as the tuning mode says.  Bad s: GBGEMM_ERR_INVALID_VALUE. */
int gbgemm_set_schedule(gbgemm_handle* h, int s);

/* How gbgemm_sgemm (one problem) chooses its schedule:
 *   mode 0 (default): the fixed heuristic;
 *   mode 1: the schedule tuner's lowest latency among the legal schedules of
 *           the handle's path (tuning a new shape on first use, which
 *           synchronises; do it before any stream capture);
 *   mode 2: the learned schedule predictor (gbgemm_predictor_select(h, 1)),
 *           among the legal schedules of the handle's path; mode 1 when the
 *           predictor has no parameters or a dimension lies outside
 *           [8, 16384].
 * Strided batches (batch > 1) always use the fixed heuristic. */
int gbgemm_set_tuning(gbgemm_handle* h, int mode);

/* ---------------------------------------------------------------------- */
/* Learned configuration predictor: a 3-layer MLP (8 -> 64 -> 64 -> 6, ReLU,
 * FP32) trained on the autotuner's timings, so that grouped plans can choose
 * configurations without timing every problem (GBGEMM_CONFIG_PREDICTED).  The
 * paper picks its micro-kernel parameters by hand (Section III-C).
 *
 * Inputs (gbgemm_predictor_features): log2(m)/14, log2(n)/14, log2(k)/14,
 * transa, transb (0 = N, 1 = T), and the 16-byte alignment class of A, B, C
 * (1 when ld % 4 == 0 and the pointer is 16-byte aligned).  Outputs: the
 * predicted log2(cost_c / cost_best) of each gbgemm_config c.  Parameters,
 * one FP32 array of GBGEMM_MLP_PARAMS: W1[64][8], b1[64], W2[64][64], b2[64],
 * W3[6][64], b3[6] (row = output unit).  Loss: mean over samples and legal
 * configurations of (output - target)^2.
 *
 * x, y, mask, legal, scores, configs, grad below are DEVICE arrays:
 *   x[n][8] features, y[n][6] targets, mask[n][6] (1 legal / 0 illegal),
 *   legal[n] bit c set when configuration c may be chosen.
 * Grouped plans predict only for shapes inside the training range (every
 * dimension in [8, 16384]); other shapes, or a handle without parameters,
 * use the tuner. */
#define GBGEMM_MLP_PARAMS 5126
/* The schedule predictor: the same network with GBGEMM_NUM_SCHEDULES outputs
 * (predicted log2(latency_s / latency_best) of every schedule s), trained on
 * gbgemm_autotune_schedules latencies; W3[39][64], b3[39]. */
#define GBGEMM_SCHED_MLP_PARAMS 7271
/* Select the network that the gbgemm_predictor_* calls below address:
 * which = 0, the configuration predictor (GBGEMM_NUM_CONFIGS outputs,
 * GBGEMM_MLP_PARAMS parameters, grouped plans); which = 1, the schedule
 * predictor (GBGEMM_NUM_SCHEDULES outputs, GBGEMM_SCHED_MLP_PARAMS
 * parameters, tuning mode 2).  A new handle addresses network 0.  Where the
 * descriptions below say 6 outputs or GBGEMM_MLP_PARAMS, read the selected
 * network's outputs and parameter count; legal then holds (outputs + 7) / 8
 * bytes per sample, bit c % 8 of byte c / 8 for output c. */
int gbgemm_predictor_select(gbgemm_handle* h, int which);
int gbgemm_predictor_set(gbgemm_handle* h, const float* params /* host */);
int gbgemm_predictor_get(gbgemm_handle* h, float* params /* host */);
int gbgemm_predictor_features(const gbgemm_problem* prob, float* x /* host, 8 floats */);
/* Batched inference on the handle's stream: scores (n x 6, may be NULL) and
 * the lowest-scoring legal configuration per sample (-1 if none). */
int gbgemm_predictor_predict(gbgemm_handle* h, const float* x, const uint8_t* legal, int64_t n, float* scores,
                             int* configs);
/* Loss and gradient of the mean loss (GBGEMM_MLP_PARAMS floats into grad)
 * for n <= 256 samples; synchronises. */
int gbgemm_predictor_loss_grad(gbgemm_handle* h, const float* x, const float* y, const float* mask, int64_t n,
                               float* loss /* host */, float* grad);
/* Train the handle's predictor with Adam (beta1 0.9, beta2 0.999, eps 1e-8)
 * on mini-batches of `batch` <= 256 samples, reshuffled every epoch from
 * `seed`; starts from He-uniform weights when none are set.  *final_loss
 * (host, may be NULL) = loss of the final parameters on all n samples.
 * Synchronises. */
int gbgemm_predictor_train(gbgemm_handle* h, const float* x, const float* y, const float* mask, int64_t n, int epochs,
                           int batch, float lr, uint64_t seed, float* final_loss);

/* ---------------------------------------------------------------------- */
/* Allocation-free split-BF16 sgemm.  (The paper has no counterpart: its
 * service process owns all buffers.  This entry point exists for users of
 * this library.)
 *
 * For callers that cannot call cudaMalloc at the time they multiply: code
 * running inside someone else's stream capture (allocation is not a
 * capturable operation), allocator or memory-pool callbacks that must not
 * re-enter the allocator, latency-bound loops that cannot afford the device
 * synchronisation cudaMalloc/cudaFree imply, or processes whose device memory
 * another framework has reserved.  It computes the same thing as
 * gbgemm_sgemm on GBGEMM_PATH_SPLIT_BF16, with the same argument checks and
 * quick returns (arguments 1-13 are the BLAS ones, same error codes), but
 * needs no handle and allocates nothing: its scratch (hi/lo panels, row
 * maxima, a status word) is a fixed array of GBGEMM_NOALLOC_SCRATCH_BYTES in
 * this library's device memory, which every GPU that loads the library
 * holds until the process exits.
 *
 * Limits and behaviour:
 *   - a problem whose gbgemm_split_workspace_bytes(m, n, k) + 256 exceeds
 *     GBGEMM_NOALLOC_SCRATCH_BYTES returns GBGEMM_ERR_SCRATCH_LIMIT without
 *     launching anything (64 MiB holds m = n = k = 2048, for example);
 *   - runs on the CURRENT device and on `cuda_stream` (a cudaStream_t, NULL =
 *     legacy default stream), asynchronously;
 *   - the first call on each device looks up the scratch array's device
 *     address (cudaGetSymbolAddress, with that device current) and caches
 *     it; make that first call before any stream capture;
 *   - every call shares the one array and leaves its contents behind; each
 *     call rewrites or zeroes what it reads, but calls whose work overlaps on
 *     the GPU (different streams, or different host threads, without
 *     ordering between them) race on the array and give wrong results:
 *     order them on one stream or with events;
 *   - `status`: NULL, or a caller-owned DEVICE int that the GEMM kernel sets
 *     to GBGEMM_ERR_DEVICE_TIMEOUT if one of its bounded waits runs out (the
 *     caller zeroes it beforehand).  With NULL the report goes to a slot of
 *     the scratch array that the caller cannot read.
 * Errors: the argument codes of gbgemm_sgemm, GBGEMM_ERR_SCRATCH_LIMIT,
 * GBGEMM_ERR_UNSUPPORTED_DEVICE (not sm_103), GBGEMM_ERR_CUDA. */
#define GBGEMM_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int gbgemm_sgemm_split_noalloc(void* cuda_stream, char transa, char transb, int64_t m, int64_t n, int64_t k,
                               float alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                               float beta, float* C, int64_t ldc, int* status);

/* ---------------------------------------------------------------------- */
/* Split-panel inspection (tests): runs the split path's scaling and packing
 * kernels alone on one operand.
 *
 * which = 'A': the K-vectors are the m rows of op(A) (rows = m, trans = transa,
 *              X = A, ldx = lda).
 * which = 'B': the K-vectors are the n columns of op(B) (rows = n, trans =
 *              transb, X = B, ldx = ldb).
 * Outputs (device, caller-owned):
 *   amax_bits[r] = bit pattern of max_p |x(r,p)| (NaN/Inf patterns kept), rows entries.
 *   panel2 (needed when k < 512, else ignored and may be NULL; allocate
 *   gbgemm_panel_bytes(rows, k) bytes): the compact lo3 panel.  Its block
 *   (j, rb), at byte offset (j * RB + rb) * 16384, holds lo3 of k chunk 2j in
 *   logical chunks 0-3 and of k chunk 2j+1 in logical chunks 4-7, rows and
 *   swizzle as below; when the number of k chunks is odd the upper half of
 *   the last block is not written, and blocks from ceil(KC/2) on are unused.
 *   The first panel then holds hi and mid (= the two-part lo).
 *   panel: BF16 hi/lo panel of gbgemm_panel_bytes(rows, k) bytes.  It is a
 *   sequence of 16 KiB blocks, block (kc, rb) at byte offset
 *   (kc * RB + rb) * 16384 with RB = ceil(rows/256)*2 and kc = p / 32.  A
 *   block holds rows 128*rb .. 128*rb+127 and k indices 32*kc .. 32*kc+31.
 *   Row r of the block occupies bytes r*128 .. r*128+127 as eight 16-byte
 *   chunks; logical chunk c is stored at chunk position c XOR (r mod 8).
 *   Chunks 0-3 hold hi of k offsets 0-31 (8 per chunk, ascending), chunks
 *   4-7 hold lo of the same offsets.  Rows >= rows and k >= k are zero.
 * hi/lo of x are those of x * 2^-e, where e = 0 when the row's max |x| is
 * 0, not finite or in [2^-48, 2^48), and otherwise e is the frexp exponent
 * of that max.
 * Asynchronous on the handle's stream. */
size_t gbgemm_panel_bytes(int64_t rows, int64_t k);
int gbgemm_split_pack(gbgemm_handle* h, char which, char trans, int64_t rows, int64_t k,
                      const float* X, int64_t ldx, uint32_t* amax_bits, void* panel, void* panel2);

#ifdef __cplusplus
}
#endif

#endif /* GBGEMM_H */
