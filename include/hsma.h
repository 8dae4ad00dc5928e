/*
 * hsma.h - C ABI of the GB300 library for the left / lower / no-transpose
 * triangular solve with multiple right-hand sides,
 *
 *     A X = alpha B,   A (m x m) lower triangular,  B (m x n) overwritten by X,
 *
 * after "Hierarchical Shared Memory-Aware Optimization for TRSM on GPU
 * Platforms" (HSMA-TRSM).  The operation is defined in Section 2.1 by the
 * forward-substitution formula
 *
 *     x_ij = (alpha b_ij - sum_{k<i} a_ik x_kj) / a_ii .
 *
 * Conventions shared by every entry point (those of the BLAS xTRSM routine,
 * which the paper follows; the paper itself fixes no calling convention):
 *
 *  - Layout: column-major.  Element (i, j) of A is A[i + j*lda], of B is
 *    B[i + j*ldb].  Complex data (HSMA_C128) is interleaved (re, im) doubles,
 *    i.e. the memory layout of C99 `double complex` / numpy complex128.
 *  - Ownership: A and B are device memory owned by the caller.  Only the lower
 *    triangle of A is read; with HSMA_UNIT only its strict lower triangle (the
 *    diagonal is taken as 1).  Rows m..ldb-1 of B are never written.  The
 *    library keeps no pointer to A or B after the work it enqueued completes.
 *  - Asynchrony: all work is enqueued on `stream` (a cudaStream_t; NULL means
 *    the legacy default stream).  A returned HSMA_OK means "validated and
 *    enqueued"; the result is ready once the stream reaches that point.
 *  - alpha: HOST pointer to one double (real dtypes) or two doubles (re, im)
 *    for HSMA_C128.
 *  - Argument errors return HSMA_ERR_INVALID_ARG and enqueue nothing:
 *    m < 0, n < 0, lda < max(1, m), ldb < max(1, m), a NULL A/B/alpha when
 *    m*n > 0, an unknown dtype or diag.
 *  - Quick returns: m == 0 or n == 0 is a no-op; alpha == 0 sets B := 0 and does
 *    not read A.
 *  - A singular A (a zero on the diagonal) is not detected; IEEE infinities and
 *    NaNs propagate, as in BLAS.
 *  - Workspace (diagonal-block inverses, refinement copies, batch schedules)
 *    is taken from a stream-ordered memory pool the library keeps per device
 *    (CUDA's default pool while `stream` is capturing a graph) on `stream`
 *    and released on the same stream; released workspace stays reserved in
 *    the pool, up to 4 GiB per device, for later calls.  HSMA_ERR_NO_MEMORY
 *    if the allocation fails.  Nothing is allocated on the small path of
 *    hsma_trsm_llnn.
 *  - CUDA errors surfacing at enqueue time return HSMA_ERR_CUDA.
 *  - Thread safety: calls on different streams may run concurrently; the
 *    tuning table is read-only after hsma_tuning_load.
 */
#ifndef HSMA_H
#define HSMA_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HSMA_API __attribute__((visibility("default")))
#else
#define HSMA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HSMA_R64 = 0,      /* double                                                */
  HSMA_C128 = 1,     /* double complex                                        */
  HSMA_R32_BF16 = 2, /* float result; trailing updates in BF16 on tensor cores
                        with FP32 accumulation                                */
  HSMA_R64_IR = 3,   /* double result from FP32-result solves plus FP64
                        iterative refinement                                  */
  HSMA_R32 = 4,      /* float: m <= 64 in FP32 on the CUDA cores; larger m as
                        HSMA_R32_BF16 (FP32 result)                           */
  HSMA_C64 = 5       /* float complex: m <= 64 in FP32 on the CUDA cores;
                        larger m solved in complex FP64 (emulated products)
                        and rounded back                                      */
} hsma_dtype_t;

typedef enum { HSMA_NON_UNIT = 0, HSMA_UNIT = 1 } hsma_diag_t;
typedef enum { HSMA_LEFT = 0, HSMA_RIGHT = 1 } hsma_side_t;
typedef enum { HSMA_LOWER = 0, HSMA_UPPER = 1 } hsma_uplo_t;
typedef enum { HSMA_NO_TRANS = 0, HSMA_TRANS = 1, HSMA_CONJ_TRANS = 2 } hsma_trans_t;

typedef enum {
  HSMA_OK = 0,
  HSMA_ERR_INVALID_ARG = 1,
  HSMA_ERR_UNSUPPORTED = 2,
  HSMA_ERR_NO_MEMORY = 3,
  HSMA_ERR_CUDA = 4,
  HSMA_ERR_TIMEOUT = 5,
  HSMA_ERR_NOT_CONVERGED = 6,
  HSMA_ERR_BUSY = 7
} hsma_status_t;

typedef enum { HSMA_PATH_AUTO = 0, HSMA_PATH_SMALL = 1, HSMA_PATH_BLOCKED = 2 } hsma_path_t;

/* Bits OR-ed into a caller-provided device status word by the batched kernel. */
#define HSMA_DEVERR_BAD_SIZE 0x1u  /* an instance had m<0, n<0, m>64 or ld < max(1,m) */
#define HSMA_DEVERR_NULL_PTR 0x2u  /* an instance with m*n > 0 had a NULL A or B      */
#define HSMA_DEVERR_BAD_PIVOT 0x8u /* hsma_getrs_vbatched: a pivot outside [k+1, m]   */

/* Blocked-path configuration values (hsma_opts_t / hsma_plan_t). */
#define HSMA_TILE_64x64 1   /* FP64 tensor-product CTA tile, rows x columns of B */
#define HSMA_TILE_128x16 2
#define HSMA_TILE_128x8 3
#define HSMA_SPLITK_AUTO 1  /* split K across CTAs when the tiles leave SMs idle */
#define HSMA_SPLITK_OFF 2
#define HSMA_LOOK_RIGHT 1   /* after X_r: B_{r+1:} -= A_{r+1:,r} X_r              */
#define HSMA_LOOK_LEFT 2    /* before X_r: B_r -= A_{r,0:r} X_{0:r} (Section 4.3)  */

/* Plan chosen for one solve (Section 4.1's dispatcher and Section 4.3.2's
 * configuration lookup: the nearest profiled (m, n) of the autotuned table). */
typedef struct {
  int32_t path;       /* hsma_path_t: SMALL (m <= 64) or BLOCKED                    */
  int32_t nb;         /* BLOCKED: diagonal block size (the paper's N_B)             */
  int32_t groups;     /* SMALL: row groups per warp G; a warp holds 32/G columns   */
  int32_t tile;       /* BLOCKED FP64 products: HSMA_TILE_*, 0 = by n (128x8 for
                         n <= 8, 128x16 for n <= 48, else 64x64)                  */
  int32_t split_k;    /* BLOCKED: HSMA_SPLITK_*                                     */
  int32_t looking;    /* BLOCKED: HSMA_LOOK_*                                       */
  int32_t panel_cols; /* emulated FP64 products: real columns per update panel     */
  int32_t reserved;
} hsma_plan_t;

/* Options for hsma_trsm_llnn_ex; zero-initialise for defaults. */
typedef struct {
  int32_t path;        /* hsma_path_t; AUTO lets the planner choose                 */
  int32_t nb;          /* BLOCKED: force N_B (16..512, a multiple of 16); 0 = table */
  int32_t groups;      /* SMALL: force G in {1,2,4,8,16,32}; 0 = planner            */
  int32_t ir_max_iter; /* R64_IR: refinement steps at most; 0 = 10                   */
  double ir_tol;       /* R64_IR: stop when ||alpha B - L X||_F / (||L||_F ||X||_F +
                          |alpha| ||B||_F) <= ir_tol; 0 = 1e-15                    */
  int32_t bf16_terms;  /* R32_BF16 / R64_IR: BF16 products per update (1 = plain,
                          3 = hi/lo split of both operands); 0 = planner           */
  int32_t ir_residual; /* R64_IR: 0 = residual products emulated in FP64 on the BF16
                          tensor cores (exact integer slices; m <= 16384, else 1),
                          1 = FP64 tensor products (DMMA)                          */
  int32_t fp64_products; /* R64 / C128 blocked path: 0 = FP64 tensor products
                          (DMMA, IEEE FP64 roundings); 1 = FP64 emulated on the
                          BF16 tensor cores: both operands cut into 10 exact
                          6-bit digit slices per row / column scale, slice-pair
                          products summed exactly in FP32 and folded into the
                          FP64 result (error below 2^-59 of row max x column
                          max per product term; N_B <= 512, default 512)      */
  int32_t tile;        /* BLOCKED FP64 products: HSMA_TILE_*; 0 = table         */
  int32_t split_k;     /* BLOCKED: HSMA_SPLITK_*; 0 = table                     */
  int32_t looking;     /* BLOCKED: HSMA_LOOK_*; 0 = table                       */
  int32_t panel_cols;  /* fp64_products = 1: real columns per update panel
                          (a multiple of 64, 512 .. 8192); 0 = table          */
} hsma_opts_t;

/* Filled by hsma_trsm_llnn_ex (host memory).  Fields describing the device
 * result (ir_iters, ir_residual) are valid after the stream is synchronised. */
typedef struct {
  hsma_plan_t plan;
  int32_t ir_iters;     /* R64_IR: refinement steps taken                          */
  int32_t converged;    /* R64_IR: 1 if ir_tol was reached                         */
  double ir_residual;   /* R64_IR: final normwise residual ratio                   */
} hsma_info_t;

/* Human-readable name of a status code (static storage). */
HSMA_API const char *hsma_status_string(int status);

/* Library version "major.minor.patch" (static storage). */
HSMA_API const char *hsma_version(void);

/*
 * Single solve  A X = alpha B  (Section 2.1; dispatch of Section 4.1).
 *
 * dtype  HSMA_R64 / HSMA_C128: A, B are double / interleaved complex double.
 *        HSMA_R32_BF16: A, B are float; the result is FP32.
 *        HSMA_R64_IR: A, B are double; FP32-result solves refined in FP64.
 *        The host reads the stopping test after each refinement step (the
 *        call then waits for the stream once per step, and returns once the
 *        refinement has stopped); on a capturing stream every allowed step
 *        is recorded instead and the device skips the steps after
 *        convergence.
 * diag   HSMA_NON_UNIT or HSMA_UNIT.
 * Paths: m <= 64 runs the small direct solve (Section 4.2; triangle in shared
 * memory, columns of X in registers, warp-shuffle forward substitution);
 * larger m runs the blocked two-phase algorithm (Section 4.3): parallel
 * inversion of the N_B x N_B diagonal blocks (Algorithm 2, O(N_B) shared
 * memory), then for each block row the solve product X_r = D_r^{-1} B_r and the
 * trailing update with tensor-core (DMMA) products.
 */
HSMA_API hsma_status_t hsma_trsm_llnn(int dtype, int diag, int64_t m, int64_t n, const void *alpha,
                             const void *A, int64_t lda, void *B, int64_t ldb, void *stream);

/* As hsma_trsm_llnn with options (may be NULL) and a host info record (may be NULL). */
HSMA_API hsma_status_t hsma_trsm_llnn_ex(int dtype, int diag, int64_t m, int64_t n, const void *alpha,
                                const void *A, int64_t lda, void *B, int64_t ldb, void *stream,
                                const hsma_opts_t *opts, hsma_info_t *info);

/*
 * The other BLAS triangular-solve variants (no paper counterpart: the paper
 * studies the left / lower / no-transpose case):
 *   side HSMA_LEFT:  op(A) X = alpha B, A is m x m (lda >= max(1, m));
 *   side HSMA_RIGHT: X op(A) = alpha B, A is n x n (lda >= max(1, n));
 *   uplo: the triangle of A that is referenced; trans: op(A) = A, A^T or A^H
 *   (A^H = A^T for real dtypes); diag as for hsma_trsm_llnn.
 * B is m x n (ldb >= max(1, m)), overwritten with X.  Every dtype.  The left /
 * lower / no-transpose case is hsma_trsm_llnn_ex itself; the others gather
 * the triangle into lower form (rows reversed when op(A) would be upper) and
 * B (transposed for the right side) into workspace of (order of A)^2 + m n
 * elements, solve, and scatter X back.  opts and info as for
 * hsma_trsm_llnn_ex (they apply to that inner solve).
 */
HSMA_API hsma_status_t hsma_trsm(int dtype, int side, int uplo, int trans, int diag, int64_t m, int64_t n,
                                 const void *alpha, const void *A, int64_t lda, void *B, int64_t ldb, void *stream,
                                 const hsma_opts_t *opts, hsma_info_t *info);

/*
 * Varlen batch of independent small solves in one persistent launch (batched
 * TRSM is the paper's future work, Section 6; each instance is the Section 2.1
 * solve done by the small kernel of Section 4.2).
 *
 * dtype  HSMA_R64, HSMA_C128, HSMA_R32 or HSMA_C64 (one dtype and one alpha for
 *        the whole batch; FP32 dtypes compute in FP32).
 * batch  number of instances (>= 0).
 * d_m, d_n, d_lda, d_ldb: DEVICE arrays of `batch` int32 sizes.
 * d_A, d_B: DEVICE arrays of `batch` device pointers.
 * max_m  host upper bound on every m_i, or 0 for "unknown" (taken as 64); up
 *        to 64 it sizes the workspace, and an instance with m_i > max_m is
 *        skipped and flagged HSMA_DEVERR_BAD_SIZE.  max_m > 64 admits
 *        instances of any size: the call then reads the batch's sizes and
 *        pointers back to the host (it waits for the stream once, so it is
 *        not capturable), runs the instances with m_i <= 64 as the batch and
 *        solves each larger one on the same stream through the single-solve
 *        path (hsma_trsm; blocked path, planner's configuration).
 * max_n  host upper bound on every n_i, or 0 if unknown (only a hint).
 * d_status: optional DEVICE uint32 word; the kernel ORs HSMA_DEVERR_* bits into
 *        it for instances it skips as invalid.  May be NULL.
 * HSMA_C128: the columns of all instances with the same m are dealt to warps
 * 32 (16 for m > 32) at a time, so a warp may serve several instances; the
 * other dtypes deal each instance's column tiles to the warps of one CTA.  An
 * instance's arithmetic never depends on the others, so results are
 * bit-identical to solving it alone through this entry point with batch = 1.
 * Workspace (stream-ordered pool): for HSMA_C128 room for the pre-scaled
 * triangle and diagonal of every instance, batch x r (r + 1) / 2 elements
 * with r = max_m rounded up to even, plus 20 bytes per instance; otherwise
 * 4 bytes per instance.
 */
HSMA_API hsma_status_t hsma_trsm_llnn_vbatched(int dtype, int diag, int32_t batch, const int32_t *d_m,
                                      const int32_t *d_n, const void *alpha, const void *const *d_A,
                                      const int32_t *d_lda, void *const *d_B, const int32_t *d_ldb,
                                      int32_t max_m, int32_t max_n, uint32_t *d_status, void *stream);

/*
 * The varlen batch for the other left-side variants (no paper counterpart):
 * op(A_i) X_i = alpha B_i with uplo / trans as for hsma_trsm; the kernel reads
 * A_i and B_i through an index map (row reversal for upper op(A), transposed
 * and conjugated reads), so there are no copies.  side must be HSMA_LEFT
 * (HSMA_RIGHT returns HSMA_ERR_UNSUPPORTED; use hsma_trsm per instance).
 * Other arguments and errors as hsma_trsm_llnn_vbatched, which is this call
 * with HSMA_LEFT, HSMA_LOWER, HSMA_NO_TRANS.
 */
HSMA_API hsma_status_t hsma_trsm_vbatched(int dtype, int side, int uplo, int trans, int diag, int32_t batch,
                                          const int32_t *d_m, const int32_t *d_n, const void *alpha,
                                          const void *const *d_A, const int32_t *d_lda, void *const *d_B,
                                          const int32_t *d_ldb, int32_t max_m, int32_t max_n, uint32_t *d_status,
                                          void *stream);

/*
 * Varlen batch of LU-factor solves: the small solve fused with its consumer,
 * for the LU factorisations that motivate the paper (Section 1; fusion at
 * small scales is its future work, Section 6).  Instance i holds
 * A_i = P_i L_i U_i as LAPACK getrf leaves it: one m_i x m_i column-major
 * array (ld d_lda[i]) with L_i's multipliers below the diagonal (unit
 * diagonal, not stored) and U_i on and above it.  Then
 *     X_i = U_i^{-1} L_i^{-1} P_i^T (alpha B_i)   overwrites B_i,
 * i.e. A_i X_i = alpha B_i.  HSMA_C128: one pass applies the row
 * interchanges, then the two triangular solves run as two launches of the
 * column-packed batch (the upper solve through the left / upper index map).
 * The other dtypes: per instance one CTA applies the interchanges, solves
 * with L_i and then with U_i, in ONE launch for the batch; the intermediate
 * stays in that CTA's cache.
 *
 * d_ipiv: NULL (no interchanges) or a DEVICE array of `batch` DEVICE pointers,
 *        each to instance i's m_i int32 pivots in LAPACK's convention
 *        (1-based; row k was interchanged with row ipiv[k] >= k, in order
 *        k = 1..m_i); a NULL entry means no interchanges for that instance.
 * dtype, batch, d_m, d_n, alpha, d_lda, d_B, d_ldb, max_m, max_n: as for
 *        hsma_trsm_llnn_vbatched (alpha = 0 gives X_i = 0).
 * d_status: as for hsma_trsm_llnn_vbatched, plus HSMA_DEVERR_BAD_PIVOT for an
 *        instance with a pivot outside [k, m_i] (that instance's B_i is left
 *        untouched).
 * Results equal two hsma_trsm_vbatched calls (unit lower, then upper) on the
 * interchanged B, bit for bit.  Errors as hsma_trsm_llnn_vbatched; with
 * max_m > 64 the instances above 64 are solved one by one through hsma_getrs
 * (hsma_potrs for the Cholesky batch below) after one read-back of the sizes,
 * pointers and pivot pointers.
 */
HSMA_API hsma_status_t hsma_getrs_vbatched(int dtype, int32_t batch, const int32_t *d_m, const int32_t *d_n,
                                           const void *alpha, const void *const *d_LU, const int32_t *d_lda,
                                           const int32_t *const *d_ipiv, void *const *d_B, const int32_t *d_ldb,
                                           int32_t max_m, int32_t max_n, uint32_t *d_status, void *stream);

/*
 * One solve with LU or Cholesky factors, any m (the factorisations that
 * motivate the paper, Section 1).  hsma_getrs: A = P L U packed as for
 * hsma_getrs_vbatched (DEVICE LU, lda >= max(1,m)); ipiv: NULL or a DEVICE
 * array of m int32 pivots in LAPACK's convention; X = U^{-1} L^{-1} P^T
 * (alpha B) overwrites B (DEVICE, ldb >= max(1,m)).  The interchanges are
 * applied as one gather through a workspace copy of B (pivots read by one
 * CTA: shared memory up to m = 28000, global memory beyond), then the
 * unit-lower and the upper solve run through hsma_trsm with `opts` (small
 * kernel or blocked path, FP64 products emulated on request).  A pivot outside
 * [k, m] sets HSMA_DEVERR_BAD_PIVOT in the device error word
 * (hsma_device_status) and the interchanges are skipped (X is then not the
 * solution).  hsma_potrs: A = L L^H with L in the lower triangle of L (the
 * strict upper triangle is not read); X = L^{-H} L^{-1} (alpha B) (L^T for
 * real dtypes).  Both: dtype any hsma_dtype_t; m = 0 or n = 0 is a no-op;
 * asynchronous on `stream`; errors as hsma_trsm.
 */
/*
 * Varlen batch of Cholesky-factor solves (the same kernels as
 * hsma_getrs_vbatched without its interchange pass): instance i holds A_i = L_i L_i^H's lower factor L_i as LAPACK
 * potrf leaves it (uplo = lower; the strict upper triangle is not read), and
 *     X_i = L_i^{-H} L_i^{-1} (alpha B_i)   overwrites B_i
 * (L_i^T for the real dtypes).  The second solve reads L_i through the
 * reversed, transposed and conjugated index map.  Arguments and errors as
 * hsma_getrs_vbatched without pivots; results equal two hsma_trsm_vbatched
 * calls (lower, then lower with HSMA_CONJ_TRANS) bit for bit.
 */
HSMA_API hsma_status_t hsma_getrs(int dtype, int64_t m, int64_t n, const void *alpha, const void *LU, int64_t lda,
                                  const int32_t *ipiv, void *B, int64_t ldb, void *stream, const hsma_opts_t *opts);
HSMA_API hsma_status_t hsma_potrs(int dtype, int64_t m, int64_t n, const void *alpha, const void *L, int64_t lda,
                                  void *B, int64_t ldb, void *stream, const hsma_opts_t *opts);

HSMA_API hsma_status_t hsma_potrs_vbatched(int dtype, int32_t batch, const int32_t *d_m, const int32_t *d_n,
                                           const void *alpha, const void *const *d_L, const int32_t *d_lda,
                                           void *const *d_B, const int32_t *d_ldb, int32_t max_m, int32_t max_n,
                                           uint32_t *d_status, void *stream);

/*
 * The varlen batch with its matrices in HOST memory (no paper counterpart:
 * the paper's solves are device-resident).  The batch is cut into `chunks`
 * groups of consecutive instances (0 = 8; 6 for the packed-triangle entry
 * point below; at most 256).  The sizes and
 * offsets are copied once; then the groups' host-to-device copies run in
 * order on an internal copy-in stream, each group's batched solve starts (on
 * one of two internal compute streams) as soon as its copy has landed, and
 * its X goes back on an internal copy-out stream as soon as it is solved, so
 * the copies overlap the solves.  Device workspace: the whole batch's A and B,
 * the per-instance tables and, for HSMA_C128, the staged triangles of two
 * chunks (stream-ordered pool, released at the end).
 *
 * h_m, h_n: HOST arrays of `batch` sizes (0 <= m_i <= 64, n_i >= 0).
 * hA, hB: HOST buffers holding every A_i (column-major, lda = m_i, m_i^2
 *        elements at element offset h_offA[i]) and every B_i (ldb = m_i, m_i n_i
 *        elements at h_offB[i]); offsets increase and regions do not overlap.
 * hX: HOST buffer receiving X_i at h_offB[i] (may equal hB).  Each group is
 *        copied as one range, so elements of hX lying between two instances
 *        of a group receive the same elements of hB; nothing outside the
 *        groups' ranges is written.
 * Use page-locked host memory for asynchronous copies (pageable memory works,
 * with synchronous staging).  The call is asynchronous on `stream`: hX is
 * valid, and hA, hB, h_m, h_n, h_offA, h_offB may be reused, once the stream
 * has been synchronised.
 * Results equal hsma_trsm_llnn_vbatched on the same data, bit for bit.
 * Errors: INVALID_ARG for a bad size, offset order or null pointer;
 * UNSUPPORTED for m_i > 64 or another dtype.  Concurrent calls share the
 * internal streams (their work is serialised, not mixed).
 */
HSMA_API hsma_status_t hsma_trsm_llnn_vbatched_host(int dtype, int diag, int32_t batch, const int32_t *h_m,
                                                    const int32_t *h_n, const void *alpha, const void *hA,
                                                    const int64_t *h_offA, const void *hB, const int64_t *h_offB,
                                                    void *hX, int32_t chunks, void *stream);

/*
 * As hsma_trsm_llnn_vbatched_host, with each A_i stored in host memory as a
 * packed lower triangle (LAPACK's packed lower format: column j holds rows
 * j .. m_i - 1, one column after the other, m_i (m_i + 1) / 2 elements from
 * element offset h_offA[i]; offsets increase by at least that much).  Only
 * the triangle crosses the link (about half the bytes of a square A for the
 * batched sizes).  HSMA_C128 batches read the packed triangles on the device
 * as they are; the other dtypes expand them into the square layout before
 * each chunk's solve (device workspace: the packed copy, and for those dtypes
 * the squares).  Results equal hsma_trsm_llnn_vbatched_host's on the same
 * triangles, bit for bit.  Other arguments, asynchrony and errors as
 * hsma_trsm_llnn_vbatched_host.
 */
HSMA_API hsma_status_t hsma_trsm_llnn_vbatched_host_tp(int dtype, int diag, int32_t batch, const int32_t *h_m,
                                                       const int32_t *h_n, const void *alpha, const void *hAp,
                                                       const int64_t *h_offA, const void *hB, const int64_t *h_offB,
                                                       void *hX, int32_t chunks, void *stream);

/*
 * Allocation-free form of hsma_trsm_llnn_vbatched (same arguments, same
 * results bit for bit).  It has no counterpart in the paper; it exists for
 * callers that cannot have the library allocate device memory during a
 * solve: a serving loop that reserved all device memory up front, an
 * application whose own allocator owns every byte of the GPU, or code that
 * runs where a call into the CUDA allocator is not allowed.
 *
 * The batch schedule is kept in one static device array inside the library
 * instead of stream-ordered workspace; every GPU that loads the library holds
 * that array (about 256 KB) until the process exits.  Limit: batch <= 65536
 * instances; a larger batch returns HSMA_ERR_UNSUPPORTED without launching.
 * The first call on a device looks up the array's device address (one
 * cudaGetSymbolAddress per device, made with that device current) and, like
 * the first varlen batch of any kind, copies a 32 KB table of per-size
 * schedule entries into a second static array; make that first call before
 * any stream capture (a capturing first call computes the entries in the
 * kernel instead).  The call itself allocates and frees nothing.  All calls share the one array: each call resets the counters it
 * needs, but calls whose work overlaps on the GPU (on different streams, or
 * from different threads, without ordering between them) race on the array
 * and must be serialised by the caller.
 */
HSMA_API hsma_status_t hsma_trsm_llnn_vbatched_noalloc(int dtype, int diag, int32_t batch, const int32_t *d_m,
                                                       const int32_t *d_n, const void *alpha,
                                                       const void *const *d_A, const int32_t *d_lda,
                                                       void *const *d_B, const int32_t *d_ldb, int32_t max_m,
                                                       int32_t max_n, uint32_t *d_status, void *stream);

/* Planner query (host only, no GPU needed): the path, N_B and G that
 * hsma_trsm_llnn would use for (dtype, m, n). */
HSMA_API hsma_status_t hsma_plan(int dtype, int64_t m, int64_t n, hsma_plan_t *out);

/* Estimated FP64 (or FP32) warp instructions of the small path for one solve
 * with G row groups (the cost model the planner minimises); host only. */
HSMA_API double hsma_small_cost(int dtype, int64_t m, int64_t n, int32_t groups);

/* Replace the compiled configuration table with the one in `path` (a text
 * file of lines "dtype m n nb" or "dtype m n nb tile split_k looking
 * panel_cols", the autotuner's output; see Section 4.3.2: the nearest tested
 * scale in (log m, log n) wins).  NULL restores the compiled table. */
HSMA_API hsma_status_t hsma_tuning_load(const char *path);

/*
 * Fill a device matrix with the seeded synthetic workload (not part of the
 * solve; used to build inputs on the device).  kind 0 = A (lower triangular:
 * off-diagonal (2u-1)/m, diagonal 1+u, zeros above), kind 1 = B (2u-1),
 * kind 2 = packed LU factors as getrf leaves them without interchanges (A's
 * entries below the diagonal; on and above it the transpose of a second
 * triangle drawn like A from the streams U_RE = 4, U_IM = 5), drawn
 * from the counter-based SplitMix64 streams described in inputs.py.  `inst` is
 * the instance id (-1 for a single solve).  rows x cols written at `dst` with
 * leading dimension ld (>= rows); dtype HSMA_R64 or HSMA_C128.
 */
HSMA_API hsma_status_t hsma_gen_matrix(int dtype, int kind, uint64_t seed, int64_t inst, int64_t m,
                              int64_t cols, void *dst, int64_t ld, void *stream);

/*
 * Serving loop (a continuous-batching server for streams of solves; batched
 * TRSM is the paper's future work, Section 6).  A server owns a scheduler thread, a
 * ring of CUDA streams and a device memory pool on the current device.
 * Submitted requests are admitted in arrival order while their device memory
 * (A, B, pivots and the blocked path's workspace) fits `budget_bytes`;
 * admitted requests with m <= 64 that are ready together run as one varlen
 * batched launch per dtype and kind (triangular solves; LU- and
 * Cholesky-factor solves through the fused factor-solve batch), larger ones
 * run the blocked path on the streams (hsma_trsm_llnn_ex, hsma_getrs,
 * hsma_potrs), overlapping on the device.  Memory is freed when a request's completion event fires; latency is
 * measured from submission to that event.  Each result equals the request
 * solved alone (up to the rounding of the path chosen for its size).
 */
typedef struct hsma_server hsma_server_t;

#define HSMA_SERVER_FAKE_DEVICE 0x1u /* no GPU: launches complete after a modelled time (tests) */
#define HSMA_SERVER_FP64_EMULATED 0x2u /* requests with m >= 384 use hsma_opts_t.fp64_products = 1 */

typedef struct {
  int32_t dtype;  /* HSMA_R64 or HSMA_C128                                        */
  int32_t diag;
  int64_t m, n;   /* >= 1                                                           */
  double alpha[2];
  /* inputs: copied from host memory when A_host != NULL (column-major, lda/ldb
     >= m; pinned memory makes the copy asynchronous), otherwise generated on
     the device from (gen_seed, gen_inst) as hsma_gen_matrix does             */
  const void *A_host;
  int64_t lda;
  const void *B_host;
  int64_t ldb;
  uint64_t gen_seed;
  int64_t gen_inst;
  /* output: copied to X_host (ldx >= m) before the request completes, or
     discarded when X_host == NULL                                            */
  void *X_host;
  int64_t ldx;
  /* what to solve with A (HSMA_REQ_*; 0 = the triangular solve)              */
  int32_t kind;
  int32_t reserved;
  /* HSMA_REQ_GETRS: m pivots (LAPACK's 1-based sequential interchanges) in
     host memory, or NULL for none; must be NULL for the other kinds        */
  const int32_t *ipiv_host;
} hsma_request_t;

/* Request kinds.  TRSM: X = alpha L^{-1} B (L the lower triangle of A, diag as
 * given).  GETRS: A holds packed LU factors (hsma_getrs), X = U^{-1} L^{-1}
 * P^T (alpha B); generated inputs use hsma_gen_matrix kind 2 (no
 * interchanges).  POTRS: A holds a lower Cholesky factor L (hsma_potrs),
 * X = L^{-H} L^{-1} (alpha B); generated inputs draw L as kind 0.  diag is
 * ignored by GETRS and POTRS. */
#define HSMA_REQ_TRSM 0
#define HSMA_REQ_GETRS 1
#define HSMA_REQ_POTRS 2

typedef struct {
  uint64_t submitted, admitted, completed;
  uint64_t bytes_in_use, peak_bytes_in_use, budget_bytes;
  uint64_t batched_launches, blocked_launches;
} hsma_server_stats_t;

/* Create a server on the current device (flags: 0, HSMA_SERVER_FAKE_DEVICE, HSMA_SERVER_FP64_EMULATED). */
HSMA_API hsma_status_t hsma_server_create(size_t budget_bytes, int n_streams, unsigned int flags,
                                          hsma_server_t **out);
/* Enqueue a request (thread-safe, non-blocking); *ticket identifies it.  Host
 * buffers must stay valid until the request completes.  A request that can
 * never fit the budget completes with HSMA_ERR_NO_MEMORY. */
HSMA_API hsma_status_t hsma_server_submit(hsma_server_t *s, const hsma_request_t *req, uint64_t *ticket);
/* *done = 1 once the request completed; then *latency_s is submission-to-
 * completion time and the return value is the request's own status. */
HSMA_API hsma_status_t hsma_server_poll(hsma_server_t *s, uint64_t ticket, int *done, double *latency_s);
/* Wait until every submitted request completed (timeout_s <= 0: no limit). */
HSMA_API hsma_status_t hsma_server_drain(hsma_server_t *s, double timeout_s);
HSMA_API hsma_status_t hsma_server_stats(hsma_server_t *s, hsma_server_stats_t *out);
/* Finish outstanding work, then free the server. */
HSMA_API hsma_status_t hsma_server_destroy(hsma_server_t *s);

/*
 * BF16 tensor-core update used by HSMA_R32_BF16 (exposed for direct use and
 * testing): C = beta*C - A * Bt^T with A (M x K) and Bt (N x K) row-major
 * BF16 (K contiguous; K a positive multiple of 64) and C (M x N) column-major
 * FP32 with leading dimension ldc.  Products accumulate in FP32 in tensor
 * memory (tcgen05.mma kind::f16).  Device pointers; A and Bt 16-byte aligned.
 */
HSMA_API hsma_status_t hsma_gemm_bf16_update(int64_t M, int64_t N, int64_t K, const void *A, const void *Bt,
                                             float beta, float *C, int64_t ldc, void *stream);

/*
 * FP64 product emulated on the BF16 tensor cores, the building block of the
 * fp64_products = 1 blocked path and of the R64_IR residual (exposed for
 * direct use and testing): C -= A X with A (M x K), X (K x N) and C (M x N)
 * column-major FP64 (device pointers, leading dimensions lda, ldx, ldc).  Each
 * row of A and column of X is scaled by a power of two, cut into 10 signed
 * 6-bit digit slices (BF16, exact), and the slice pairs with p + q <= 11 are
 * multiplied with FP32 accumulation that stays exact for K <= 16384; each
 * group of equal-weight pairs is added to C in FP64.  Error per entry: below
 * 2^-59 x (max |A row|) x (max |X column|) x K, plus one FP64 rounding per
 * group (10 groups when K <= 1600).  Errors: INVALID_ARG for negative sizes,
 * short leading dimensions or null pointers; UNSUPPORTED for K > 16384 or
 * M, N beyond INT32_MAX.  Workspace comes from the library's stream-ordered
 * pool.
 */
HSMA_API hsma_status_t hsma_gemm_f64_emulated(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                                              const double *X, int64_t ldx, double *C, int64_t ldc, void *stream);

/*
 * Device-side error bits the library's kernels raise (a bounded wait that ran
 * out: HSMA_DEVERR_TIMEOUT; a refinement that did not converge:
 * HSMA_DEVERR_NOT_CONVERGED).  Synchronises the device, returns the bits
 * accumulated since the last call in *out, and clears them.
 */
#define HSMA_DEVERR_TIMEOUT 0x4u
/* R64_IR: the refinement took ir_max_iter steps without reaching ir_tol.  The
 * same solve called with a non-NULL hsma_info_t also returns
 * HSMA_ERR_NOT_CONVERGED; without one this bit is the only report. */
#define HSMA_DEVERR_NOT_CONVERGED 0x10u
HSMA_API hsma_status_t hsma_device_status(unsigned int *out);

/*
 * Self-check of the failure-detection path: one thread waits, with the same
 * bounded mbarrier wait the tensor-core kernels use, on a barrier that nothing
 * arrives on.  The wait gives up after limit_ns nanoseconds of wall time
 * (1 ms .. 2 s), ORs HSMA_DEVERR_TIMEOUT into the device error word and the
 * kernel writes 2 to the DEVICE int *d_returned (1 would mean the wait
 * completed).  The context stays usable.  Asynchronous on `stream`.  Errors:
 * INVALID_ARG for a null d_returned or a limit out of range.
 */
HSMA_API hsma_status_t hsma_check_wait_timeout(uint64_t limit_ns, int *d_returned, void *stream);

/*
 * Phase tracing (off by default; also switched on by HSMA_PHASE_TIMING=1 in
 * the environment).  When on, the library records a pair of CUDA events
 * around every kernel it launches, named by phase: "small_single",
 * "vbatched_schedule", "vbatched_solve", "diag_inverse", "solve_gemm",
 * "update_gemm", "convert", "residual", ...  Launches captured into a CUDA
 * graph are not traced.
 */
HSMA_API hsma_status_t hsma_trace_enable(int on);
/* Total device milliseconds and launch count of `phase` since the last reset
 * (waits for the recorded events). */
HSMA_API hsma_status_t hsma_trace_read(const char *phase, double *total_ms, long long *count);
/* Kernel launches made by the library since the last reset (counted whether
 * or not tracing is on; captured launches included). */
HSMA_API long long hsma_trace_launches(void);
HSMA_API void hsma_trace_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* HSMA_H */
