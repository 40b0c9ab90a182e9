/*
 * tsqr.h — C ABI of the GB300 (sm_103a) tall-skinny QR library.
 *
 * The library computes the QR factorization A = Q R of a tall, skinny, column-major
 * m-by-n FP64 matrix (m >= n, n <= 128) by TSQR, "Tall and Skinny QR": the rows are
 * split into P block-rows ("domains", the leaves), each leaf is factored by
 * Householder reflections, and the leaves' n-by-n triangular R factors are reduced
 * by a tree whose basic operation is the QR factorization of stacked triangles
 * (paper §2.3). The reduce operator is associative, so every tree shape yields the
 * same R; the library returns R with a non-negative diagonal, which makes it unique
 * for full-rank A (paper §2.2). Q is kept implicitly as the set of Householder
 * reflectors H = I - tau v v^T of every leaf and tree node (paper §2.2), and can be
 * applied (Q^T B, Q B) or formed explicitly (thin Q, paper §4 Table 2 / Property 1).
 *
 * Conventions for every entry point:
 *   - Matrices are column-major: element (i, j) of X is X[i + j*ldx], ldx >= rows.
 *   - Pointers to matrix data are DEVICE pointers (memory allocated by the caller,
 *     e.g. through PyTorch or cudaMalloc) unless an entry point says otherwise.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Every call is stream-ordered and asynchronous: it returns after enqueuing the
 *     work; results are valid once the stream reaches that point. Argument errors are
 *     detected on the host and returned before anything is enqueued.
 *   - The caller owns A, B, R, Q, X. The library owns a tsqr_factors object until
 *     tsqr_free(). A factor set must only be used on the device it was created on.
 *   - Numerical range: entries are squared without rescaling, so matrices with
 *     entries of magnitude above about 1e150 or columns whose squared norms
 *     underflow (below about 1e-300) are outside the supported range.
 */
#ifndef TSQR_H
#define TSQR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TSQR_OK = 0,
  TSQR_ERR_ARG = 1,         /* invalid argument (see each entry point) */
  TSQR_ERR_OOM = 2,         /* device allocation failed */
  TSQR_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  TSQR_ERR_SINGULAR = 4,    /* least squares: R has an exactly zero diagonal entry */
  TSQR_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  TSQR_ERR_UNSUPPORTED = 6  /* valid request this build cannot serve */
} tsqr_status;

typedef enum {
  TSQR_FP64 = 0,  /* every operation in FP64 */
  TSQR_MIXED = 1, /* leaf factorizations in FP32 (A rounded on load), tree and
                     refinement in FP64 */
  TSQR_AUTO = 2   /* batch items only: FP64 or MIXED by a cost model (R-only items: FP64) */
} tsqr_prec;

/* flags for tsqr_factor */
enum {
  TSQR_INPLACE = 1,   /* the reflectors overwrite A (A is then not const) */
  TSQR_TWO_LEVEL = 2, /* two-level tree: a flat chain over the leaves inside each
                         CTA, then the arity-k tree across CTAs (the GPU form of the
                         paper's topology-aware tree, §2.3 and §3) */
  TSQR_CLUSTER = 4    /* with arity 2: the binary tree's levels run three at a time in
                         thread-block clusters of 8 CTAs, whose combines exchange their
                         triangles row by row through distributed shared memory and run
                         as a pipeline (the cluster tier of a hierarchical tree, §2.3 and
                         §3: CTA -> cluster -> grid). Ignored for other arities or when a
                         combine's triangles do not fit one CTA's shared memory
                         (n + extra columns beyond about 80). Same R and reflectors as
                         the plain binary tree. */
};

typedef struct tsqr_factors tsqr_factors; /* opaque factor set */

/*
 * tsqr_factor — TSQR factorization A = Q R (paper §2.3; reflectors §2.2).
 *
 *   A       device, m-by-n column-major FP64, leading dimension lda >= m. Read only,
 *           unless flags has TSQR_INPLACE, in which case it receives the reflectors.
 *   m, n    1 <= n <= 128, m >= n.
 *   leaf_h  rows per leaf (domain), n <= leaf_h. P = max(1, floor(m / leaf_h)) leaves;
 *           the last leaf takes the remaining m - (P-1)*leaf_h rows. A leaf taller
 *           than the on-chip tile limit is itself factored as a flat chain of tiles.
 *   arity   tree over the leaves (or over the CTA chains with TSQR_TWO_LEVEL):
 *           2..16 = k-ary tree, level by level, consecutive siblings grouped;
 *           0 = flat tree (one left-to-right chain). A trailing group of size one
 *           passes up unchanged.
 *   prec    TSQR_FP64 only (TSQR_MIXED is accepted by tsqr_lstsq).
 *   flags   TSQR_INPLACE | TSQR_TWO_LEVEL | TSQR_CLUSTER.
 *   stream  cudaStream_t.
 *   F       out: the new factor set (host pointer to an opaque handle).
 *   R       device, n-by-n column-major, ldr >= n, out: the R factor with
 *           diag(R) >= 0 (sign(0) = +1) and zeros below the diagonal. May be NULL.
 *   Errors: TSQR_ERR_ARG for n < 1, n > 128, m < n, leaf_h < n, lda < m, ldr < n,
 *           arity not in {0, 2..16}, null A or F, unknown prec/flags;
 *           TSQR_ERR_UNSUPPORTED for prec = TSQR_MIXED; TSQR_ERR_OOM; TSQR_ERR_CUDA.
 */
tsqr_status tsqr_factor(const double *A, int64_t m, int32_t n, int64_t lda, int32_t leaf_h,
                        int32_t arity, int32_t prec, int32_t flags, void *stream,
                        tsqr_factors **F, double *R, int64_t ldr);

/*
 * tsqr_caqr — QR factorization A = Q R of a wider m-by-n matrix (n up to 4096) by CAQR,
 * the communication-avoiding QR whose panel factorization is TSQR (paper §2.4; the
 * switch from TSQR to CAQR for large n, §6, and Property 5 of §4). The columns are split
 * into panels of `panel` columns. Panel p (its columns, rows p*panel..m-1 of the updated
 * matrix) is factored by TSQR as tsqr_factor does, and its Q_p^T is applied to the
 * trailing columns (the trailing-matrix update, overlapped with the panel's reduction
 * tree as in tsqr_factor_qt); the top `panel` rows of the updated trailing columns are
 * rows of R, and the next panel is the trailing block below them. Q = Q_0 Q_1 ... with
 * each Q_p acting on rows p*panel..m-1.
 *   A       device, m-by-n column-major FP64, lda >= m. Read only, unless flags has
 *           TSQR_INPLACE: A then receives every panel's reflectors and trailing updates.
 *           Otherwise the factor set holds an m-by-n working copy.
 *   m, n    1 <= n <= 4096, m >= n.
 *   panel   columns per panel, 1..128; 0 = 64.
 *   leaf_h, arity, flags (TSQR_INPLACE | TSQR_TWO_LEVEL)  as tsqr_factor, for every
 *           panel; leaf_h >= min(panel, n).
 *   F       out: a factor set that tsqr_apply_qt, tsqr_apply_q, tsqr_form_q,
 *           tsqr_solve_r, tsqr_factors_info and tsqr_free take like a TSQR one
 *           (tsqr_factors_info reports totals over the panels).
 *   R       device, n-by-n (ldr >= n), out: R with diag(R) >= 0, zeros below. May be NULL.
 *   Errors: TSQR_ERR_ARG (n outside [1, 4096], m < n, lda < m, panel outside [0, 128],
 *           leaf_h below the panel width, bad arity or flags, null A or F), TSQR_ERR_OOM,
 *           TSQR_ERR_CUDA.
 */
tsqr_status tsqr_caqr(const double *A, int64_t m, int32_t n, int64_t lda, int32_t panel, int32_t leaf_h,
                      int32_t arity, int32_t flags, void *stream, tsqr_factors **F, double *R,
                      int64_t ldr);

/*
 * tsqr_apply_qt — B <- Q^T B for the m-by-m orthogonal Q of F (paper §4, Table 2).
 *   B  device, m-by-k column-major, ldb >= m, 1 <= k. Rows 0..n-1 of the result are
 *      Q_thin^T B with the sign convention diag(R) >= 0; the other rows hold B's
 *      coordinates in an orthogonal complement that depends on the tree.
 *   Errors: TSQR_ERR_ARG (null F/B, k < 1, ldb < m), TSQR_ERR_CUDA.
 */
tsqr_status tsqr_apply_qt(const tsqr_factors *F, double *B, int64_t ldb, int32_t k,
                          void *stream);

/*
 * tsqr_factor_qt — tsqr_factor and then B <- Q^T B as tsqr_apply_qt, in one call that
 * overlaps them: the apply's launch over the leaves' reflectors runs as soon as the leaves
 * are factored, while the reduction tree's levels (which keep few SMs busy) run, and each
 * of the apply's tree levels follows the same level of the factorization. The overlap uses
 * a helper stream of the library (one per device) joined back to `stream` with events; all
 * of the call's work is ordered before work enqueued later on `stream`, and B's result is
 * bitwise that of tsqr_factor + tsqr_apply_qt.
 *   B, ldb, k  as tsqr_apply_qt (device, m-by-k, ldb >= m, k >= 1), overwritten.
 *   Other arguments as tsqr_factor; TSQR_INPLACE is not supported (TSQR_ERR_ARG).
 *   Errors: as tsqr_factor, plus TSQR_ERR_ARG for null B, k < 1 or ldb < m.
 */
tsqr_status tsqr_factor_qt(const double *A, int64_t m, int32_t n, int64_t lda, double *B, int64_t ldb,
                           int32_t k, int32_t leaf_h, int32_t arity, int32_t prec, int32_t flags,
                           void *stream, tsqr_factors **F, double *R, int64_t ldr);

/* tsqr_apply_q — B <- Q B (the inverse of tsqr_apply_qt). Same arguments. */
tsqr_status tsqr_apply_q(const tsqr_factors *F, double *B, int64_t ldb, int32_t k,
                         void *stream);

/*
 * tsqr_form_q — the thin Q = Q [I_n; 0] (m-by-n, orthonormal columns) with
 * A = Q R and diag(R) >= 0 (paper §4, Property 1: "Q and R" costs about twice "R").
 *   Q  device, m-by-n column-major, ldq >= m, out.
 */
tsqr_status tsqr_form_q(const tsqr_factors *F, double *Q, int64_t ldq, void *stream);

/*
 * tsqr_orthonormalize — Q-only TSQR: an orthonormal basis Q (m-by-n) of the columns of A,
 * with A = Q R and diag(R) >= 0, as tsqr_factor followed by tsqr_form_q and tsqr_free in
 * one call. This is the orthogonalization step of block iterative methods (block
 * eigensolvers, block Krylov), the use the paper gives TSQR beside CAQR's panel (§2.5, §6).
 *   A, m, n, lda, leaf_h, arity, flags  as tsqr_factor; TSQR_INPLACE is not supported.
 *              n > 128 (up to 4096) runs tsqr_caqr with the default panel width.
 *   prec       TSQR_FP64 only (TSQR_MIXED: TSQR_ERR_UNSUPPORTED).
 *   Q          device, m-by-n column-major, ldq >= m, out. Q may alias A (Q == A and
 *              ldq == lda orthonormalizes the block in place): A is fully read before Q is
 *              written.
 *   R          device n-by-n (ldr >= n), out, or NULL.
 *   Stream-ordered; the factor set's scratch (m-by-n reflectors plus O(leaves * n)
 *   scalars) is freed in stream order at the end of the call.
 *   Errors: as tsqr_factor, plus TSQR_ERR_ARG for null Q or ldq < m.
 */
tsqr_status tsqr_orthonormalize(const double *A, int64_t m, int32_t n, int64_t lda, double *Q,
                                int64_t ldq, double *R, int64_t ldr, int32_t leaf_h, int32_t arity,
                                int32_t prec, int32_t flags, void *stream);

/*
 * tsqr_lstsq — X = argmin ||A X - B||_F column by column: X = R^{-1} (Q^T B)[0:n].
 *   A          device m-by-n (lda >= m), not modified. n > 128 (up to 4096, TSQR_FP64
 *              only; TSQR_MIXED: TSQR_ERR_UNSUPPORTED) is factored by tsqr_caqr with the
 *              default panel width, then Q^T B and the back substitution.
 *   B          device m-by-k (ldb >= m, 1 <= k <= 64), not modified.
 *   X          device n-by-k (ldx >= n), out.
 *   leaf_h, arity, flags as in tsqr_factor (TSQR_INPLACE is ignored).
 *   prec       TSQR_FP64: FP64 TSQR of [A | B] (Q^T B fused into the factorization),
 *              then back substitution.
 *              TSQR_MIXED: the batched engine on one item (see tsqr_batch_item): FP32 leaf
 *              chains of 128-row tiles, the FP64 tree with `arity` (0 = binary), and
 *              corrected semi-normal-equation refinement in FP64 from X = 0 (r = B - A X,
 *              R^T R dX = A^T r), at most max_refine + 1 steps, stopping once the predicted
 *              remaining ||dX||_F/||X||_F is below 1e-10 or the corrections stop
 *              shrinking; leaf_h and flags do not apply. k <= 64, refined in groups of 8.
 *              Synchronizes the stream.
 *   info       host array of length max_refine + 1 or NULL: info[s] = ||dX||_F/||X||_F
 *              of correction s (the largest over the groups of 8 right-hand sides; 0 for
 *              steps not run) for TSQR_MIXED, info[0] = 0 for TSQR_FP64. Filling it
 *              synchronizes the stream.
 *   Errors: TSQR_ERR_ARG, TSQR_ERR_SINGULAR (some r_jj == 0; X is then undefined),
 *           TSQR_ERR_OOM, TSQR_ERR_CUDA. Detecting a singular R synchronizes the
 *           stream.
 */
tsqr_status tsqr_lstsq(const double *A, int64_t m, int32_t n, int64_t lda, const double *B,
                       int64_t ldb, int32_t k, double *X, int64_t ldx, int32_t leaf_h,
                       int32_t arity, int32_t prec, int32_t flags, int32_t max_refine,
                       void *stream, double *info);

/*
 * tsqr_solve_r — X = R^{-1} C[0:n] with F's R (diag(R) >= 0): the back substitution of
 * least squares after tsqr_apply_qt (C = Q^T B, ldc >= n, 1 <= k; X n-by-k, ldx >= n).
 *   status  device int32 or NULL: set to TSQR_ERR_SINGULAR when some r_jj == 0 (X then
 *           holds non-finite values); never cleared by the call.
 *   Errors: TSQR_ERR_ARG (null F/C/X, k < 1, ldc < n, ldx < n), TSQR_ERR_CUDA.
 */
tsqr_status tsqr_solve_r(const tsqr_factors *F, const double *C, int64_t ldc, int32_t k,
                         double *X, int64_t ldx, int32_t *status, void *stream);

/*
 * tsqr_lstsq_static — FP64 least squares X = argmin ||A X - B||_F that allocates
 * nothing. The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory at the point of the call (code in host callbacks, plugins whose
 * framework owns all allocations, applications that reserve the whole device up front
 * and forbid later cudaMalloc/cudaMallocAsync). It computes what tsqr_lstsq computes
 * with prec = TSQR_FP64, leaf_h = the on-chip tile height, arity = 2, TSQR_TWO_LEVEL,
 * but keeps every scratch buffer in one 64 MiB static device array that the library
 * reserves on every GPU that loads it, for the life of the process.
 *   A  device m-by-n (lda >= m), B device m-by-k (ldb >= m), X device n-by-k (ldx >= n);
 *      n >= 1, k >= 1, n + k <= 128. A and B are not modified.
 *   The scratch needed is about 8 * m * (n + k) bytes plus the plan: for n = 64, k = 1
 *   at most about 129,000 rows.
 *   The stream must belong to the current device. The first call on a device looks up the
 *   array's address with that device current. Every call waits for its stream to finish
 *   (it reads back the singularity flag), so no call, the first one included, may be made
 *   on a stream that is being captured into a CUDA graph. All calls share the array and
 *   it keeps the previous call's contents: calls that may overlap on the GPU (several
 *   streams or host threads) race and must be serialized by the caller. A call that
 *   fails after enqueuing work waits for its stream before it returns.
 *   Errors (described by tsqr_last_error): TSQR_ERR_ARG (null pointers, bad sizes or
 *           leading dimensions, a stream of another device), TSQR_ERR_UNSUPPORTED (the
 *           problem needs more scratch than the static array holds; nothing is
 *           enqueued), TSQR_ERR_SINGULAR, TSQR_ERR_CUDA.
 */
tsqr_status tsqr_lstsq_static(const double *A, int64_t m, int32_t n, int64_t lda,
                              const double *B, int64_t ldb, int32_t k, double *X,
                              int64_t ldx, void *stream);

/*
 * tsqr_qr_solve_host — the whole FP64 path on HOST buffers in one stream-ordered call:
 * A (and B) are copied to the device, A is factored by TSQR (paper §2.3), the thin Q
 * (§4, Property 1), R (diag >= 0) and X = R^{-1} (Q^T B)[0:n] are computed (Q^T B and the
 * back substitution on the library's helper stream, beside the thin Q), and Q, R and X are
 * copied back. Device memory comes from the library's stream-ordered pool and is released
 * in stream order. With page-locked (pinned) host buffers every copy is asynchronous:
 * results are valid once `stream` reaches the end of the call; pageable buffers work but
 * the driver stages their copies.
 *   A       host m-by-n (lda >= m), 1 <= n <= 128, m >= n.
 *   B, X    host m-by-k (ldb >= m) and n-by-k (ldx >= n), k >= 1, or both NULL.
 *   Q       host m-by-n (ldq >= m) or NULL.   R  host n-by-n (ldr >= n) or NULL.
 *   status  host int32 or NULL: receives TSQR_ERR_SINGULAR (4) or 0 with the outputs
 *           (valid once the stream reaches the end of the call).
 *   leaf_h, arity, flags  as tsqr_factor (TSQR_TWO_LEVEL | TSQR_CLUSTER).
 *   after   cudaEvent_t or NULL: the call's first kernel waits for it (after the input
 *           copies are enqueued), so consecutive calls on two streams can run their kernels
 *           one after another while each call's copies overlap the other's kernels.
 *   done    cudaEvent_t or NULL: recorded after the call's last kernel, before the output
 *           copies.
 *   Errors: as tsqr_factor, plus TSQR_ERR_ARG for bad B/X/Q/R arguments.
 */
tsqr_status tsqr_qr_solve_host(const double *A, int64_t m, int32_t n, int64_t lda, const double *B, int64_t ldb,
                               int32_t k, double *Q, int64_t ldq, double *R, int64_t ldr, double *X, int64_t ldx,
                               int32_t *status, int32_t leaf_h, int32_t arity, int32_t flags, void *stream,
                               void *after, void *done);

/* tsqr_free — releases F (stream-ordered on the stream F was created on). NULL is
 * accepted. */
tsqr_status tsqr_free(tsqr_factors *F);

/* tsqr_factors_info — host-side description of F: out[0] = m, out[1] = n,
 * out[2] = number of leaves P, out[3] = tile rows, out[4] = number of jobs,
 * out[5] = number of tiles, out[6] = number of kernel launches of a factorization,
 * out[7] = CTAs per SM of the factor kernel. `out` is a host array of 8 int64. */
tsqr_status tsqr_factors_info(const tsqr_factors *F, int64_t *out);

/*
 * tsqr_plan_describe — host only, touches no GPU: the leaf partition and reduction
 * tree tsqr_factor (nc = n) or the fused least-squares factorization (nc = n + k)
 * would build on a device with `sms` SMs and the given shared-memory sizes in bytes
 * (per SM, reserved per block, opt-in maximum per block).
 *   out       host int64[8], as tsqr_factors_info.
 *   tiles     host int64 array of 5*max_tiles or NULL: for tile t in execution order
 *             {row0, rows, kind (0 leaf QR, 1 triangle-on-tile, 2 triangle-on-triangle),
 *             job, launch}.
 *   jobs      host int64 array of 4*max_jobs or NULL: {pivot row, first tile, tiles, launch}.
 * Errors: TSQR_ERR_ARG as tsqr_factor, or when max_tiles / max_jobs is too small while
 * the array is non-NULL (out is filled first so the caller can size the arrays).
 */
tsqr_status tsqr_plan_describe(int64_t m, int32_t n, int32_t nc, int32_t leaf_h, int32_t arity,
                               int32_t flags, int32_t sms, int64_t smem_per_sm,
                               int64_t smem_reserved, int64_t smem_optin, int64_t *out,
                               int64_t *tiles, int64_t max_tiles, int64_t *jobs,
                               int64_t max_jobs);

/*
 * tsqr_plan_clusters — host only, touches no GPU: the cluster schedule tsqr_factor builds
 * with TSQR_CLUSTER (arity 2) for the same arguments as tsqr_plan_describe.
 *   out        host int64[2]: {cluster launches, slots}; 0 slots when the combines do not
 *              fit one CTA's shared memory (the flag is then ignored).
 *   launches   host int32[4 * max_launches] or NULL: {first slot, clusters, first and last
 *              binary tree level (launch index of tsqr_plan_describe) of the launch}.
 *   slots      host int32[3 * max_slots] or NULL, 8 per cluster: {job (index of
 *              tsqr_plan_describe's jobs) or -1, cluster rank of the pivot child, of the
 *              tile child} (-1: a triangle complete before the launch).
 * Errors: as tsqr_plan_describe.
 */
tsqr_status tsqr_plan_clusters(int64_t m, int32_t n, int32_t nc, int32_t leaf_h, int32_t flags, int32_t sms,
                               int64_t smem_per_sm, int64_t smem_reserved, int64_t smem_optin, int64_t *out,
                               int32_t *launches, int64_t max_launches, int32_t *slots, int64_t max_slots);

/*
 * Batched factorization / least squares: many independent problems in ONE persistent
 * kernel launch. Every CTA takes chain jobs (runs of leaves) of any problem from a device
 * queue; when a job finishes, the last child to arrive at a tree node performs that
 * node's combine (the reduce operator of paper §2.3), so tree levels of different
 * problems overlap and no CTA ever waits.
 */
typedef struct tsqr_batch_item {
  const double *A;  /* device, m-by-n column-major, lda >= m; not modified */
  int64_t m;
  int32_t n;        /* 1 <= n <= 128, m >= n */
  int64_t lda;
  const double *B;  /* device, m-by-k (ldb >= m) right-hand sides, or NULL with k = 0;
                       not modified */
  int64_t ldb;
  int32_t k;        /* 0 <= k <= 64; FP64 items: n + k <= 144 */
  double *R;        /* device, n-by-n (ldr >= n) output with diag(R) >= 0, or NULL */
  int64_t ldr;
  double *X;        /* device, n-by-k (ldx >= n) least-squares solution; may be NULL only
                       for FP64 items */
  int64_t ldx;
  int32_t prec;     /* TSQR_FP64: FP64 TSQR of [A | B], X by back substitution.
                       TSQR_MIXED: FP32 leaf chains + FP64 tree for R; with k > 0, X by
                       corrected semi-normal-equation refinement in FP64 from X = 0
                       (r = B - A X, R^T R dX = A^T r), at most 10 steps, stopping once the
                       predicted remaining ||dX||_F/||X||_F is below 1e-10 or the
                       corrections stop shrinking; R-only MIXED items carry FP32 accuracy.
                       TSQR_AUTO: one of the two by a cost model (R-only items: FP64). */
} tsqr_batch_item;

/*
 * tsqr_batch_solve — factor every item (and solve for its right-hand sides) in one launch.
 *   items        host array of count items (device pointers inside).
 *   chain_tiles  tiles per chain (leaves per flat chain inside a CTA); 0 = automatic.
 *   arity        tree arity 2..16 over each item's chains; 0 = automatic (binary).
 *   status       host array of count int32 or NULL: 0, or TSQR_ERR_SINGULAR when the
 *                item's R has an exactly zero diagonal entry (its X is then undefined).
 *                Filling it synchronizes the stream.
 *   info         host array of 2 * count doubles or NULL: for item q, info[2q] = refinement
 *                steps run and info[2q + 1] = the last ||dX||_F / ||X||_F (the largest over
 *                its groups of 8 right-hand sides); both 0 for items solved without
 *                refinement. Filling it synchronizes the stream.
 *   Errors: TSQR_ERR_ARG (invalid item; nothing is enqueued), TSQR_ERR_OOM, TSQR_ERR_CUDA.
 */
tsqr_status tsqr_batch_solve(const tsqr_batch_item *items, int32_t count, int32_t chain_tiles,
                             int32_t arity, void *stream, int32_t *status, double *info);

/*
 * tsqr_batch_describe — host only, touches no GPU and no item data: the job table the
 * batched kernel would run for these items on a device with `sms` SMs and the given
 * shared-memory sizes (as tsqr_plan_describe).
 *   out   host int64[4]: {chain jobs, jobs, tiles, CTAs of the persistent launch}.
 *   jobs  host int64[7 * max_jobs] or NULL, chain jobs first (queue order) then tree nodes:
 *         {item, parent job or -1 at an item's root, children a node waits for, pivot
 *         row, row of its triangle in the tree storage, first tile, tiles}.
 * Errors: TSQR_ERR_ARG (as tsqr_batch_solve, a bad device description, or max_jobs too
 * small while jobs is non-NULL; out is filled first).
 */
tsqr_status tsqr_batch_describe(const tsqr_batch_item *items, int32_t count, int32_t chain_tiles, int32_t arity,
                                int32_t sms, int64_t smem_per_sm, int64_t smem_reserved, int64_t smem_optin,
                                int64_t *out, int64_t *jobs, int64_t max_jobs);

/*
 * Autotuners: each times its candidates on the caller's own data with CUDA events on the
 * caller's stream (which it synchronizes) and returns the fastest. A candidate runs once
 * untimed (planning, memory-pool growth), then twice timed; its time is the faster run.
 *
 * tsqr_batch_autotune(items, count, sample, stream, &chain_tiles, &arity, ms_table)
 *   Runs the first `sample` items (0 = min(count, 1000)) as tsqr_batch_solve does, for
 *   every chain length in {2, 4, 8, 16, 32} and tree arity in {2, 4}, and returns the
 *   fastest pair (pass them to tsqr_batch_solve, tsqr_batch_plan_create or the server).
 *   ms_table: host array of 10 floats or NULL: each pair's time in ms, chain length
 *   outer, arity inner. The timing runs write the sampled items' outputs (the values a
 *   tsqr_batch_solve call writes). Errors: TSQR_ERR_ARG (an invalid item as for
 *   tsqr_batch_solve, count < 1, NULL items or outputs), TSQR_ERR_OOM, TSQR_ERR_CUDA.
 * tsqr_factor_autotune(A, m, n, lda, stream, &leaf_h, &arity, &flags, &best_ms)
 *   Times tsqr_factor (FP64) of A, which is not modified, for leaves of 1, 4 and 16
 *   on-chip tiles, arity 2 and 4, the two-level and the pure tree, plus the flat tree
 *   (arity 0) while A has at most one tile per SM, and returns the fastest leaf_h, arity
 *   and flags (TSQR_TWO_LEVEL or 0); best_ms (may be NULL) receives its time in ms.
 *   Errors: as tsqr_factor; TSQR_ERR_ARG for NULL outputs.
 */
tsqr_status tsqr_batch_autotune(const tsqr_batch_item *items, int32_t count, int32_t sample, void *stream,
                                int32_t *chain_tiles, int32_t *arity, float *ms_table);
tsqr_status tsqr_factor_autotune(const double *A, int64_t m, int32_t n, int64_t lda, void *stream,
                                 int32_t *leaf_h, int32_t *arity, int32_t *flags, float *best_ms);

/*
 * Reusable batch plans: a batch whose items keep their shapes and buffers (an iterative
 * method factoring new data in the same arrays, a benchmark loop) is planned once and
 * replayed as a CUDA graph, so a run costs no host planning and no table uploads.
 *
 * tsqr_batch_plan_create(items, count, chain_tiles, arity, &plan)
 *   Validates the items as tsqr_batch_solve does, plans them, allocates the plan's device
 *   workspace (cudaMalloc, synchronous) and captures one run as a CUDA graph. The item
 *   structs are copied; the device buffers they point to must stay valid while the plan
 *   exists. Errors: TSQR_ERR_ARG, TSQR_ERR_OOM, TSQR_ERR_UNSUPPORTED, TSQR_ERR_CUDA.
 * tsqr_batch_plan_run(plan, stream)
 *   Enqueues one run on stream: reads every item's A (and B) as they are when the run
 *   executes and writes R and X, exactly as tsqr_batch_solve with the same chain_tiles
 *   and arity. Runs of one plan must not overlap (the workspace is the plan's).
 * tsqr_batch_plan_results(plan, status, info)
 *   Waits for the last run and fills status (count int32) and info (2 * count doubles),
 *   as tsqr_batch_solve does; either may be NULL. TSQR_ERR_ARG before the first run.
 * tsqr_batch_plan_destroy(plan)  waits for the last run and frees the plan.
 */
typedef struct tsqr_batch_plan tsqr_batch_plan;
tsqr_status tsqr_batch_plan_create(const tsqr_batch_item *items, int32_t count, int32_t chain_tiles,
                                   int32_t arity, tsqr_batch_plan **plan);
tsqr_status tsqr_batch_plan_run(tsqr_batch_plan *plan, void *stream);
tsqr_status tsqr_batch_plan_results(tsqr_batch_plan *plan, int32_t *status, double *info);
tsqr_status tsqr_batch_plan_destroy(tsqr_batch_plan *plan);

/*
 * Continuous-batching server (the paper has no counterpart; it serves many independent
 * least-squares requests with the batched kernel above). A worker thread owned by the
 * server keeps up to `streams` batches in flight on the current device; whenever a
 * stream is free it admits the oldest pending requests that fit the device-memory budget
 * still free, up to max_batch of them, and runs them as one tsqr_batch_solve launch.
 * Results are bitwise identical to solving the request alone with tsqr_batch_solve and
 * the same chain_tiles (the batched kernel is deterministic per item).
 *
 * tsqr_server_create(max_bytes, max_batch, streams, chain_tiles, ctas_per_sm, &srv)
 *   max_bytes    optional device-memory budget for in-flight requests' workspaces
 *                (bytes); <= 0 = none. Every admission also requires the batch to fit the
 *                device memory free at that moment (cudaMemGetInfo plus the unused reserve
 *                of the library's stream-ordered pool) less 5%. A request larger than
 *                either runs alone once nothing else is in flight.
 *   max_batch    >= 1, requests per launch.   streams  1..16 batches in flight.
 *   chain_tiles  as for tsqr_batch_solve (0 = automatic).
 *   ctas_per_sm  CTAs per SM of the persistent kernel: 0 = as many as fit (2), 1 = one,
 *                leaving room on every SM for the other streams' refinement launches.
 *   Errors: TSQR_ERR_ARG, TSQR_ERR_OOM, TSQR_ERR_CUDA.
 * tsqr_server_submit(srv, item, &ticket)
 *   Validates the item (TSQR_ERR_ARG as tsqr_batch_solve, nothing queued) and queues a
 *   copy of it; the item's device buffers must stay valid, and A/B unmodified, until its
 *   ticket is returned by tsqr_server_poll. Tickets count up from 0 per server.
 * tsqr_server_poll(srv, max, tickets, latency_s, status, &count)
 *   Moves up to max completed requests into the host arrays (any may be NULL):
 *   ticket, seconds from submission to completion, and the item status (0, or
 *   TSQR_ERR_SINGULAR, or the error that made its batch fail). Never blocks.
 * tsqr_server_drain(srv)       blocks until every submitted request has completed.
 * tsqr_server_stats(srv, out)  out[6] (host): submitted, completed, batches launched,
 *                              largest batch, budget bytes (or, without a budget, the free
 *                              device memory seen at the last admission), bytes in flight.
 * tsqr_server_destroy(srv)     finishes every queued request, then frees the server.
 */
typedef struct tsqr_server tsqr_server;
tsqr_status tsqr_server_create(int64_t max_bytes, int32_t max_batch, int32_t streams, int32_t chain_tiles,
                               int32_t ctas_per_sm, tsqr_server **srv);

/*
 * Resident server (the paper has no counterpart): the same requests, admitted into a
 * persistent kernel that is already running. One kernel stays on the GPU and takes work
 * from a ring in device memory; the server's worker thread appends each admitted request
 * to the ring while the kernel runs, so a request starts as soon as its uploads land, not
 * when a launch slot frees up. FP64 and mixed requests both run inside the kernel: the
 * refinement steps of mixed least-squares requests are queued by the kernel itself. The
 * kernel ends after idle_us without work and is launched again when requests arrive.
 * Short requests (at most 8 chain jobs) go to a ring of their own that the kernel serves
 * first, so they do not wait behind the chain jobs of a long request.
 * Results are bitwise those of tsqr_batch_solve on the request alone (same plan, same
 * arithmetic; the compact-WY leaf of tsqr_set_mixed_wy_min_n is not used here).
 *
 * tsqr_server_create_resident(max_bytes, chain_tiles, ctas_per_sm, idle_us, &srv)
 *   max_bytes    device memory reserved at creation for requests in flight (the arena;
 *                admission waits for room in it); <= 0 = a quarter of the memory free now.
 *   chain_tiles  as for tsqr_batch_solve (0 = automatic).
 *   ctas_per_sm  0 or 2: two CTAs per SM; 1: one, with twice the shared memory per CTA
 *                (needed by FP64 requests with n + k above about 100 columns).
 *   idle_us      >= 0, how long the kernel polls for work before it ends (about).
 *   Errors: TSQR_ERR_ARG, TSQR_ERR_OOM (the arena), TSQR_ERR_CUDA.
 * tsqr_server_submit on a resident server also plans the request and returns
 * TSQR_ERR_UNSUPPORTED (nothing queued) when it needs more shared memory per CTA than the
 * kernel has, or more device memory than the arena. tsqr_server_stats: out[2] = launches
 * of the resident kernel, out[3] = most requests in flight at once, out[4] = arena bytes,
 * out[5] = arena bytes in use. poll, drain and destroy are as above. While the kernel
 * runs, a device-wide synchronization (cudaDeviceSynchronize) waits for it to go idle.
 */
tsqr_status tsqr_server_create_resident(int64_t max_bytes, int32_t chain_tiles, int32_t ctas_per_sm,
                                        int32_t idle_us, tsqr_server **srv);

/*
 * tsqr_debug_resident_ring_entries — test hook: both work rings of resident servers created
 * after the call hold `entries` entries (a power of two >= 16; 0 restores the default of
 * 2^20), so that a test can make them wrap around within a few requests. A request with
 * more chain jobs or refinement tasks per step than a ring holds is refused at submission
 * (TSQR_ERR_UNSUPPORTED). Errors: TSQR_ERR_ARG for any other value.
 */
tsqr_status tsqr_debug_resident_ring_entries(int64_t entries);
tsqr_status tsqr_server_submit(tsqr_server *srv, const tsqr_batch_item *item, int64_t *ticket);
tsqr_status tsqr_server_poll(tsqr_server *srv, int32_t max, int64_t *tickets, double *latency_s,
                             int32_t *status, int32_t *count);
tsqr_status tsqr_server_drain(tsqr_server *srv);
tsqr_status tsqr_server_stats(tsqr_server *srv, int64_t *out);
tsqr_status tsqr_server_destroy(tsqr_server *srv);

/*
 * tsqr_set_mixed_wy_min_n — the FP32 leaf chains of mixed-precision items (tsqr_lstsq with
 * TSQR_MIXED, batch items and the launching server's; the resident server always runs the
 * unblocked chains) with at least `min_n` columns (and more than 16)
 * are factored in panels of 16 columns whose 16 reflectors are applied to the trailing
 * columns at once in compact-WY form, I - V T V^T (paper §2.2's blocked Householder
 * update), with V^T C and V (T^T W) on the tensor cores as 3xTF32 products (FP32 operands
 * split into two TF32 parts, FP32 accumulation); narrower items, and every item when
 * min_n = 0, keep the unblocked FP32 register-tile chains. R agrees with the unblocked
 * chains to FP32 rounding; refined solutions meet the same 1e-10. Process-wide, for
 * batches planned after the call; returns the previous value. No error.
 */
int32_t tsqr_set_mixed_wy_min_n(int32_t min_n);

/*
 * tsqr_set_apply_tile_pairs — kernel choice for applying Q^T or Q (tsqr_apply_qt,
 * tsqr_apply_q, the overlapped Q^T B of tsqr_factor_qt and tsqr_lstsq) to ONE column
 * (paper §2.3: the implicit Q is applied tile by tile along each flat chain). With `on`
 * (the default) a launch whose jobs hold several tiles gives each job one warp whose two
 * half-warps run consecutive tiles of the chain one reflector apart; with 0 one warp runs
 * the job's tiles one after the other. The two differ only in summation order (results
 * agree to rounding). Process-wide, for calls made after it; returns the previous value.
 * No error.
 */
int32_t tsqr_set_apply_tile_pairs(int32_t on);

/*
 * tsqr_debug_fail_allocations — failure injection for tests: the next `count` device
 * allocations the library makes fail as if the device were out of memory (the calls
 * return TSQR_ERR_OOM; a server batch whose workspace allocation fails reports
 * TSQR_ERR_OOM for each of its requests and the server goes on serving). 0 clears it.
 * Touches no GPU. No paper counterpart.
 */
tsqr_status tsqr_debug_fail_allocations(int32_t count);

/* launch classes reported by the profiler */
enum {
  TSQR_PROF_FACTOR_CHAINS = 0, /* leaf / flat-chain launch of the factorization */
  TSQR_PROF_FACTOR_TREE = 1,   /* one tree level of the factorization */
  TSQR_PROF_APPLY_QT = 2,
  TSQR_PROF_APPLY_Q = 3,
  TSQR_PROF_FORM_Q = 4,
  TSQR_PROF_SMALL = 5,         /* sign fix, scaling, triangular solve */
  TSQR_PROF_BATCH = 6,         /* the persistent batched kernel */
  TSQR_PROF_REFINE = 7         /* batched least-squares refinement steps */
};

/*
 * tsqr_profile_start / tsqr_profile_stop — opt-in launch timing. Between the two calls
 * every kernel launch the library makes is bracketed by a pair of CUDA events recorded
 * on the launching stream (the events add no synchronization). tsqr_profile_stop waits
 * for the recorded events, writes up to max_records entries (launch class, elapsed ms)
 * into the host arrays kind/ms (either may be NULL to discard), the total number of
 * recorded launches into *count (host, may be NULL), and stops recording.
 */
tsqr_status tsqr_profile_start(void);
tsqr_status tsqr_profile_stop(int64_t max_records, int32_t *kind, float *ms, int64_t *count);

/*
 * tsqr_probe_fp64_peak — measures the device's burst FP64 FMA throughput (TFLOP/s, host
 * *tflops): independent DFMA chains on every SM, best of three timed launches of about
 * 17 ms, and the SM clock that launch ran at (MHz, host *sm_mhz, may be NULL). The FP64
 * kernels' roofline denominator; synchronizes the stream. No paper counterpart.
 */
tsqr_status tsqr_probe_fp64_peak(void *stream, double *tflops, double *sm_mhz);

/*
 * tsqr_probe_dmma_peak — the same measurement for the FP64 tensor cores (DMMA: independent
 * mma.sync m8n8k4 FP64 accumulator chains in every warp of every SM). The evidence for
 * running the FP64 factorization on the FMA pipe: on GB300 the FP64 tensor rate is no
 * higher than the FP64 FMA rate. Synchronizes the stream. No paper counterpart.
 */
tsqr_status tsqr_probe_dmma_peak(void *stream, double *tflops, double *sm_mhz);

/*
 * tsqr_error_word — reads and clears the current device's error word after waiting for
 * `stream`: bit 1 is set when a bounded device-side wait gave up (the TSQR_CLUSTER tree's
 * waits for a child's progress; the results of that launch are then undefined), bit 2
 * when an index check of a build compiled with TSQR_CHECK failed. *word (host) receives
 * the bits. Returns TSQR_ERR_TIMEOUT when bit 1 was set, else TSQR_OK (TSQR_ERR_CUDA on a
 * failed copy). No paper counterpart.
 */
tsqr_status tsqr_error_word(void *stream, int32_t *word);

/* tsqr_strerror — static description of a status code. */
const char *tsqr_strerror(tsqr_status s);

/* tsqr_last_error — host string describing the last error of the calling thread
 * (empty when none). */
const char *tsqr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TSQR_H */
