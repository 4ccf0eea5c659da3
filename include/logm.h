/*
 * logm.h -- C ABI of the GB300 (sm_103a) matrix-logarithm library.
 *
 * Method: inverse scaling and squaring with computation-graph polynomials,
 * Jarlebring, Sastre and Ibanez, "Polynomial approximations for the matrix
 * logarithm with computation graphs" (arXiv 2401.10089), Algorithm 1 (Sec. 6):
 *   log A = 2^s log(A^{1/2^s})                 (Sec. 2.1, eq. matrix_logarithm_identity)
 *   A^{1/2} by the scaled Denman-Beavers iteration  (Sec. 6, eq. ScalDB)
 *   log(I + B) ~= -z(-B), z a degree-optimal graph  (Sec. 3, eqs. Taylor_log,
 *                                                     logipASTM, five_mult_degopt)
 *   s and the number of products k chosen by the backward-error bound
 *   alpha_m <= Theta_m                        (Sec. 5 Table Table_theta; Sec. 6
 *                                               eqs. alphaapprox, AI2, normAm9)
 *   optional balancing T^{-1} A T / T L T^{-1}   (Algorithm 1, Steps 1 and 'Step_Postproc')
 *
 * Conventions shared by every call:
 *  - Matrices are dense, square, row-major. A batch holds `count` matrices.
 *    With n_uniform > 0 matrix b starts at element b * n_uniform^2. With
 *    n_uniform == 0 the sizes and element offsets come from the device arrays
 *    `n` and `offset`, and n_max must bound every n (a matrix whose n lies
 *    outside [1, n_max] is not read and gets LOGM_INFO_BAD_SIZE).
 *  - Pointers named *_dev, and every matrix pointer, are DEVICE pointers that
 *    the caller allocates and owns; the library never allocates, frees or
 *    keeps them after the call returns.
 *  - `ws` is caller-owned device workspace of at least logm_workspace_size()
 *    bytes, 256-byte aligned. It may be reused between calls on one stream.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Every call only
 *    enqueues work on it: no host synchronisation, no allocation.
 *  - Return value: LOGM_SUCCESS, or a negative LOGM_ERR_* for an invalid
 *    argument or a CUDA launch error (nothing is enqueued after an argument
 *    error). Per-matrix outcomes go to the caller's `info_dev[count]`
 *    (LOGM_INFO_*); kernels never trap and every loop is bounded.
 */
#ifndef LOGM_H
#define LOGM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes of every call. */
#define LOGM_SUCCESS 0
#define LOGM_ERR_INVALID_ARG (-1)
#define LOGM_ERR_UNSUPPORTED (-2)
#define LOGM_ERR_WORKSPACE (-3)
#define LOGM_ERR_CUDA (-4)

/* Per-matrix status written to info_dev. */
#define LOGM_INFO_BAD_SIZE (-1)    /* ragged batch: this matrix's n is outside [1, n_max] */
#define LOGM_INFO_OK 0
#define LOGM_INFO_SINGULAR 1       /* exact zero (or non-finite) pivot in a left division */
#define LOGM_INFO_NO_CONVERGENCE 2 /* Denman-Beavers iteration hit max_db_iter */
#define LOGM_INFO_MAX_SQRT 3       /* square-root count hit max_sqrt (maxiter of Algorithm 1) */
#define LOGM_INFO_NONFINITE 4      /* NaN or Inf in the input */
#define LOGM_INFO_TIMEOUT 5        /* a grid barrier of the whole-GPU (large n) kernel timed out; result invalid */
#define LOGM_INFO_BACKWARD_LIMIT 6 /* logm_backward: the forward's levels or iterations exceed what it records */

/* Storage type of A, L, X, Z (arithmetic is FP64 except where `precision` says). */
#define LOGM_DTYPE_F64 0
#define LOGM_DTYPE_F32 1

/* Arithmetic of the graph products (Sec. 3). Square roots, norm estimates and
 * the 2^s scaling are FP64 in every precision. */
#define LOGM_PREC_FP64 0
#define LOGM_PREC_TF32X3 1  /* a = hi + lo in TF32, hi*hi + hi*lo + lo*hi, FP32 accumulation */
#define LOGM_PREC_BF16X3 2  /* a = a0 + a1 + a2 in BF16, the 6 products with i + j <= 2, FP32 accumulation */

typedef struct logm_batch {
  int32_t count;          /* number of matrices, >= 0 */
  int32_t dtype;          /* LOGM_DTYPE_* of A, L, X, Z */
  int32_t n_uniform;      /* > 0: every matrix is n_uniform x n_uniform */
  int32_t n_max;          /* ragged batches: upper bound of n (ignored if n_uniform > 0) */
  const int32_t* n;       /* ragged: device int32[count] of sizes, 1 <= n <= n_max */
  const int64_t* offset;  /* ragged: device int64[count] element offset of each matrix */
} logm_batch;

/* Form of the Denman-Beavers square root (logm_options.db_form). */
#define LOGM_DB_TWO_INVERSE 0 /* eq. (ScalDB): X_k^{-1} and Y_k^{-1} each step */
#define LOGM_DB_PRODUCT 1     /* product form (the variant cited in Sec. 2): M_k = X_k Y_k,
                                 one inversion M_k^{-1} and one product X_k M_k^{-1} per step,
                                 mu_k = |det M_k|^{-1/(2n)}; the same iterates X_k in exact
                                 arithmetic, none of the first step's product */

/* Preprocessing of Algorithm 1, Step 1 (logm_options.balance). */
#define LOGM_BALANCE_NONE 0   /* T = I */
#define LOGM_BALANCE_SCALE 1  /* T diagonal, powers of two (radix-2 Parlett-Reinsch on the
                                 1-norms of the off-diagonal parts of rows and columns);
                                 A <- T^{-1} A T before, L <- T L T^{-1} after, both exact */

/* How the whole-GPU kernel (n > 256) forms the FP64 products of its
 * Gauss-Jordan inversions (logm_options.fp64_products). Not in the paper:
 * an implementation choice for the left divisions of Sec. 6, eq. (ScalDB). */
#define LOGM_FP64_PIPE 0      /* FP64 FMAs (DMMA tiles) */
#define LOGM_FP64_TC_SLICED 1 /* each operand split into eight exact BF16 digits (per-row and
                                 per-column powers of two over up to 128 terms), digit products
                                 accumulated exactly in FP32 on the tensor cores (tcgen05), the
                                 exact integer dot product rounded to FP64 once; the inversions
                                 run as blocked Gauss-Jordan (same pivots, updates outside a
                                 128-column super-panel gathered into one product of 128 terms)
                                 and the graph products this way, everything else as with PIPE */

typedef struct logm_options {
  int32_t k_max;          /* largest number of graph products, 1..6 (Table Table_theta;
                             k = 3 is T_8 by eq. eqP8pol, k = 4 the 14+ scheme of Sec. 3
                             with coefficients solved from T_14, k = 5 Table
                             table_simple_experiment, k = 6 a degree-64 scheme in the same
                             form fitted to -log(1 - x), m_6 = 20+, Theta_6 = 0.372).
                             k_max = 6: FP64 products only (else LOGM_ERR_INVALID_ARG), and
                             n_max <= 256 without a backward context (else
                             LOGM_ERR_UNSUPPORTED); Theta_6 is fixed */
  int32_t precision;      /* LOGM_PREC_* of the graph products */
  int32_t max_sqrt;       /* maxiter of Algorithm 1 (default 40) */
  int32_t max_db_iter;    /* cap on Denman-Beavers iterations per root (default 50) */
  int32_t db_form;        /* LOGM_DB_* (default LOGM_DB_TWO_INVERSE) */
  int32_t balance;        /* LOGM_BALANCE_*, logm_execute / logm_backward only (default NONE) */
  int32_t fp64_products;  /* LOGM_FP64_*, the whole-GPU kernel's inversions (logm_execute,
                             logm_sqrt; default LOGM_FP64_PIPE) */
  int32_t reserved;       /* 0 */
  double theta[5];        /* Theta_{m_k} for k = 1..5; 0 selects
                             the paper's 1.83e-8, 1.53e-4, 1.33e-2, 9.31e-2, 2.46e-1
                             (Table Table_theta) */
} logm_options;

/* Bytes of device workspace the calls below need for this batch and options
 * (the maximum over all calls). Returns 0 for an invalid batch. */
size_t logm_workspace_size(const logm_batch* batch, const logm_options* opts);

/* Bytes of the checkpoint context logm_execute writes for logm_backward
 * (per-level square-root inputs). Returns 0 for an invalid batch. */
size_t logm_context_size(const logm_batch* batch, const logm_options* opts);

/* logm_plan -- the decision of one pass of Algorithm 1's while loop and the
 * order search (Sec. 6, eqs. alphaapprox, normAm9, alpha2term1,
 * normAm9plus1, min_in, min_inp, roughmax_even), at the given A.
 *   A       : device, the current A (F64 or F32 per batch->dtype).
 *   AI2     : device or NULL. NULL means s = 0: finish = ||A - I||_1 <= Theta
 *             first, else the power norms are estimated with A - I. Non-NULL
 *             is A_I2 = (A - I)^2 of eq. (AI2) (same dtype), s >= 1.
 *   finish_dev int32[count]: 1 if alpha_{m_kmax} <= Theta_kmax.
 *   k_dev      int32[count]: products the order search picks (k_max if not finished).
 *   alpha_dev  double[count]: the alpha_{m_kmax} value of the test.
 *   info_dev   int32[count]: LOGM_INFO_OK or LOGM_INFO_NONFINITE. */
int logm_plan(const logm_batch* batch, const logm_options* opts, const void* A,
              const void* AI2, int32_t* finish_dev, int32_t* k_dev, double* alpha_dev,
              int32_t* info_dev, void* ws, size_t ws_bytes, void* stream);

/* logm_sqrt -- one square root A <- A^{1/2} by the scaled Denman-Beavers
 * iteration (Sec. 6, eq. ScalDB; two LU-type left divisions per iteration,
 * mu_k from their determinants; or its product form, opts->db_form), plus
 * A_I2 = A_2 - 2A + I (eq. AI2).
 *   A         : device in/out (dtype per batch). Replaced by its square root.
 *   A2_out    : device or NULL; receives the input A (the A_2 of Algorithm 1).
 *   AI2_out   : device or NULL; receives (A^{1/2} - I)^2 = A_2 - 2 A^{1/2} + I.
 *   active_dev: device int32[count] or NULL; matrices with 0 are left as they are.
 *   iters_dev : device int32[count] or NULL; Denman-Beavers iterations taken.
 *   info_dev  : int32[count]; LOGM_INFO_OK / SINGULAR / NO_CONVERGENCE / NONFINITE. */
int logm_sqrt(const logm_batch* batch, const logm_options* opts, void* A, void* A2_out,
              void* AI2_out, const int32_t* active_dev, int32_t* iters_dev, int32_t* info_dev,
              void* ws, size_t ws_bytes, void* stream);

/* logm_graph_eval -- Z = z(X) with the degree-optimal graph of k products
 * (Sec. 3, eq. five_mult_degopt): P_1 = I, P_2 = X, P_3 = X^2 and
 * P_{j+2} = (sum_i h_{j,i} P_i)(sum_i g_{j,i} P_i), z = sum_i y_i P_i, with
 * Table table_simple_experiment for k = 5, exact Taylor T_2, T_4 (eq.
 * Taylor_log) for k = 1, 2, T_8 with three products (eq. eqP8pol, its
 * coefficients solved in closed form) for k = 3 and the 14+ scheme (degree
 * 16, T_14 matched, coefficients solved numerically) for k = 4; with FP64
 * products and n <= 256 also k = 6 (degree 64, coefficients fitted to
 * -log(1 - x), Taylor terms matched to order 34).
 *   X    : device (dtype per batch).
 *   P3   : device or NULL; X^2 if the caller has it (saves one product, as
 *          Algorithm 1 does with A_I2 when s >= 1).
 *   k_dev: device int32[count], each 1..5; also 6 with FP64 products on
 *          matrices with n <= 256 (Z of a matrix with another k is left
 *          unwritten).
 *   Z    : device output (dtype per batch).
 *   precision: LOGM_PREC_* for the products. */
int logm_graph_eval(const logm_batch* batch, int32_t precision, const void* X, const void* P3,
                    const int32_t* k_dev, void* Z, void* ws, size_t ws_bytes, void* stream);

/* logm_execute -- L = log(A) by Algorithm 1 (balancing T per opts->balance;
 * diag(T) goes to ctx when given, else to the workspace).
 *   A      : device input, untouched.   L : device output (dtype per batch).
 *   s_dev, k_dev : device int32[count] or NULL; square roots and products used.
 *   info_dev     : device int32[count].
 *   stats_dev    : device int32[4 * count] or NULL; per matrix the work done:
 *                  Denman-Beavers iterations, n x n inverses (left divisions),
 *                  n x n graph products, estimator matrix-vector products.
 *   ctx    : device buffer of logm_context_size() bytes or NULL. When given,
 *            the inputs of every square-root level and the plan are saved for
 *            logm_backward. */
int logm_execute(const logm_batch* batch, const logm_options* opts, const void* A, void* L,
                 int32_t* s_dev, int32_t* k_dev, int32_t* info_dev, int32_t* stats_dev, void* ctx,
                 void* ws, size_t ws_bytes, void* stream);

/* Bytes of device workspace logm_backward needs (one slot per resident block
 * of 49 n_max^2 doubles: forward recompute, adjoints and the recorded
 * inverses of up to 16 Denman-Beavers iterations). Returns 0 for an invalid
 * batch or n_max > 256. */
size_t logm_backward_workspace_size(const logm_batch* batch, const logm_options* opts);

/* logm_backward -- dA = adjoint of the computed map A -> L at the forward's
 * plan, applied to dL (i.e. the gradient of sum(dL o L) with respect to A):
 * the graph products (Sec. 3, eq. five_mult_degopt) and the Denman-Beavers
 * iterations (eq. ScalDB) of every level are reversed; the iterates of a level
 * are recomputed from the level's input, which logm_execute checkpointed in
 * ctx. The plan (s, k) and the scalings mu_k are held fixed (they do not
 * change the converged root). With balancing, the adjoint of L = T z T^{-1},
 * B = T^{-1} A T is applied with the forward's T (saved in ctx); opts must be
 * the forward's. The levels are always recomputed with eq. (ScalDB): after a
 * forward in the product form the recomputed roots equal the forward's to
 * rounding.
 *   A   : the forward's input.  ctx: the forward's context (logm_context_size
 *         bytes, filled by logm_execute).  dL, dA: device, dtype per batch.
 *   ws  : logm_backward_workspace_size bytes.  n_max <= 256.
 *   info_dev: 0, 1 (the forward had no result), 6 (a level needed more than 16
 *         Denman-Beavers iterations or s exceeded the 12 checkpointed levels). */
int logm_backward(const logm_batch* batch, const logm_options* opts, const void* A,
                  const void* ctx, const void* dL, void* dA, int32_t* info_dev, void* ws,
                  size_t ws_bytes, void* stream);

/* logm_execute_noalloc -- logm_execute for callers that cannot allocate
 * device memory (no counterpart in the paper: it exists for callers such as
 * code running under a host framework that owns every device allocation, or
 * real-time code with a fixed device-memory budget). The caller still passes
 * A, L and the per-matrix outputs; the scratch space lives in a file-scope
 * device array of 32 MiB that every GPU loading the library keeps until the
 * process exits. The call runs as many matrices at a time as that array
 * holds (7 n_max^2 doubles each), FP64 precision only, n_max <= 256, no
 * balancing; larger n_max, another precision or balancing return
 * LOGM_ERR_UNSUPPORTED. It calls no cudaMalloc, cudaFree or other allocating
 * routine. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * Every call shares the one array and leaves its contents behind: calls whose
 * work overlaps on the GPU (different streams, or different host threads on
 * one device) race on it and must be serialised by the caller.
 *   Arguments as logm_execute, without stats, ctx and workspace. */
int logm_execute_noalloc(const logm_batch* batch, const logm_options* opts, const void* A, void* L,
                         int32_t* s_dev, int32_t* k_dev, int32_t* info_dev, void* stream);

/* logm_execute_host -- logm_execute on HOST buffers, for callers whose data
 * lives in host memory: copies A to the device, runs logm_execute and copies
 * L, s, k and info back, all enqueued on `stream` (one cudaMemcpyAsync per
 * buffer; the results are in the host buffers once the stream has finished).
 * Uniform batches only (n_uniform > 0; a ragged batch returns
 * LOGM_ERR_UNSUPPORTED). Host buffers should be page-locked for the copies to
 * be asynchronous; pageable memory works but the copies then block the host.
 *   A_host   : host, count * n^2 elements of the batch dtype, row-major.
 *   L_host   : host, same size; s_host, k_host (may be NULL), info_host: host int32[count].
 *   ws       : device, >= logm_host_workspace_size() bytes, 256-byte aligned:
 *              the workspace of logm_execute, then device copies of A and L
 *              and the three int32 arrays.
 * Returns as logm_execute, or LOGM_ERR_CUDA if a copy cannot be enqueued. */
size_t logm_host_workspace_size(const logm_batch* batch, const logm_options* opts);
int logm_execute_host(const logm_batch* batch, const logm_options* opts, const void* A_host, void* L_host,
                      int32_t* s_host, int32_t* k_host, int32_t* info_host, void* ws, size_t ws_bytes,
                      void* stream);

/* Per-size-bucket choice of the one-block-per-matrix kernel configuration
 * used by logm_execute (batching form). Buckets: n <= 8, 16, 32, 64, 128, 256.
 * Variants: 0 = 256-thread blocks, 64 x 64 DMMA tiles, any n <= 256;
 *           1 = 128-thread blocks, 32 x 32 tiles, n <= 64 (buckets 0-3);
 *           2 = 64-thread blocks, 32 x 32 tiles, n <= 32 (buckets 0-2);
 *           3 = 256-thread blocks as 0, three per SM (registers capped), any n <= 256;
 *           4 = 64-thread blocks as 2 (buckets 0-2) with the working matrices in the
 *               block's shared memory instead of an L2-resident workspace slot
 *               (execute only; as many blocks per SM as fit).
 * Smaller configurations keep more small matrices in flight per SM; a
 * uniform batch that variant 1 would run in two rounds of five blocks per SM
 * but that fits one round of seven runs on its 7-per-SM build instead. The
 * project's autotuner (paper_2401_10089_gb300.autotune) times the candidates
 * on a sample of each bucket and writes the table it picks to JSON. */
typedef struct logm_tuning {
  int32_t variant[6];
} logm_tuning;

/* Set the process-wide table (NULL restores all-0). Returns LOGM_SUCCESS, or
 * LOGM_ERR_INVALID_ARG for a variant a bucket cannot use. Not thread-safe
 * against concurrent logm_execute calls. */
int logm_set_tuning(const logm_tuning* t);

/* Copy the current table to *t. */
int logm_get_tuning(logm_tuning* t);

/* Library version (major * 10000 + minor * 100 + patch). */
int logm_version(void);

/* logm_probe_barrier -- self-test of the bound on the whole-GPU kernel's grid
 * barrier (the only spin-wait in the library). Two co-resident blocks (one
 * cooperative launch) wait at a barrier that expects 2 + missing arrivals, so
 * with missing > 0 it never completes: each block gives up after timeout_s
 * seconds and the status word becomes 1 (in logm_execute that is
 * LOGM_INFO_TIMEOUT); with missing = 0 both arrive and it stays 0.
 *   missing   : 0..8 arrivals that never come.
 *   timeout_s : 1e-6 .. 60 seconds.
 *   ws        : device, >= 16 bytes, 8-byte aligned, owned by the caller:
 *               [0, 8) the arrival counter, [8, 12) int32 status written by the
 *               kernel (read it after the stream has finished).
 * Returns LOGM_SUCCESS, LOGM_ERR_INVALID_ARG, LOGM_ERR_WORKSPACE or
 * LOGM_ERR_CUDA (launch failure). Does not synchronise the host. */
int logm_probe_barrier(int32_t missing, double timeout_s, void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif
