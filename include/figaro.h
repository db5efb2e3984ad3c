/*
 * figaro.h -- C ABI of the GB300 (sm_103a) Figaro two-table library.
 *
 * Computes, for two tables A (m1 x n1, int32 key per row) and B (m2 x n2,
 * int32 key per row), the upper-triangular R of QR(J) and the singular values
 * of J, where J is the natural (inner) join of A and B: one row [A_i, B_j] for
 * every pair of rows with equal keys ("Figaro on GPUs: Two Tables",
 * arXiv 2503.23385, Section 1: the Cartesian product, the QR head / QR tail
 * operators and Claim 1; Section 3: singular values of J as those of R).
 * J is never formed.  The path is: stable radix sort of each table by key,
 * runs and matched keys, the per-key-group QR head and QR tail rows of
 * Claim 1 (weighted by sqrt(m2g) on A's side and sqrt(m1g) on B's side), a
 * CholeskyQR2 of that reduced matrix, and a one-sided Jacobi SVD of R (or,
 * with FIGARO_FLAG_SIGMA_DQDS, bidiagonalisation of R and dqds).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Layout: features are row-major with a leading dimension `ld` >= n
 *    (elements).  R is n x n row-major (n = n1 + n2) with leading dimension
 *    `ldr` >= n, columns ordered [A's n1 | B's n2] as in Section 1, lower
 *    triangle written as zeros, rows scaled so the diagonal is >= 0.
 *    sigma has n entries, descending; rank-deficient joins give zeros.
 *  - Memory: every pointer is a device pointer unless the table's `memory`
 *    field (inputs) or FIGARO_FLAG_HOST_OUTPUT (outputs) says host.  Host
 *    inputs are staged through the workspace with stream-ordered copies;
 *    pinned host memory keeps those copies asynchronous.
 *  - Ownership: the caller owns inputs, outputs and the workspace.  The
 *    library never allocates device memory in these calls and never frees
 *    caller memory.  Query the workspace size first.
 *  - Ordering: calls enqueue work on `stream` (a cudaStream_t; NULL = the
 *    legacy default stream) and return without waiting.  Argument errors are
 *    returned at once.  Errors found on the device (numerical breakdown, a
 *    bounded wait that ran out) are recorded in the workspace; read them with
 *    figaro_get_status() after the stream has reached that point.
 *  - Limits: m1, m2 < 2^31; 1 <= n1, n2 and n1 + n2 <= 512, and each table
 *    at most 256 columns when n1 + n2 > 128 (other widths return
 *    FIGARO_ERR_UNSUPPORTED); both tables have the same dtype.  Up to 128
 *    columns the n x n steps run in one CTA each; wider joins take the
 *    multi-CTA path (Q = X W written to the workspace, cooperative launches
 *    for the Cholesky factorisations and the Jacobi SVD).
 *  - Workspace must be 256-byte aligned.  Concurrent calls need distinct
 *    workspaces.
 */
#ifndef FIGARO_H_
#define FIGARO_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FIGARO_API __attribute__((visibility("default")))
#else
#define FIGARO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum figaro_status {
  FIGARO_OK = 0,
  FIGARO_ERR_INVALID_ARG = 1,          /* null pointer, bad size, bad enum, mismatched dtypes */
  FIGARO_ERR_WORKSPACE_TOO_SMALL = 2,  /* ws_bytes below figaro_workspace_size() */
  FIGARO_ERR_CUDA = 3,                 /* a CUDA launch or copy failed */
  FIGARO_ERR_NOT_SPD = 4,              /* Cholesky met a non-finite pivot (NaN/Inf in the input) */
  FIGARO_ERR_NO_CONVERGENCE = 5,       /* Jacobi reached max sweeps; sigma is still written */
  FIGARO_ERR_DEVICE_TIMEOUT = 6,       /* a bounded device-side wait gave up; results are invalid */
  FIGARO_ERR_UNSUPPORTED = 7,          /* width or size outside the limits above */
  /* A factorisation found a column with a non-zero norm numerically dependent
   * on the columns before it (pivot below rank_tol times its diagonal): the
   * join is rank-deficient, or too ill-conditioned for the path (on the mixed
   * path a condition number of a few hundred along some direction suffices).
   * R (with a zero row there) and sigma are still written, and
   * figaro_info.dependent_columns counts the zero rows.  Rerun with
   * FIGARO_PATH_FP64 or FIGARO_FLAG_SHIFTED_CHOLQR3 for an ill-conditioned
   * full-rank join; set FIGARO_FLAG_ALLOW_RANK_DEFICIENT to accept the
   * zero rows (a rank-deficient join) without this status.                */
  FIGARO_ERR_RANK_DEFICIENT = 8
} figaro_status;

typedef enum figaro_dtype { FIGARO_F32 = 0, FIGARO_F64 = 1 } figaro_dtype;

/* FIGARO_PATH_FP64: every step in FP64 (the plain reference form).
 * FIGARO_PATH_MIXED: head/tail in FP32 with compensated (float-float) group
 * sums; Gram products on the tensor cores in 3xTF32 (split operands) with
 * FP32 accumulation drained into float-float or FP64 partial sums; the two
 * n x n Cholesky factorisations, the triangular inverse and the Jacobi
 * sweeps in FP32; the assembly in extended precision: the inverse refined
 * by one Newton step and R = R2 R1 formed in float-float (n <= 32) or FP64,
 * and each singular value an extended-precision Rayleigh quotient
 * ||R v_j|| / ||v_j|| (the FP32 column norm below 1e-3 sigma_max).  Its
 * error against the FP64 oracle is about 2e-7 (R and sigma, relative
 * Frobenius) on well-conditioned joins; per singular value it grows with
 * sigma_max / sigma_j.                                                       */
typedef enum figaro_path { FIGARO_PATH_FP64 = 0, FIGARO_PATH_MIXED = 1 } figaro_path;

typedef enum figaro_memory { FIGARO_MEM_DEVICE = 0, FIGARO_MEM_HOST = 1 } figaro_memory;

/* Gram engine for the reduced-matrix products.                               */
typedef enum figaro_gram_engine {
  FIGARO_GRAM_AUTO = 0,     /* chosen per width by the library */
  FIGARO_GRAM_SIMT = 1,     /* CUDA-core FMA */
  FIGARO_GRAM_TCGEN05 = 2   /* 5th-generation tensor cores (mixed path only) */
} figaro_gram_engine;

enum {
  FIGARO_FLAG_HOST_OUTPUT = 1,     /* R / sigma pointers are host memory */
  /* Fault injection for tests (mixed path, tensor-core Gram of widths 4, 8,
   * 16 or 32): the Gram's producer never loads its first tile, so the
   * workers' bounded wait runs out (after about spin_limit / 16 suspended
   * polls) and the call records FIGARO_ERR_DEVICE_TIMEOUT. */
  FIGARO_FLAG_TEST_WITHHOLD = 1 << 8,
  /* figaro_batch_join: when the batch's shape class has no tuned schedule
   * yet, time the candidate schedules on this batch first (the call then
   * waits for the stream; it must not be made during stream capture, where
   * the flag is ignored) and keep the fastest for later calls. */
  FIGARO_FLAG_AUTOTUNE = 1 << 2,
  /* Dependent columns (zero rows of R) are accepted silently: the call does
   * not report FIGARO_ERR_RANK_DEFICIENT (figaro_info still counts them). */
  FIGARO_FLAG_ALLOW_RANK_DEFICIENT = 1 << 3,
  /* Shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa,
   * SIAM J. Sci. Comput. 42 (2020)) in place of CholeskyQR2: the first
   * factorisation is of G1 + s I (s = 10 n u trace(G1), u = 2^-24 on the
   * mixed path and 2^-53 on the FP64 path, on the non-zero diagonal), which
   * succeeds for ill-conditioned joins, and a third Gram pass follows.  It
   * costs one more pass over the reduced matrix.  Measured: the FP64 path
   * factors a join of condition number 1.2e8 (where its CholeskyQR2 reports
   * a dependent column) with R within 4e-15 and every singular value within
   * 2e-10 of Householder QR; the mixed path reaches its 1e-6 bar up to
   * condition 1e5 (its CholeskyQR2 up to 1e3) and reports joins beyond that,
   * whose small directions its FP32 data cannot resolve.  Single calls only:
   * figaro_batch_join runs such instances one after another.               */
  FIGARO_FLAG_SHIFTED_CHOLQR3 = 1 << 4,
  /* Each table's rows are already in ascending key order (non-decreasing
   * int32 keys; Section 2 of the paper assumes such inputs).  The radix sort
   * is skipped: the permutation is the identity and the keys are the sorted
   * keys.  Within a key the rows keep their order, as after the stable sort.
   * A table that is not in order makes the call's device status
   * FIGARO_ERR_INVALID_ARG (results invalid).  Single calls only:
   * figaro_batch_join runs such instances one after another.              */
  FIGARO_FLAG_PRESORTED = 1 << 5,
  /* figaro_join_singular_values and figaro_batch_join: sigma from R by
   * Householder bidiagonalisation and dqds (Section 3 names this
   * square-root-free method for the case where only the singular values are
   * wanted; see figaro_triangular_singular_values) instead of one-sided
   * Jacobi.  Up to 128 columns the FP64 path bidiagonalises in FP64 and runs
   * dqds in float-float, the mixed path runs both in FP32 (normwise error of
   * order 2^-24 ||R||, no per-value relative accuracy for graded spectra);
   * wider joins (up to 512) take the FP64 / float-float form in one CTA on
   * either path, much slower than the block Jacobi.  Householder
   * bidiagonalisation keeps the values to absolute accuracy (of order
   * n u ||R||), not to the relative accuracy one-sided Jacobi reaches on
   * column-graded R.  figaro_join_svd, which needs the rotations, returns
   * FIGARO_ERR_UNSUPPORTED with it.  figaro_info.jacobi_sweeps then counts
   * dqds transforms; FIGARO_ERR_NO_CONVERGENCE means dqds ran out of
   * transforms (30 n + 64) and sigma holds its current estimates.           */
  FIGARO_FLAG_SIGMA_DQDS = 1 << 6
};

typedef struct figaro_table {
  const void* x;       /* features: m rows, row-major, leading dimension ld */
  const int32_t* key;  /* m join keys */
  int64_t m;           /* rows (0 allowed) */
  int64_t ld;          /* leading dimension in elements, >= n */
  int32_t n;           /* feature columns, >= 1 */
  int32_t dtype;       /* figaro_dtype */
  int32_t memory;      /* figaro_memory of x and key */
  int32_t reserved;
} figaro_table;

/* Phase boundaries recorded into figaro_options.phase_events (tracing):
 * start, grouping done, head/tail A done, head/tail B done, Gram pass 1 done,
 * Cholesky 1 done, Gram pass 2 done, Cholesky 2 done, Jacobi done.         */
#define FIGARO_NUM_PHASE_EVENTS 9

typedef struct figaro_options {
  int32_t path;               /* figaro_path */
  int32_t gram_engine;        /* figaro_gram_engine */
  int32_t max_jacobi_sweeps;  /* 0 = library default (40) */
  int32_t flags;              /* FIGARO_FLAG_* */
  int64_t spin_limit;         /* polls per bounded device wait; 0 = default (about a second) */
  double rank_tol;            /* relative pivot below which a column counts as dependent; 0 = default */
  void* const* phase_events;  /* NULL, or FIGARO_NUM_PHASE_EVENTS cudaEvent_t recorded on the stream
                                 at the phase boundaries (single-instance calls only) */
} figaro_options;

/* Fills `opt` with the defaults (mixed path, automatic Gram engine). */
FIGARO_API figaro_status figaro_default_options(figaro_options* opt);

/* Bytes of workspace one call needs for these shapes and options. */
FIGARO_API figaro_status figaro_workspace_size(const figaro_table* A, const figaro_table* B, const figaro_options* opt,
                                    size_t* bytes);

/*
 * figaro_join_group -- the key grouping of both tables (Section 2 assumes
 * inputs sorted by the join attribute; this call produces that order).
 * Per table, into caller device buffers (m = that table's rows):
 *   perm[m]          input row of the i-th row in key order (stable: equal
 *                    keys keep their input order)
 *   sorted_key[m]    key of the i-th row in key order
 *   run_key[m]       distinct keys ascending (first num_runs entries valid)
 *   run_offset[m+1]  start of each run in key order, run_offset[num_runs] = m
 *   other_count[m]   rows with the same key in the other table (0 = the key
 *                    has no partner and contributes no join rows)
 *   num_runs[1]      (int64) number of runs
 * num_groups (device int64[1], may be NULL): keys present in both tables.
 * All outputs are exact integers (bit-exact against a stable sort).
 */
typedef struct figaro_grouping {
  int32_t* perm;
  int32_t* sorted_key;
  int32_t* run_key;
  int32_t* run_offset;
  int32_t* other_count;
  int64_t* num_runs;
} figaro_grouping;

FIGARO_API figaro_status figaro_join_group(const figaro_table* A, const figaro_table* B, const figaro_options* opt,
                                const figaro_grouping* outA, const figaro_grouping* outB, int64_t* num_groups,
                                void* ws, size_t ws_bytes, void* stream);

/*
 * figaro_join_head_tail -- the reduced matrix of Claim 1 (Section 1), one
 * slot per row so that no compaction pass is needed:
 *   head   [m1 x (n1+n2)]  row u (u < number of runs of A, in key order):
 *                          [sqrt(m2g) H(A_g), sqrt(m1g) H(B_g)] for the key
 *                          group g of that run, zero if the key has no
 *                          partner in B.
 *   tail_a [m1 x n1]       row i (i-th row of A in key order, local index
 *                          j >= 1 inside its run): sqrt(m2g) T(A_g)_j; zero
 *                          for the first row of each run and for runs
 *                          without a partner.
 *   tail_b [m2 x n2]       the same for B with weight sqrt(m1g).
 * H(X) = (1/sqrt m) sum_k X_k;  T(X)_j = (sqrt(j) X_{j+1} - S_j/sqrt(j)) /
 * sqrt(j+1) with S_j the sum of the first j rows.  Element type: double for
 * FIGARO_PATH_FP64, float for FIGARO_PATH_MIXED.  Dense, leading dimension
 * equal to the width.  The Gram matrix of all these rows equals J^T J.
 */
FIGARO_API figaro_status figaro_join_head_tail(const figaro_table* A, const figaro_table* B, const figaro_options* opt,
                                    void* head, void* tail_a, void* tail_b, void* ws, size_t ws_bytes,
                                    void* stream);

/*
 * figaro_join_qr_r -- R of QR(J) (Section 1: R with R^T R = J^T J), by a
 * CholeskyQR2 of the reduced matrix (CholeskyQR3 with
 * FIGARO_FLAG_SHIFTED_CHOLQR3).  Dependent columns (a short or rank-deficient
 * join) get zero rows in R, and the call's device status is then
 * FIGARO_ERR_RANK_DEFICIENT unless FIGARO_FLAG_ALLOW_RANK_DEFICIENT is set;
 * a column that is zero in J gets a zero row without that status.
 */
FIGARO_API figaro_status figaro_join_qr_r(const figaro_table* A, const figaro_table* B, const figaro_options* opt, double* R,
                               int64_t ldr, void* ws, size_t ws_bytes, void* stream);

/*
 * figaro_join_singular_values -- sigma(J) = sigma(R) (Section 3), with R
 * computed as in figaro_join_qr_r and written to R_out when R_out != NULL.
 */
FIGARO_API figaro_status figaro_join_singular_values(const figaro_table* A, const figaro_table* B, const figaro_options* opt,
                                          double* sigma, double* R_out, int64_t ldr, void* ws, size_t ws_bytes,
                                          void* stream);

/*
 * figaro_triangular_singular_values -- singular values of `count` upper
 * triangular n x n matrices (Section 3: sigma(J) = sigma(R); the method is
 * the one the section names for singular values alone, the square-root-free
 * dqds of Rutishauser in the differential form of Fernando and Parlett).
 * Matrix b is R + b * stride (device, FP64, row-major with leading dimension
 * ldr >= n; only the upper triangle is read, so the lower one may hold
 * anything).  Each is reduced to upper bidiagonal form by Householder
 * reflections from both sides in FP64 (backward error of order eps ||R||),
 * then dqds with shifts finds the squares of the bidiagonal's singular
 * values to high relative accuracy.  sigma + b * n (device) receives the
 * n values, descending; info (device, may be NULL) receives per matrix the
 * number of dqds transforms, or -1 when dqds stopped after 30 n + 64
 * transforms (sigma then holds its current estimates; NaN when the matrix
 * holds NaN or Inf).  1 <= n <= 128 (else FIGARO_ERR_UNSUPPORTED for
 * n > 128, FIGARO_ERR_INVALID_ARG for n < 1); stride >= 0; count >= 0
 * (0 enqueues nothing).  One CTA per matrix, enqueued on `stream`; needs
 * no workspace.  The device is the one that holds R.
 */
FIGARO_API figaro_status figaro_triangular_singular_values(const double* R, int64_t ldr, int64_t stride, int32_t n,
                                                int32_t count, double* sigma, int32_t* info, void* stream);

/*
 * figaro_join_svd -- singular values and right singular vectors of J
 * (Section 1's applications: the SVD of J for its principal components;
 * Section 3: J = Q R, so J and R share sigma and V).  sigma[n] (device,
 * descending) as in figaro_join_singular_values; V (device, n x n
 * row-major, leading dimension ldv >= n): column j is the unit right
 * singular vector of sigma_j, with the sign that makes its largest-magnitude
 * component positive (the principal axes of J, which is not centred).
 * Computed by one-sided Jacobi on R with the rotations accumulated (FP32
 * sweeps and FP64 Rayleigh quotients on the mixed path, so V is accurate to
 * FP32 level there; FP64 on the plain path); for repeated singular values
 * any orthonormal basis of their subspace is returned.  R_out (may be NULL)
 * receives R as in figaro_join_qr_r.  Device outputs only
 * (FIGARO_FLAG_HOST_OUTPUT returns FIGARO_ERR_UNSUPPORTED).
 */
FIGARO_API figaro_status figaro_join_svd(const figaro_table* A, const figaro_table* B, const figaro_options* opt,
                              double* sigma, double* V, int64_t ldv, double* R_out, int64_t ldr, void* ws,
                              size_t ws_bytes, void* stream);

/*
 * figaro_join_least_squares -- least squares over the join (Section 1's
 * applications: the closed-form solution of linear regression).  The label
 * y is B's last column, so J = [J_x | y] with J_x = the n - 1 other columns
 * ([A's n1 | B's first n2 - 1]).  From R = [[R11, r], [0, rho]] of QR(J)
 * (the same path as figaro_join_qr_r): beta = R11^{-1} r, which minimises
 * ||J_x beta - y||_2, written to beta[n - 1] (device, FP64), and the
 * residual norm |rho| = min ||J_x beta - y||_2 to residual[1].  A feature
 * column that depends on the others (zero row of R) gets beta_i = 0.
 * Requires n1 + n2 >= 2.  FIGARO_FLAG_HOST_OUTPUT makes beta and residual
 * host pointers.
 */
FIGARO_API figaro_status figaro_join_least_squares(const figaro_table* A, const figaro_table* B,
                                        const figaro_options* opt, double* beta, double* residual, void* ws,
                                        size_t ws_bytes, void* stream);

/*
 * figaro_join_singular_values_fixed -- figaro_join_singular_values with
 * scratch owned by the library instead of a caller-supplied workspace.  The
 * paper has no counterpart: this is a convenience of this library for
 * callers that cannot allocate device memory where they call it, e.g. a
 * plugin whose host framework owns and budgets all device memory, or a
 * latency-bound loop that must not pay cudaMalloc's implicit device-wide
 * synchronisation.  The call itself allocates nothing.
 *
 * The scratch is one fixed array of FIGARO_FIXED_SCRATCH_BYTES per device,
 * reserved when the library's device code is loaded on that device.  An
 * input pair whose figaro_workspace_size exceeds it is rejected with
 * FIGARO_ERR_WORKSPACE_TOO_SMALL before any device work is enqueued.  That
 * size depends on the device's SM count (per-SM partial sums): on a 152-SM
 * GB300 the limit is about 1.4e5 + 1.4e5 rows at 8 + 8 FP32 columns and
 * 7.9e4 + 7.9e4 rows at 16 + 16.
 * Arguments, layouts and outputs are those of figaro_join_singular_values;
 * the device is the one that holds the first non-empty device-resident
 * table, else the current device.  Every call looks up the scratch's address
 * in the current context (a host-side query that allocates nothing; not
 * cached, so a cudaDeviceReset or another context is followed correctly).
 * The first call on a device may load the library's device code there:
 * make it outside any stream capture.  Nothing in the scratch needs to start at
 * zero: every call clears the counters and flags it uses before using them.
 * Calls share the one array, so two calls in flight on the same device at
 * the same time race (wrong results or FIGARO_ERR_DEVICE_TIMEOUT): order
 * them on one stream.  *scratch_out (when scratch_out != NULL) receives the
 * scratch's device address, which figaro_get_status / figaro_get_info accept
 * as `ws` to read the device status of the last call.
 */
#define FIGARO_FIXED_SCRATCH_BYTES ((size_t)32 << 20)

FIGARO_API figaro_status figaro_join_singular_values_fixed(const figaro_table* A, const figaro_table* B,
                                                const figaro_options* opt, double* sigma, double* R_out,
                                                int64_t ldr, void** scratch_out, void* stream);

/*
 * Batched form: `count` independent instances (A[i], B[i]) with their own
 * shapes, each writing R[i] (n_i x n_i, leading dimension n_i) and sigma[i].
 * R and sigma are host arrays of `count` device pointers (entries may be
 * NULL to skip an output; an instance with neither is skipped).  One
 * workspace covers the whole batch: its front holds the instances' plans and
 * job lists, the rest one workspace per instance.
 *
 * Instances with n_i <= 128, device-resident tables and device outputs run
 * together, one launch per phase for the whole batch (grouping, head/tail,
 * each Gram pass, each dense step), the Gram products on CUDA cores; the
 * plans reach the device as kernel arguments, so the call can be captured in
 * a CUDA graph and replayed.  Other instances (wider joins, host memory) run
 * one after another in the same call.  figaro_options.phase_events, when
 * set, is recorded around the batched phases.  Device-side status is
 * recorded per instance, in that instance's part of the workspace.
 */
FIGARO_API figaro_status figaro_batch_workspace_size(int32_t count, const figaro_table* A, const figaro_table* B,
                                          const figaro_options* opt, size_t* bytes);

FIGARO_API figaro_status figaro_batch_join(int32_t count, const figaro_table* A, const figaro_table* B,
                                const figaro_options* opt, double* const* R, double* const* sigma, void* ws,
                                size_t ws_bytes, void* stream);

/* The schedule figaro_batch_join uses for these shapes and options: rows of
 * a Gram block per CTA and the head/tail CTA budget per SM, as tuned by an
 * earlier FIGARO_FLAG_AUTOTUNE call of the same shape class (instances,
 * path, and the batch's input rows and summed widths rounded down to powers
 * of two), else the defaults (4096 rows, 2 CTAs per SM).  Host only.        */
FIGARO_API figaro_status figaro_batch_schedule(int32_t count, const figaro_table* A, const figaro_table* B,
                                    const figaro_options* opt, int64_t* gram_rows_per_cta, int32_t* ht_ctas_per_sm);

/* Waits for `stream`, then returns the first non-OK device-side status the
 * instances of the last figaro_batch_join on workspace `ws` recorded (same
 * count, tables and options as that call), else FIGARO_OK.                 */
FIGARO_API figaro_status figaro_batch_get_status(int32_t count, const figaro_table* A, const figaro_table* B,
                                      const figaro_options* opt, const void* ws, void* stream);

/* Waits for `stream`, then returns the device-side status the last call
 * using workspace `ws` recorded (FIGARO_OK when nothing went wrong).        */
FIGARO_API figaro_status figaro_get_status(const void* ws, void* stream);

/* Facts about the last call that used workspace `ws` (waits for `stream`):
 * distinct keys of A and of B, keys present in both (key groups), rows of
 * the reduced matrix (sum over groups of m1g + m2g - 1), Jacobi sweeps run,
 * and the columns the final factorisation marked dependent (zero rows of R,
 * including columns that are zero in J).                                   */
typedef struct figaro_info {
  int64_t num_runs_a;
  int64_t num_runs_b;
  int64_t num_groups;
  int64_t reduced_rows;
  int32_t jacobi_sweeps;
  int32_t dependent_columns;
} figaro_info;

FIGARO_API figaro_status figaro_get_info(const void* ws, void* stream, figaro_info* info);

/* Static English text for a status code. */
FIGARO_API const char* figaro_status_string(figaro_status status);

/* Library version, e.g. 100 for 0.1.0 (major * 10000 + minor * 100 + patch). */
FIGARO_API int32_t figaro_version(void);

/* Number of kernels this library has launched in this process so far
 * (host-side count; a replayed CUDA graph does not go through it). */
FIGARO_API int64_t figaro_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* FIGARO_H_ */
