/*
 * hss.h -- C ABI of the GB300 HSS-ULV factorization and solve.
 *
 * The library factors a symmetric positive definite HSS (hierarchically
 * semiseparable) matrix with the ULV algorithm of Sec. 3 of "O(N) distributed
 * direct factorization of structured dense matrices using runtime systems"
 * (Alg. 2), solves with the factor (the solve formula of Sec. 3.2) and returns
 * the log-determinant.  Everything runs on one CUDA device in hand-written
 * kernels; there is no CPU fallback.
 *
 * Matrix format (Sec. 2, HSS construction and Eq. hss-block-notation), for a
 * uniform binary tree with leaves at level L and the root at level 0:
 *   - node i of level l has children 2i and 2i+1 of level l+1;
 *   - leaf diagonal blocks D_i (leaf x leaf), i = 0 .. 2^L - 1;
 *   - leaf bases U_i (leaf x rank);
 *   - transfer matrices E_{l;i} (2 rank x rank), levels l = 1 .. L-1, giving the
 *     nested basis Ũ_{l;i} = blkdiag(Ũ_{l+1;2i}, Ũ_{l+1;2i+1}) E_{l;i};
 *   - couplings S_{l;k} (rank x rank), levels l = 1 .. L, between siblings
 *     2k and 2k+1 of level l:  A(I_{2k+1}, I_{2k}) = Ũ_{2k+1} S_{l;k} Ũ_{2k}ᵀ
 *     (and its transpose above the diagonal).
 * All blocks are column-major FP64, packed without gaps:
 *   D: 2^L blocks of leaf*leaf, U: 2^L blocks of leaf*rank,
 *   E: level 1 first, then 2, ... L-1; level l holds 2^l blocks of 2rank*rank,
 *   S: level 1 first, then 2, ... L;   level l holds 2^(l-1) blocks of rank*rank.
 * The bases need full column rank; they need not be orthonormal.
 * Vectors are in cluster (tree) order: rows i*leaf .. (i+1)*leaf-1 belong to
 * leaf i.  Multi-column vectors are column-major with leading dimension ld.
 *
 * Streams: every call that takes `stream` (a cudaStream_t, NULL = legacy
 * default stream) is asynchronous on it unless stated.  Errors detected on the
 * device (a non-positive pivot) surface at the next synchronizing call:
 * hss_logdet, hss_last_info, hss_sync, or hss_solve of a mixed-precision factor.
 *
 * Return codes: HSS_OK (0) or a negative HSS_ERR_* code; hss_strerror names it.
 */
#ifndef HSS_GB300_H
#define HSS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HSS_OK 0
#define HSS_ERR_INVALID_ARG (-1)   /* bad pointer, size or option */
#define HSS_ERR_NOT_FACTORIZED (-2) /* solve / logdet before a successful factorize */
#define HSS_ERR_NOT_SPD (-3)        /* a Cholesky pivot was not positive (see hss_last_info) */
#define HSS_ERR_CUDA (-4)           /* a CUDA runtime call or kernel launch failed */
#define HSS_ERR_OOM (-5)            /* device allocation failed */
#define HSS_ERR_TIMEOUT (-6)        /* a bounded device wait gave up */
#define HSS_ERR_NO_CONVERGENCE (-7) /* iterative refinement hit its iteration limit */
#define HSS_ERR_TOO_LARGE (-8)      /* problem exceeds the fixed scratch of hss_matvec_noalloc */

typedef struct hss_s* hss_t;

/* Arithmetic of the factorization.  HSS_FP64 computes every step in FP64.
 * The mixed modes compute the per-level steps of Alg. 2 (diagonal product,
 * partial Cholesky, merge) in lower precision and use the factor as the
 * preconditioner of FP64 iterative refinement in hss_solve; the root
 * Cholesky, residual and update are FP64.
 * HSS_MIXED_FP32: every per-level step in FP32 (FP32 accumulation).
 * HSS_MIXED_TF32 / HSS_MIXED_BF16: as FP32, but the two dense contractions of
 * the diagonal product (W = A V and A - Y'Vᵀ - V Y'ᵀ) run on the tensor cores
 * (tcgen05) with TF32 / BF16 inputs and FP32 accumulation in tensor memory;
 * every operand is split into hi + lo input-type parts and hi·hi + hi·lo + lo·hi
 * is accumulated, so the contraction keeps most of the FP32 accuracy that the
 * refinement needs. */
typedef enum {
  HSS_FP64 = 0,
  HSS_MIXED_TF32 = 1,
  HSS_MIXED_BF16 = 2,
  HSS_MIXED_FP32 = 3
} hss_precision;

typedef struct {
  int32_t n;      /* matrix order: leaf * 2^levels, or the sum of node_sizes */
  int32_t leaf;   /* leaf block order (1 .. 1024); with node_sizes, the largest leaf
                     order.  Above 768 the FP64 factorization takes rank <= 176 (the
                     basis kernel's shared memory; hss_factorize reports
                     HSS_ERR_INVALID_ARG beyond); the FP32 one any rank. */
  int32_t rank;   /* rank of every basis (1 .. min(leaf, 256)); with node_sizes the
                     largest rank, see below */
  int32_t levels; /* L >= 1 */
  const int32_t* node_sizes; /* NULL: uniform tree.  Otherwise a host array of the
                     2^levels leaf orders b_i (1 .. leaf, summing to n): an uneven
                     tree, e.g. from median bisection of n points with n a multiple
                     of nothing.  Ranks follow the orders: r_i = min(rank, b_i) at
                     leaf i, r_p = min(rank, r_c1 + r_c2) at a parent of c1, c2.  The
                     generators are then packed block after block with those
                     shapes: D_i b_i x b_i, U_i b_i x r_i, E_{l;p} (r_c1 + r_c2) x r_p,
                     S_{l;k} r_{2k+1} x r_{2k}.  The library embeds the tree in the
                     uniform (leaf, rank) format -- identity on the padded diagonal,
                     identity columns on the padded basis directions, zero padded
                     couplings -- which is the matrix A ⊕ I up to a row
                     permutation, so x and log det are those of A; vectors stay
                     n x nrhs in cluster order (the library scatters and gathers
                     them), hss_export returns the padded blocks. */
} hss_shape;

/* Arithmetic of the refinement residual r = b - A x of the mixed modes.
 * HSS_RESIDUAL_FP64: the HSS matvec in FP64 (the chip's FP64 pipe).
 * HSS_RESIDUAL_PAIR32: the same matvec with every value held as an unevaluated
 * sum of two FP32 numbers (48-bit significand) and every product and sum done
 * with error-free FP32 transformations on the FP32 pipe; a dot product of
 * length K then carries a relative error of about sqrt(K) 2^-48 (~1e-13 for the
 * leaf products), two orders below the 1e-12 that the refinement stops at.
 * The update x += d and the convergence test stay FP64. */
typedef enum { HSS_RESIDUAL_FP64 = 0, HSS_RESIDUAL_PAIR32 = 1 } hss_residual;

/* Method of the basis completion (Eq. 2-3); both give the same V, T and L_B up
 * to rounding (the Householder QL with LAPACK's dlarfg signs).
 * HSS_BASIS_HOUSEHOLDER (default): the Householder kernel, one CTA per node
 * with a CTA-wide reduction per column.
 * HSS_BASIS_CHOLQR: Cholesky QR twice of the reversed basis as level-wide
 * products, then the Householder vectors reconstructed from the orthonormal
 * factor by an unpivoted LU of its top block (one CTA per node); nodes whose
 * Gram matrix is not numerically positive definite in the working precision,
 * and ranks too large for the per-node kernels (above 165 in FP64, 234 in
 * FP32), use the Householder kernel. */
typedef enum { HSS_BASIS_HOUSEHOLDER = 0, HSS_BASIS_CHOLQR = 1,
               HSS_BASIS_AUTO = 2 /* the choice of hss_tune, else HOUSEHOLDER */ } hss_basis_method;

/* Schedule of the solve's upper levels (the levels of at most 64 nodes above
 * the leaves).  HSS_SCHEDULE_ASYNC: one launch per direction for all of them,
 * with no barrier between levels (asynchronous execution of the tree, Sec. 4.2):
 * going up, the CTA that finishes the second child of a node goes on with the
 * node; going down, a cooperative launch in which each node waits for its
 * parent's ready flag (a bounded wait, see wait_budget; an expired wait makes
 * the solve report HSS_ERR_TIMEOUT).  HSS_SCHEDULE_LEVELS: one launch per level
 * and direction.  Both give the same result. */
typedef enum { HSS_SCHEDULE_ASYNC = 0, HSS_SCHEDULE_LEVELS = 1,
               HSS_SCHEDULE_AUTO = 2 /* the choices of hss_tune (schedule and the sweeps'
                                        panel staging), else ASYNC */ } hss_schedule;

typedef struct {
  int32_t precision;   /* hss_precision */
  int32_t ir_max_it;   /* refinement iteration limit (mixed modes), e.g. 30 */
  double ir_tol;       /* stop when every column has ‖b - A x‖₂ / ‖b‖₂ <= ir_tol */
  int32_t residual;    /* hss_residual (mixed modes) */
  int32_t basis;       /* hss_basis_method: how the basis completion is computed */
  int64_t wait_budget; /* polls a device-side wait (tensor-core pipeline, ready flags of
                          the solve) makes before it gives up and the call reports
                          HSS_ERR_TIMEOUT (at the next synchronizing call); 0 = the
                          default, 2^24 polls.  A negative value makes
                          every such wait give up at once: a way to exercise the failure
                          path.  The final wait of a kernel for tensor-core work it has
                          already issued always uses the default, so that tensor memory
                          is never released under a pending MMA. */
  int32_t schedule;    /* hss_schedule: how the solve's upper levels are launched */
  int32_t ql_panel;    /* columns per register panel of the Householder basis kernel:
                          16 or 32 in the FP32 arithmetic (FP64 always 16); 0 = the
                          default (32 in FP32).  With basis = HSS_BASIS_AUTO the
                          choice of hss_tune is used instead.  Other values:
                          HSS_ERR_INVALID_ARG. */
  int32_t ir_lanes;    /* refinement lanes of a mixed solve with the FP64 residual: 1 or 2;
                          0 = the choice of hss_tune under schedule = HSS_SCHEDULE_AUTO,
                          else 1.  Other values: HSS_ERR_INVALID_ARG. */
  int32_t reserved;    /* 0 */
} hss_options;

/* Create a device-resident HSS object from its generators (format above).
 * D, U, E, S are host pointers (on_device = 0) or device pointers of the current
 * device (on_device = 1; uniform trees only); they are copied and the caller
 * keeps ownership.  The
 * object owns one device arena (inputs, factor, workspace for up to 32
 * right-hand-side columns per pass); it is tied to the device current at
 * creation.  E may be NULL when levels = 1.  Synchronous (returns after the
 * copies).  Errors: INVALID_ARG (sizes out of range, NULL pointers), OOM, CUDA. */
int hss_create(const hss_shape* shape, const double* D, const double* U, const double* E,
               const double* S, int on_device, hss_t* out);

/* ULV factorization, Alg. 2: for l = L .. 1, for every node of level l,
 * (a) complete the node basis to an orthogonal Q = [Q^R Q^S] (Householder QL,
 *     Eq. 2-3), (b) form Qᵀ A_i Q (diagonal product, Eq. dense-split),
 * (c) partial Cholesky of the redundant block with the TRSM and SYRK of Eq.
 *     partial-Cholesky, and (d) merge sibling Schur complements and the
 *     rescaled coupling into the parent's 2rank x 2rank block; then the root
 *     Cholesky.  The factor replaces any previous one.  opt may be NULL (FP64).
 * Asynchronous; a non-positive pivot is reported by the next synchronizing
 * call as HSS_ERR_NOT_SPD with its level, node and column. */
int hss_factorize(hss_t h, const hss_options* opt, void* stream);

/* Solve A x = b with the factor (Sec. 3.2): forward sweep leaves -> root
 * (apply Qᵀ, L^RR⁻¹, update and push the skeleton part to the parent), root
 * Cholesky solve, backward sweep root -> leaves.  b and x are device pointers,
 * n x nrhs column-major with leading dimension ld >= n; x may equal b.  With an
 * FP64 factor the call is asynchronous.  With a mixed factor it runs iterative
 * refinement with an FP64 iterate, update and stopping test (residual by the HSS
 * matvec in the arithmetic hss_options.residual selects) and synchronizes once per
 * iteration; it returns HSS_ERR_NO_CONVERGENCE if ir_max_it is reached (x then
 * holds the last iterate).  With the FP64 residual and the autotuner's choice
 * (schedule = HSS_SCHEDULE_AUTO after hss_tune) a pass of columns may run on two
 * lanes (streams) of half the columns each, one lane's FP32 sweeps beside the
 * other's FP64 matvec; each lane stops on its own columns, so a column's
 * result does not depend on the split.  Errors: NOT_FACTORIZED, INVALID_ARG,
 * CUDA.
 * Every leaf order up to 1024 is solved in every precision (the sweeps stage their
 * panels in as much shared memory as the device grants). */
int hss_solve(hss_t h, const double* b, double* x, int32_t nrhs, int32_t ld, void* stream);

/* log det A from the factorized form (Eq. hss-ulv-final-form): twice the sum of
 * the logs of the diagonals of every L^RR and of the root factor.  Writes one
 * host double.  For a mixed factor it is the log-determinant of that
 * lower-precision factor (root in FP64), not refined.  Synchronizes the
 * object's last stream.  Errors: NOT_FACTORIZED, NOT_SPD. */
int hss_logdet(hss_t h, double* out);

/* y = A x with the HSS generators (the product A·b of the construction-error
 * formula in Sec. 5.1): upward pass through U and E, sibling couplings, downward
 * pass, leaf blocks.  FP64.  x and y are device pointers (n x nrhs, ld), must
 * not overlap.  Asynchronous.  Needs no factorization. */
int hss_matvec(hss_t h, const double* x, double* y, int32_t nrhs, int32_t ld, void* stream);

/* y = A x as hss_matvec, every product and sum in pair-of-FP32 arithmetic
 * (HSS_RESIDUAL_PAIR32): the generators are split once into hi = fl32(g) and
 * lo = fl32(g - hi) (done by any mixed factorization, or by the first call),
 * x is split per column after scaling by a power of two near 1 / ‖x_j‖₂, and y
 * is returned in FP64, scaled back.  Relative error about sqrt(K) 2^-48 of
 * |A| |x| for inner dimension K.  Allocates the FP32 workspace on first use.
 * x and y are device pointers (n x nrhs, ld), must not overlap.  Asynchronous.
 * Errors: INVALID_ARG, OOM, CUDA. */
int hss_matvec_pair(hss_t h, const double* x, double* y, int32_t nrhs, int32_t ld, void* stream);

/* y = A x like hss_matvec, but allocating nothing: no cudaMalloc, no cudaFree,
 * no allocating library call.  The paper has no counterpart; this entry point
 * exists for callers that must not allocate device memory at call time -- for
 * example a host application that reserves the whole device up front for its
 * own memory pool, or a latency-critical loop in which a cudaMalloc (which can
 * synchronize the device) is not acceptable.  Such callers cannot use
 * hss_create, which allocates the object's arena.
 *   shape, D, U, E, S: the generators in the packed layout of hss_create, as
 *     DEVICE pointers on the current device, owned by the caller and only read.
 *   x, y: device pointers, n x nrhs column-major with leading dimension ld;
 *     they must not overlap.
 * The per-level intermediate vectors live in one static device array of
 * 2^21 doubles (16 MiB) that every device which loads the library holds until
 * the process exits.  A problem fits when 2 (2^(levels+1) - 2) rank <= 2^21
 * (one right-hand-side column); larger ones return HSS_ERR_TOO_LARGE before any
 * device work.  Columns are processed in passes of as many as fit (at most 32).
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  The
 * address is kept for the life of the process, so do not call this entry point
 * again after a cudaDeviceReset (or any other teardown of the device's primary
 * context): the module may then be loaded at another address.  Every call
 * shares the one array and overwrites all of the part it reads, so no state
 * carries over between calls -- but two calls that overlap on the GPU (other
 * streams, other host threads) race on it: serialize them.
 * Uniform trees only (shape->node_sizes must be NULL).
 * Asynchronous on `stream`.  Errors: INVALID_ARG, TOO_LARGE, CUDA. */
int hss_matvec_noalloc(const hss_shape* shape, const double* D, const double* U, const double* E,
                       const double* S, const double* x, double* y, int32_t nrhs, int32_t ld,
                       void* stream);

/* Choices of the autotuner (hss_tune) for one object: the basis method, the
 * panel width of the Householder basis kernel (16 or 32 columns: the wider
 * panel holds more of the basis in registers, the narrower one lets two CTAs
 * share an SM), the schedule of the solve's upper levels, the panel staging of
 * the solve's sweep kernels (0 = the largest shared-memory panels, 1 = the
 * panels that let the fewest waves of CTAs cover a level), the refinement
 * lanes of a mixed solve, and the measured times of the chosen configuration. */
typedef struct {
  int32_t basis;      /* hss_basis_method */
  int32_t schedule;   /* hss_schedule */
  int32_t staging;    /* 0 or 1 */
  int32_t from_cache; /* 1 when read from the cache file instead of measured */
  double factor_ms;   /* one factorization with the chosen basis method */
  double solve_ms;    /* one solve of min(nrhs, 16) columns with the chosen schedule */
  double factor_ms_by_basis[2];        /* every candidate measured: [basis method] */
  double solve_ms_by_config[2][2];     /* [schedule][staging]; 0 where not measured */
  int32_t ql_panel;                    /* 16 or 32 */
  int32_t ir_lanes;                    /* refinement lanes, 1 or 2 (see hss_solve) */
  double factor_ms_by_panel[2];        /* Householder basis with 16 / 32-column panels;
                                          0 where not measured (FP64 has 16 only) */
  double solve_ms_by_lanes[2];         /* best solve with 1 / 2 refinement lanes; 0 where
                                          not measured */
} hss_tuning;

/* Autotuner: for the object's shape and the arithmetic of opt (precision,
 * residual), times every candidate configuration on the object itself with
 * CUDA events on `stream` -- each basis method (the Householder one with each
 * panel width its arithmetic has) on hss_factorize, each pair of
 * solve schedule and sweep panel staging on hss_solve of min(nrhs, 16)
 * columns of a fixed test vector -- best of two runs each, and keeps the
 * fastest; later hss_factorize calls with basis = HSS_BASIS_AUTO or schedule =
 * HSS_SCHEDULE_AUTO use them.  cache_path (may be NULL): a text file of
 * earlier choices, one line per key (device name, precision, residual, n,
 * leaf, rank, levels, columns); a matching line is used instead of measuring,
 * and a new measurement is appended.  Leaves the object factorized with the
 * chosen configuration.  Allocates two n x 16 vectors for the duration of the
 * call.  Synchronous.  out may be NULL.  Errors: as hss_factorize and
 * hss_solve, OOM. */
int hss_tune(hss_t h, const hss_options* opt, int32_t nrhs, const char* cache_path, void* stream,
             hss_tuning* out);

/* Block until the object's work is done and report any device-side failure
 * (HSS_ERR_NOT_SPD ...). */
int hss_sync(hss_t h);

/* Details of the last factorization / solve (any pointer may be NULL): the
 * level, node and column of a failed pivot (-1 if none), and the refinement
 * iteration count and final max relative residual of the last mixed solve.
 * Synchronizes.  Returns the pending device error code, if any. */
int hss_last_info(hss_t h, int32_t* level, int32_t* node, int32_t* col, int32_t* ir_iters,
                  double* ir_resid);

/* Copy one per-level array of the factor to host memory, for inspection and
 * per-step tests.  what: 0 = V (Householder vectors, b x rank per node, unit
 * diagonal explicit), 1 = T (compact-WY factor, rank x rank upper; Q = I - V T Vᵀ),
 * 2 = L_B (rank x rank lower, L_B = Q^Sᵀ B), 3 = factored block (b x b: lower
 * triangle holds L^RR, L^SR and the Schur complement Â^SS), 4 = basis fed to
 * the basis completion of level l < L (2 rank x rank per node: the merge output
 * blkdiag(L_B(2i), L_B(2i+1)) E_{l;i}).
 * dst receives 2^l blocks back to back; count is its capacity in doubles.
 * Synchronizes.  Errors: INVALID_ARG, NOT_FACTORIZED, and INVALID_ARG when the
 * factor is not FP64. */
int hss_export(hss_t h, int32_t what, int32_t level, double* dst, size_t count);

/* Kernel classes reported by the tracer (one per kernel function). */
typedef enum {
  HSS_K_QL = 0,        /* basis completion by the Householder kernel (QL + compact-WY T) */
  HSS_K_GEMM = 1,      /* batched GEMM, 64x64 tiles (diagonal product, merge) */
  HSS_K_GEMM_SKINNY = 2, /* batched GEMM with <= 32 columns (solve, matvec) */
  HSS_K_SYR2K = 3,     /* lower-triangle rank-2k update (diagonal product) */
  HSS_K_PCHOL = 4,     /* partial Cholesky + merge epilogue, root Cholesky */
  HSS_K_TRSV_FWD = 5,  /* forward triangular sweep of the solve */
  HSS_K_TRSV_BWD = 6,  /* backward triangular sweep of the solve */
  HSS_K_OTHER = 7,     /* log-det reduction, precision conversion, refinement helpers */
  HSS_K_TC_GEMM = 8,   /* tensor-core (tcgen05) W = A V of the mixed diagonal product */
  HSS_K_TC_SYR2K = 9,  /* tensor-core (tcgen05) rank-2r update of the mixed diagonal product */
  HSS_K_PAIR_GEMM = 10, /* pair-of-FP32 GEMM of the refinement residual (logged as FP32) */
  HSS_K_BASIS_GEMM = 11, /* level-wide products of the basis completion (Cholesky QR, reconstruction) */
  HSS_K_BASIS_NODE = 12, /* per-node Cholesky / LU / triangular inverses of the basis completion */
  HSS_K_COUNT = 13,
  HSS_K_FP32 = 13      /* added to a class: the same kernel run in FP32 (mixed modes) */
} hss_kernel_kind;

/* Per-kernel timing: with enable = 1 every later launch of the object is
 * bracketed by two CUDA events on its launch stream and logged with its
 * algorithmic flop count (the operation's definition, not the executed
 * instructions); enable = 0 stops logging.  Enabling clears the log.
 * enable = 2 logs as 1 and also serializes the factorization: the basis
 * completion chain, which otherwise runs ahead on the object's second stream,
 * runs on the caller's stream, so that every logged duration is the kernel's
 * own and not shared with a concurrent kernel (for roofline accounting; the
 * results are the same). */
int hss_trace(hss_t h, int32_t enable);

/* Sum of the logged launches of one kernel class (0 .. 2*HSS_K_COUNT-1; classes
 * from HSS_K_FP32 on are the FP32 launches): total device milliseconds, number
 * of launches and algorithmic flops.  Synchronizes the logged streams.
 * Errors: INVALID_ARG. */
int hss_trace_read(hss_t h, int32_t kind, double* ms, int64_t* launches, double* flops);

/* Number of kernel launches the object has issued since creation. */
int hss_launch_count(hss_t h, int64_t* out);

/* Free the object and its device memory. NULL is ignored. */
void hss_destroy(hss_t h);

/* ---- batches of independent HSS matrices (FP64) ------------------------------
 * Many matrices of uneven order, leaf size, rank and depth factored and solved
 * together; each step of Alg. 2 runs as one launch per (leaf, rank) group and
 * tree height for all matrices of the group (the "Batching" of uneven problems;
 * the paper factors one matrix at a time).  Matrices with equal (leaf, rank)
 * share launches whatever their depth: per group the level arrays are
 * concatenated by height above the leaves, deepest matrices first, so the
 * nodes of every height form one uniform batch. */
typedef struct hss_batch_s* hss_batch_t;

/* Create a batch of `count` matrices: shapes[i] and the generators D[i], U[i],
 * E[i], S[i] of matrix i as HOST pointers in the packed layout of hss_create
 * (E[i] may be NULL when levels = 1).  Copies them; the caller keeps ownership.
 * Synchronous.  Errors: INVALID_ARG, OOM, CUDA. */
int hss_batch_create(int32_t count, const hss_shape* shapes, const double* const* D,
                     const double* const* U, const double* const* E, const double* const* S,
                     hss_batch_t* out);

/* Factor every matrix (Alg. 2, FP64; opt may be NULL, precision must be FP64).
 * Asynchronous on `stream` (the groups run on internal streams joined to it). */
int hss_batch_factorize(hss_batch_t b, const hss_options* opt, void* stream);

/* With enable = 1, later hss_batch_factorize calls run from a CUDA graph: the
 * first such call runs the factorization once, then captures its launches (on
 * an internal stream) into a graph; every call after that replays the graph,
 * ordered after earlier work on `stream` and before later work on it. */
int hss_batch_set_graph(hss_batch_t b, int32_t enable);

/* Solve A_i x_i = b_i for every matrix: b[i], x[i] are device pointers to
 * n_i x nrhs column-major blocks with leading dimension n_i (x[i] may equal b[i]);
 * the arrays b and x are host arrays of `count` pointers.  Returns after the
 * work is queued and the pointer tables are consumed (it synchronizes `stream`
 * once per 16 right-hand-side columns).  Errors: INVALID_ARG, NOT_FACTORIZED, CUDA. */
int hss_batch_solve(hss_batch_t b, const double* const* bvec, double* const* x, int32_t nrhs,
                    void* stream);

/* log det of every matrix into out[0 .. count-1] (host).  Synchronizes the
 * device.  Errors: NOT_FACTORIZED, NOT_SPD (first failure of any matrix). */
int hss_batch_logdet(hss_batch_t b, double* out);

void hss_batch_destroy(hss_batch_t b);

/* Static string naming a return code. */
const char* hss_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* HSS_GB300_H */
