/*
 * hm.h - C ABI of the GB300 library for randomized compression of
 * rank-structured matrices (Martinsson, "Compressing rank-structured matrices
 * via randomized sampling", arXiv:1503.07152).
 *
 * The library sees the N x N operator A only through a black box that applies
 * A or A^T to a block of vectors (Sec. 1; Sec. 3: "black-box matrix-matrix
 * multiplier"; Sec. 5.3: the black box acts on N x l blocks), and returns a
 * HODLR (Sec. 2.8, Sec. 3) or HBS / HBS-ID (Secs. 2.9, 4) representation that
 * can be applied, transposed and read back block by block.
 *
 * Conventions for every entry point:
 *  - Matrices of vectors (X, Y, sample blocks) are column-major with a leading
 *    dimension ld >= rows; element (i, j) is at ptr[i + j * ld].
 *  - Dense operators handed to hm_dense_operator_create are row-major:
 *    element (i, j) is at A[i * lda + j].
 *  - "device pointer" means memory of the current CUDA device; "host pointer"
 *    means ordinary (pageable or pinned) host memory.
 *  - Element type follows the precision of the call: HM_FP64 and HM_A32 ->
 *    double, HM_MIXED -> float.
 *  - Work is enqueued on the caller's stream (a cudaStream_t passed as void*;
 *    NULL = legacy default stream).  Unless stated otherwise a call returns
 *    after enqueueing (asynchronous); the compress calls synchronize the stream
 *    once at their end to read device-side status flags.
 *  - Every entry point returns an hm_status.  On failure nothing is returned
 *    through output handles (no partial handles), and hm_last_error() gives a
 *    thread-local message describing the first error of the failing call.
 */
#ifndef HM_H_
#define HM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HM_OK = 0,
  HM_EINVAL = 1,           /* bad argument (null pointer, size, ld, mode) */
  HM_ENOMEM = 2,           /* device or host allocation failed */
  HM_ECUDA = 3,            /* a CUDA runtime call or kernel launch failed */
  HM_ECALLBACK = 4,        /* the black-box apply returned non-zero */
  HM_ERANK_SATURATED = 5,  /* strict mode only: an adaptive rank reached r */
  HM_ENONFINITE = 6,       /* NaN/Inf detected in the samples */
  HM_ETIMEOUT = 7,         /* a bounded device-side wait gave up */
  HM_EUNSUPPORTED = 8      /* valid request outside what this library version supports */
} hm_status;

/* HM_FP64: FP64 operator and pipeline.  HM_MIXED: FP32 samples, bases and
 * peeling (small solves of the ID in FP64).  HM_A32: FP32 operator applied in
 * FP64 (the black box receives and returns double blocks), FP64 pipeline. */
typedef enum { HM_FP64 = 0, HM_MIXED = 1, HM_A32 = 2 } hm_precision;
typedef enum { HM_FORMAT_HODLR = 0, HM_FORMAT_HBS = 1, HM_FORMAT_HBSID = 2 } hm_format;

/*
 * Black box (Sec. 1, T_mult; Fig. "Randomized compression of a HODLR matrix":
 * the products A*Omega and A^*Omega).  Computes Y(0:n, 0:ncols) = op(A) X with
 * op = A (trans = 0) or A^T (trans = 1).  X and Y are device pointers,
 * column-major, element type double (HM_FP64, HM_A32) or float (HM_MIXED).  The
 * callback must enqueue its work on `stream` (a cudaStream_t) and return 0; any
 * other value aborts the compression with HM_ECALLBACK.  X is read-only and is
 * not retained after the call returns.
 */
typedef int (*hm_apply_fn)(void* ctx, int trans, int64_t n, int64_t ncols,
                           const void* X, int64_t ldx, void* Y, int64_t ldy,
                           void* stream);

typedef struct {
  hm_apply_fn apply;  /* required */
  void* ctx;          /* passed through unchanged; owned by the caller */
  int64_t n;          /* operator size N */
} hm_operator;

/*
 * Compression options.  Mode 2 / mode 3 of Sec. 2.6: fixed rank k
 * (mode_tol = 0) or tolerance tol (mode_tol = 1).  r = k + p random vectors
 * per level (p: oversampling, Sec. 2.5, default 10).  In tolerance mode r is
 * given directly by `r` (must be > 0).  leaf_size: the tree's m (Sec. 2.7).
 * seed: key of the Philox4x32-10 test matrices.  prec: HM_FP64, HM_A32 or HM_MIXED.
 * hbs_id: for hm_compress_hbs, 1 converts to HBS-ID with adaptive ranks
 * (Sec. 4.3), 0 keeps the fixed-rank HBS form.  strict_rank: 1 makes a
 * saturated adaptive rank an error (HM_ERANK_SATURATED) instead of a counter
 * in hm_info.
 * lookahead: the A-side test matrix of every level is a fresh Gaussian block
 * (Sec. 3, Sec. 4.2), so its product with A does not depend on the levels
 * before it; the compression can then apply the black box to the next level's
 * block on a second stream of its own while it factors the current level's
 * samples (and to the identity probe during the last level).  The results are
 * the same bit for bit.  0: on for the library's own black boxes
 * (hm_dense_operator_create, hm_log_kernel_operator_create), off for a user
 * callback; 1: on for any black box, which must then enqueue its work on the
 * stream it is given and accept two calls in flight at once on two streams;
 * -1: off.  hm_compress_batched does not look ahead.
 */
typedef struct {
  int32_t mode_tol;
  int32_t k;
  double tol;
  int32_t p;
  int32_t r;
  int32_t leaf_size;
  uint64_t seed;
  int32_t prec;
  int32_t hbs_id;
  int32_t strict_rank;
  int32_t lookahead;
} hm_opts;

typedef struct hm_tree hm_tree;
typedef struct hm_handle hm_handle;

typedef struct {
  int32_t format;          /* hm_format */
  int32_t prec;            /* hm_precision */
  int64_t n;
  int32_t levels;          /* L */
  int32_t r;               /* random vectors per level and side */
  int32_t max_rank;        /* largest rank kept in any block */
  int32_t min_rank;
  int32_t saturated;       /* number of blocks whose adaptive rank hit r */
  int64_t cols_A;          /* black-box columns applied with A */
  int64_t cols_At;         /* black-box columns applied with A^T */
  int64_t bytes;           /* device bytes held by the representation (M) */
  double eps_abs;          /* absolute truncation threshold used (mode 3) */
  double t_compress_ms;    /* wall time of the compress call */
  double t_blackbox_ms;    /* time inside the black box (T_compress - T_net) */
  int32_t launches;        /* kernels launched by the last compress call */
} hm_info_t;

/* ---------------------------------------------------------------- tree --- */

/*
 * Binary tree over [0, n) (Sec. 2.7, Fig. 1): uniform depth
 * L = ceil(log2(n / leaf_size)), a node of size s splits into floor(s/2)
 * (left) and s - floor(s/2) (right); heap numbering, root = 1.  Host-side
 * object (plus a small device copy of the node table); owned by the caller.
 */
hm_status hm_tree_create(int64_t n, int32_t leaf_size, hm_tree** out);
void hm_tree_destroy(hm_tree* t);
/* Levels below the root (L). */
int32_t hm_tree_levels(const hm_tree* t);
/* Index range [start, start + size) of heap node `node` (1 <= node < 2^(L+1)). */
hm_status hm_tree_node(const hm_tree* t, int64_t node, int64_t* start, int64_t* size);

/* --------------------------------------------------------- black boxes --- */

/*
 * Dense test operator: wraps a row-major N x N device matrix A (lda >= N) as a
 * black box whose apply is the library's sampling GEMM.  dtype 0: double
 * matrix, double blocks (HM_FP64); 1: float matrix, float blocks (HM_MIXED) on
 * the tensor cores (three-way BF16 split, FP32 accumulation drained into
 * compensated FP32 sums); 2: float matrix, double blocks with FP64 products and
 * sums (HM_A32); 3: as 1 on the CUDA cores (FP32 FMA, compensated sums); 4: as 2
 * on the tensor cores: rows of A (per 256-wide window of columns) and columns
 * of X (per 256-row window) are cut into four 8-bit integer BF16 slices under a
 * power-of-two scale, the products of each order are summed exactly in FP32 accumulators
 * over 256-wide K windows, orders above 5 are
 * dropped (relative weight <= 2^-32), and the window sums are added in FP32
 * double-float; results whose magnitude exceeds the FP32 range are not
 * representable (use 2).  The row and column scales of A are read once, at the
 * first dtype-4 apply (one extra pass over A); if A's entries later grow past
 * them, the affected outputs come back NaN (create a new operator after
 * changing A).  The
 * matrix is NOT copied or owned: it must outlive the operator.  dtypes 1 and 4
 * grow a device workspace (the BF16 split of X) on first use of a larger block
 * and need a 16-byte aligned A with lda % 4 == 0 and n >= 128 (TMA); other
 * layouts run on the CUDA cores (dtype 3, resp. 2).  The returned operator's ctx is released by
 * hm_dense_operator_destroy.  Per-call scratch (zero-tile flags, the split of
 * X) comes in two sets: one for calls through the callback or hm_dense_apply,
 * one for a compression's look-ahead stream (hm_opts.lookahead), so one
 * compression may have a product of each kind in flight.  Calls that use the
 * same set and may overlap on the GPU (one operator applied from two streams,
 * or compressed by two calls at once) race on it: give each concurrent user an
 * operator of its own.
 */
hm_status hm_dense_operator_create(const void* A, int64_t n, int64_t lda, int32_t dtype,
                                   hm_operator* out);
void hm_dense_operator_destroy(hm_operator* op);

/*
 * Matrix-free black box (Sec. 5: the paper's black boxes are fast matrix-vector
 * multipliers, an FMM in Sec. 5.3, not stored matrices): the log kernel of n
 * points on the ellipse x_i = (cos t_i, 0.5 sin t_i), t_i = 2 pi i / n, with
 * its entries formed in registers inside the sampling GEMM and never stored.
 * With d = pi (i - j) / n and f = pi (i + j) / n,
 *   |x_i - x_j|^2 = sin^2(d) (1 + 3 sin^2(f)),
 * so log|x_i - x_j| = S[|i - j|] + P[i + j] with the tables
 *   S[m] = log|sin(pi m / n)|,  P[s] = log(1 + 3 sin^2(pi s / n)) / 2,
 * each computed in FP64 on the host and kept as a float pair (hi = the value
 * rounded to FP32, lo = the remainder rounded to FP32).  The operator's entries
 * are DEFINED as fl32(fl32(Sh + Ph) + fl32(Sl + Pl)) for i != j and 1 on the
 * diagonal: within about one FP32 ulp of log|x_i - x_j| even where the two
 * terms cancel (distances near 1).  It is
 * symmetric; its products are those of dtype 4 of hm_dense_operator_create
 * (FP64 blocks, exact-accumulation split on the tensor cores) on these
 * entries, with no operator bytes read from HBM (24 n bytes of tables).
 * Element type double (HM_A32).  2 <= n <= 524288 (HM_EINVAL otherwise: the
 * GEMM tracks its K tiles in one shared-memory bitmask).  Destroy with
 * hm_dense_operator_destroy.
 */
hm_status hm_log_kernel_operator_create(int64_t n, hm_operator* out);

/*
 * Entries A(r0:r1, c0:c1) of a matrix-free log-kernel operator, written
 * row-major to the device buffer `out` (element (i, j) at
 * out[(i - r0) * ld + (j - c0)], ld >= c1 - c0).  For checks and for forming a
 * dense copy; the compression never calls it.
 */
hm_status hm_log_kernel_entries(const hm_operator* op, int64_t r0, int64_t r1, int64_t c0,
                                int64_t c1, float* out, int64_t ld, void* stream);

/*
 * Status of a dense operator's tensor-core GEMMs (dtypes 1 and 4): synchronizes
 * `stream`, then returns HM_ETIMEOUT if one of their bounded device-side waits
 * gave up since the last check (those outputs were written as NaN; the flag is
 * cleared), else HM_OK.  The compress calls run this check themselves at their
 * end for dense operators and return HM_ETIMEOUT ahead of HM_ENONFINITE.
 */
hm_status hm_dense_operator_check(const hm_operator* op, void* stream);

/*
 * Poll limit of the bounded mbarrier waits inside the tensor-core GEMMs'
 * pipelines (process-wide; polls <= 0 restores the default 2^25, seconds of
 * waiting).  A wait that runs out makes the block give up: it raises the
 * operator's error flag, writes NaN, and leaves only after its own TMA copies
 * have landed and its issued MMAs have completed (those waits always take the
 * default limit).  A small limit makes normal calls fail with HM_ETIMEOUT; it
 * exists to exercise that path.
 */
hm_status hm_set_wait_limit(int64_t polls);

/*
 * The sampling GEMM behind the dense operator, callable directly:
 * Y = op(A) X for the row-major dense A above.  Same argument rules as
 * hm_apply_fn.  Returns HM_OK or an error status.
 */
hm_status hm_dense_apply(const hm_operator* op, int trans, int64_t ncols, const void* X,
                         int64_t ldx, void* Y, int64_t ldy, void* stream);

/*
 * The level-`level` test matrix X = [Omega_2 | Omega_1] (n x 2r, column-major,
 * device, ldx >= n) of the compression sweeps (Fig. "Randomized compression of
 * a HODLR matrix": Omega_1 = randn on the left child of every parent on
 * `level`, Omega_2 = randn on the right child; both zero elsewhere).  Entry
 * (i, c) of the level's Gaussian field is Philox4x32-10 (key = seed, counter =
 * (i, c / 2, level, 0)) followed by Box-Muller in FP64; HM_MIXED rounds it to
 * FP32 and then to BF16 (round to nearest even) and stores float, HM_FP64
 * stores double.  Right children get columns [0, r), left children [r, 2r).
 */
hm_status hm_gaussian_test_matrix(const hm_tree* tree, int32_t level, int32_t r, uint64_t seed,
                                  int32_t prec, void* X, int64_t ldx, void* stream);

/* ---------------------------------------------------------- compression --- */

/*
 * HODLR compression by randomized peeling (Sec. 3, Fig. "Randomized
 * compression of a HODLR matrix", diagonal-B variant of Remark 4).  op->n must
 * equal the tree's n.  On success *out owns all device memory of the
 * representation.  Synchronizes `stream` once at the end.
 */
hm_status hm_compress_hodlr(const hm_operator* op, const hm_tree* tree, const hm_opts* opts,
                            void* stream, hm_handle** out);

/*
 * HBS compression with nested bases (Sec. 4.2, Fig. "A storage efficient
 * algorithm for compressing an HBS matrix"), followed when opts->hbs_id = 1 by
 * the upward sweep that converts it to HBS-ID with adaptive ranks (Sec. 4.3,
 * Fig. "An algorithm for computing the HBS-ID representation").  Every leaf
 * must hold at least r indices.  Synchronizes `stream` once at the end.
 */
hm_status hm_compress_hbs(const hm_operator* op, const hm_tree* tree, const hm_opts* opts,
                          void* stream, hm_handle** out);

/*
 * Batched compression of nops independent operators of uneven size and rank
 * (each the problem of Sec. 1 on its own): operator i with trees[i] and
 * opts[i] is compressed exactly as hm_compress_hodlr (format HM_FORMAT_HODLR)
 * or hm_compress_hbs (format HM_FORMAT_HBSID) would, and outs[i] receives its
 * handle, equal bit for bit to the one-call result.  HODLR: level by level from
 * the calling thread (the loop over the boxes of a level in the HODLR figure of
 * Sec. 3 taken across operators): each level's black-box products and peels
 * run per operator on max_concurrency internal streams (0: 8), and each TSQR
 * round and the panel SVD of the level run as one launch over the nodes of
 * every HM_A32 operator.  HBS-ID: one hm_compress_hbs per operator, from up to
 * max_concurrency host threads (0: 8), so the black boxes are called from
 * several threads at once and must allow it (the dense operators of this
 * library do, one operator per entry).  The internal streams start after the
 * work already queued on `stream`; all work is complete when the call returns.
 * Trees may be shared between operators.  On the first failure every handle of
 * the call is destroyed, outs[] is set to NULL and the error names the
 * operator.
 */
hm_status hm_compress_batched(int32_t nops, const hm_operator* ops, hm_tree* const* trees,
                              const hm_opts* opts, int32_t format, int32_t max_concurrency,
                              void* stream, hm_handle** outs);

/*
 * Autotuner of hm_compress_batched's concurrency (no counterpart in the paper:
 * a launch schedule, not a step of the method).  The handles of a batch do
 * not depend on max_concurrency (the same kernels on the same nodes), only its
 * time does, and the best value depends on the batch (operator sizes, ranks,
 * depths) and on the device.  Runs the batch once to warm up, then once per
 * candidate (candidates[0 .. ncand-1], each >= 1), timing each call on the host
 * from a synchronized start to its return, destroys the handles, and writes
 * the fastest candidate to *best and the time of each candidate in ms to
 * ms_out[0 .. ncand-1] (ms_out may be NULL).  Errors as hm_compress_batched.
 */
hm_status hm_tune_batched(int32_t nops, const hm_operator* ops, hm_tree* const* trees,
                          const hm_opts* opts, int32_t format, const int32_t* candidates,
                          int32_t ncand, void* stream, int32_t* best, double* ms_out);

/* ---------------------------------------------------------- using it ----- */

/*
 * Y = A_c X (trans = 0) or A_c^T X (trans = 1) for the compressed A_c: the
 * HODLR product of Sec. 2.8 (block diagonal plus every sibling block), or the
 * HBS / HBS-ID product of Fig. "Application of A^(m) in the HBS framework"
 * with m = L plus the leaf blocks.  X, Y: device, column-major, n x ncols,
 * element type of the handle's precision.  X and Y must not overlap.
 */
hm_status hm_apply(const hm_handle* h, int trans, int64_t ncols, const void* X, int64_t ldx,
                   void* Y, int64_t ldy, void* stream);

/*
 * Same product with HOST buffers: copies X to the device, applies, copies Y
 * back, and synchronizes the stream before returning.  Scratch is allocated
 * and released inside the call.
 */
hm_status hm_apply_host(const hm_handle* h, int trans, int64_t ncols, const void* X_host,
                        int64_t ldx, void* Y_host, int64_t ldy, void* stream);

/*
 * Dense block A_c(r0:r1, c0:c1) of the compressed matrix written to `out`
 * (device, column-major, ld >= r1 - r0, handle's element type).
 * 0 <= r0 <= r1 <= n, 0 <= c0 <= c1 <= n.
 */
hm_status hm_reconstruct_block(const hm_handle* h, int64_t r0, int64_t r1, int64_t c0,
                               int64_t c1, void* out, int64_t ld, void* stream);

/*
 * ||A - A_c||_F / ||A||_F for a dense row-major device matrix A (dtype 0 =
 * double, 1 = float), streamed tile by tile with FP64 accumulation (Sec. 5
 * error measure; no N x N scratch).  Writes the result to *err (host) and
 * synchronizes the stream.
 */
hm_status hm_rel_frob_error(const hm_handle* h, const void* A, int64_t lda, int32_t dtype,
                            double* err, void* stream);

/*
 * Copies the HODLR factors of node level `level` (1..L): U gets U_a B_ab for
 * every node a of the level (the sibling matrix absorbed into the column
 * basis), V gets V_a; both n x r, column-major (ld n), rows I_a of node a,
 * columns past the block's rank zero.  A_c(I_a, I_b) = U(I_a,:) V(I_b,:)^T for
 * siblings a, b (Sec. 2.8).  Device buffers of the handle's element type.
 */
hm_status hm_hodlr_export_level(const hm_handle* h, int32_t level, void* U, void* V,
                                void* stream);

/*
 * Phase profile of a compression (the time split of Sec. 5's tables, T_net
 * against the black box, refined per level and phase).  With profiling on
 * (process-wide, hm_set_profiling(1)), the compress calls record a CUDA event
 * at the start of every phase of every level and side, and the handle keeps
 * one segment per phase: node level `level` (0 .. L - 1 for the sweeps, L for
 * the identity probe), side 0 (samples of A) or 1 (samples of A^T), phase, and
 * its device time in ms.  hm_profile copies up to cap segments to `out` (host)
 * and writes the total count to *count.  Profiling adds a few hundred events
 * per compression; off by default.
 */
typedef enum {
  HM_PHASE_SAMPLE = 0,  /* test matrix, black-box calls, non-finite check */
  HM_PHASE_PEEL = 1,    /* subtraction of A^(l) Omega (partial apply) */
  HM_PHASE_TSQR = 2,    /* Householder QR of the sample panels */
  HM_PHASE_SVD = 3,     /* SVD of the panels' R factors and the rank decision */
  HM_PHASE_ORTH = 4,    /* bases from the SVD (Q = P T1), CholQR pass */
  HM_PHASE_BASES = 5,   /* gathers, scatters, short bases, coefficient copies */
  HM_PHASE_ID = 6       /* HBS-ID upward sweep (interpolative decompositions) */
} hm_phase;
typedef struct {
  int32_t level;
  int32_t side;
  int32_t phase;
  double ms;
} hm_phase_t;
hm_status hm_set_profiling(int32_t on);
hm_status hm_profile(const hm_handle* h, hm_phase_t* out, int32_t cap, int32_t* count);

/*
 * Fast direct solver for a HODLR handle (Sec. 1: fast inversion is what the
 * compressed formats are for).  With A^(j) the block-diagonal part of A_c on
 * the nodes of level j, A_c = D (I + W_L Z_L^T) ... (I + W_1 Z_1^T), where for a
 * parent with children a, b: W = diag((A^(j)|a)^{-1} U_a, (A^(j)|b)^{-1} U_b) and
 * Z^T = [[0, V_b^T], [V_a^T, 0]]; each factor is inverted by
 * Sherman-Morrison-Woodbury with a 2k x 2k matrix per parent.
 * hm_hodlr_factorize builds the factors (leaf inverses, W per level, the
 * Woodbury matrices; O(k N log N) device memory held by the handle, O(k^2 N
 * log^2 N) work; leaves of at most 256 points) and synchronizes the stream.
 * HM_ENONFINITE if a leaf block or a Woodbury matrix is singular to working
 * precision.  Calling it again recomputes the factors.
 */
hm_status hm_hodlr_factorize(hm_handle* h, void* stream);

/*
 * X = A_c^{-1} B (trans = 0) or A_c^{-T} B (trans = 1) for a factorized HODLR
 * handle; B, X device, column-major, n x ncols, the handle's element type.
 * O(k N log N) per column.  HM_EINVAL if the handle is not factorized.
 */
hm_status hm_solve(const hm_handle* h, int trans, int64_t ncols, const void* B, int64_t ldb,
                   void* X, int64_t ldx, void* stream);

/*
 * Black box built from compressed handles (Sec. 5.2: operators such as the
 * Neumann-to-Dirichlet map S (I/2 + D)^{-1} are compressed by peeling the
 * product through its factors' fast applies and solves; Sec. 1: sums and
 * products of rank-structured matrices).  The operator is
 *   op(X) = alpha F_0 F_1 ... F_{nf-1} X + shift X,
 * where F_i is, by kinds[i], handles[i] (HM_FACTOR_APPLY), its transpose
 * (HM_FACTOR_TRANSPOSE), its inverse (HM_FACTOR_SOLVE) or its inverse
 * transpose (HM_FACTOR_SOLVE_TRANSPOSE; the solves need a HODLR handle
 * factorized by hm_hodlr_factorize).  Its transpose is applied exactly
 * (reversed order, transposed factors), so it can be compressed like any black
 * box.  All handles have the same n and element type (double: HM_FP64 and
 * HM_A32, float: HM_MIXED); they are referenced, not copied, and must outlive
 * the operator.  Each apply takes two n x ncols temporaries from the stream's
 * memory pool.  Release with hm_product_operator_destroy.
 */
typedef enum {
  HM_FACTOR_APPLY = 0,
  HM_FACTOR_TRANSPOSE = 1,
  HM_FACTOR_SOLVE = 2,
  HM_FACTOR_SOLVE_TRANSPOSE = 3
} hm_factor_kind;
hm_status hm_product_operator_create(int32_t nf, const hm_handle* const* handles,
                                     const int32_t* kinds, double alpha, double shift,
                                     hm_operator* out);
void hm_product_operator_destroy(hm_operator* op);

/*
 * Checkpoint of a compressed handle (HODLR or HBS-ID): hm_save writes the
 * representation (its device arrays copied to the host, behind a header with
 * the tree, rank and precision data and an FNV-1a checksum of the payload) to
 * `path` (synchronizes the device); hm_load reads it back and builds an
 * equivalent handle on the current device (the applies, reconstructions and
 * infos of the loaded handle equal the saved one's bit for bit).  Solver
 * factors are not stored: call hm_hodlr_factorize after loading.  hm_load
 * returns HM_EINVAL for a file that is not a complete, uncorrupted checkpoint.
 * The format is this library version's: native byte order and struct layout.
 */
hm_status hm_save(const hm_handle* h, const char* path);
hm_status hm_load(const char* path, void* stream, hm_handle** out);

/* Summary of the representation (ranks, black-box column counts, bytes M). */
hm_status hm_info(const hm_handle* h, hm_info_t* out);
/* Rank of the sibling block (node, node ^ 1) (HODLR) or of node's basis (HBS,
 * HBS-ID incoming skeleton).  Synchronous small read. */
hm_status hm_node_rank(const hm_handle* h, int64_t node, int32_t* rank);
/*
 * Skeleton index set of an HBS-ID node (Sec. 4.3: the row skeleton I~_tau of
 * the incoming interpolative decomposition, side 0, or the column skeleton
 * I^_tau of the outgoing one, side 1; B_skel = A(I~_alpha, I^_beta)).  Writes
 * the node's k global indices in [0, n), in the pivot order of its
 * interpolative decomposition, to idx[0 .. k) and -1 to idx[k .. r); idx is a
 * HOST buffer of at least r entries (r = hm_info's r).  2 <= node < 2^(L+1).
 * Synchronous (a small device-to-host copy); HM_EINVAL for other handles.
 */
hm_status hm_skeleton(const hm_handle* h, int64_t node, int32_t side, int64_t* idx, int32_t* k);
void hm_destroy(hm_handle* h);

/* ------------------------------------------- factored HODLR and adjoint --- */

/*
 * Factored HODLR apply with explicit factors (the HODLR product of Sec. 2.8
 * with sibling matrices B = I): for every level j = 1..L and sibling pair
 * (a, b) on level j, y(I_a) += U_j(I_a, :) (V_j(I_b, :)^T x(I_b)), plus
 * y(I_t) += D_t x(I_t) for every leaf t.
 *  U, V: device float, L blocks of N x k, column-major each (ld N), level j
 *        at offset (j - 1) * N * k.
 *  D:    device float, one n_max x n_max column-major block per leaf
 *        (ld n_max, entries beyond the leaf size are ignored).
 *  x, y: device float vectors of length N (y is overwritten).
 * trans = 1 applies H^T.  1 <= k <= 64.  Stream-ordered scratch as for the
 * adjoint below.  The per-leaf kernel keeps the leaf's slice of x in shared
 * memory: leaves too large for the device's per-block shared memory (about
 * 55k points on a GB300) return HM_EINVAL naming the sizes.
 */
hm_status hm_hodlr_factored_apply(const hm_tree* tree, int32_t k, const float* U,
                                  const float* V, const float* D, int trans, const float* x,
                                  float* y, void* stream);

/*
 * hm_hodlr_factored_apply without per-call device allocation (the paper has no
 * counterpart: this is an interface for callers, not a step of the method).
 * Same arguments, layouts and results as hm_hodlr_factored_apply, computed by
 * the same kernels; only the scratch differs.  For callers that cannot let the
 * library allocate device memory on each call: applications whose own
 * allocator has reserved the device memory (a per-call allocation from the
 * CUDA memory pool could then fail), or loops that must not touch the memory
 * pool at all.
 *  - Scratch: a fixed 8 MiB buffer compiled into the library (reserved on every
 *    device where the library's device code is loaded).  A call needs
 *    4 * k * (c + 2^(L+1)) bytes, c = the number of 256-row chunks over all
 *    nodes of levels 1..L (about L * N / 256); larger requests return
 *    HM_EINVAL naming the size, before anything is launched.
 *  - Nothing in the scratch needs to start at zero: every element a call reads
 *    is written earlier in the same call.
 *  - All calls on one device share the one buffer: two calls whose work may
 *    overlap (different streams, or different host threads, without ordering
 *    between them) race on it and give wrong results.  Order them on one
 *    stream or with events.
 *  - The first call on a device looks up the buffer's address
 *    (cudaGetSymbolAddress, with that device current) and caches it for the
 *    life of the process; make that first call before any stream capture.  A
 *    cudaDeviceReset of that device invalidates the cached address: do not
 *    call this entry point again in the same process after one.
 *  - The tree's index tables must already be on the current device (uploading
 *    them allocates): one call of hm_hodlr_factored_apply with this tree, on
 *    the same device, uploads them; otherwise (not uploaded, or uploaded to
 *    another device) HM_EINVAL.
 */
hm_status hm_hodlr_factored_apply_noalloc(const hm_tree* tree, int32_t k, const float* U,
                                          const float* V, const float* D, int trans,
                                          const float* x, float* y, void* stream);

/*
 * Hand-written adjoint (vector-Jacobian product) of y = H x at the factors
 * above.  Given r (device, length N), writes
 *   gx = scale * H^T r,            gU_j(I_a) = scale * r(I_a) (V_j(I_b)^T x(I_b))^T,
 *   gV_j(I_b) = scale * x(I_b) (U_j(I_a)^T r(I_a))^T,   gD_t = scale * r(I_t) x(I_t)^T
 * (same layouts as x, U, V, D; outputs are overwritten; any output may be NULL
 * to skip it; gD entries beyond a leaf's size are written as zero).  With
 * r = H x - b and scale = 2 these are the gradients of ||H x - b||^2.
 * Stream-ordered scratch of O(k * (N / 256 * L + 2^(L+1))) floats is taken
 * from the CUDA memory pool of the stream's device and released in order.
 * Leaves too large for the per-leaf kernel's shared memory (about 37k points
 * on a GB300) return HM_EINVAL naming the sizes.
 */
hm_status hm_hodlr_factored_adjoint(const hm_tree* tree, int32_t k, const float* U,
                                    const float* V, const float* D, const float* x,
                                    const float* r, float scale, float* gx, float* gU,
                                    float* gV, float* gD, void* stream);

/*
 * One training step of the factored HODLR form: the forward product, the
 * residual and the adjoint above at it, in one call,
 *   y = H x,  r = y - b,  then gx, gU, gV, gD exactly as hm_hodlr_factored_adjoint
 *   with this r (scale = 2: the gradients of ||H x - b||^2).
 * The forward's projections V_j(I_b)^T x(I_b) are the ones the adjoint needs, so
 * they are computed once: every factor is read twice per call (U, V and D by
 * the forward and by the adjoint), where the two separate calls read V three
 * times.  b: device, length N.  y, r: device outputs of length N, or NULL (then
 * kept in scratch).  Gradient outputs as in hm_hodlr_factored_adjoint (any may
 * be NULL).  Scratch of O(k * (N / 256 * L + 2^(L+1)) + 2 N) floats is taken
 * from the stream's CUDA memory pool and released in order.  Results equal the
 * two separate calls up to the summation order of the node projections
 * (FP32 rounding).  Errors as hm_hodlr_factored_adjoint.
 */
hm_status hm_hodlr_factored_loss_grad(const hm_tree* tree, int32_t k, const float* U,
                                      const float* V, const float* D, const float* x,
                                      const float* b, float scale, float* y, float* r,
                                      float* gx, float* gU, float* gV, float* gD, void* stream);

/* ------------------------------------------------------ workload helpers --- */

/*
 * Writes the FP32 log-kernel test operator: points x_i = (cos t_i, 0.5 sin t_i),
 * t_i = 2 pi i / n; A(i, j) = log |x_i - x_j| (FP64, rounded once to FP32),
 * A(i, i) = 1.  Row-major, device, lda >= n.  An input generator, not part of
 * the compression method.
 */
hm_status hm_gen_log_kernel(float* A, int64_t n, int64_t lda, void* stream);

/* Thread-local description of the last error ("" if none). */
const char* hm_last_error(void);
/* Library version string. */
const char* hm_version(void);
/* Number of CUDA kernels this library has launched in the process so far
 * (black-box GEMMs of the dense operator included). */
int64_t hm_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* HM_H_ */
