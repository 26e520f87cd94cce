// Internal declarations shared by the host orchestration and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/hm.h"

namespace hm {

// ------------------------------------------------------------ errors ------
void set_error(const std::string& msg);
const char* get_error();
void clear_error();

#define HM_CUDA_TRY(expr)                                                        \
  do {                                                                           \
    cudaError_t _e = (expr);                                                     \
    if (_e != cudaSuccess) {                                                     \
      ::hm::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));       \
      return HM_ECUDA;                                                           \
    }                                                                            \
  } while (0)

#define HM_TRY(expr)                    \
  do {                                  \
    hm_status _s = (expr);              \
    if (_s != HM_OK) return _s;         \
  } while (0)

hm_status check_launch(const char* what);
// Poll limit of the tensor-core GEMMs' pipeline waits (hm_set_wait_limit).
long long wait_limit();
// For a black box made by hm_dense_operator_create: reads and clears the flag
// its GEMMs raise when a bounded wait gave up (HM_ETIMEOUT if it was set).
// Other black boxes: HM_OK.  Synchronous (the caller has synchronized).
hm_status dense_take_timeout(const hm_operator* op);
// True for the black boxes the library makes itself (hm_dense_operator_create,
// hm_log_kernel_operator_create): they enqueue on the stream they are given and
// keep separate scratch per slot.
bool library_operator(const hm_operator* op);
// The product of a library black box with the scratch of `slot` (0 or 1); the
// callback's return convention (0 = enqueued).
int library_apply(const hm_operator* op, int slot, int trans, int64_t ncols, const void* X,
                  int64_t ldx, void* Y, int64_t ldy, cudaStream_t st);
// Process-wide count of kernels launched by the library (all devices).
void count_launches(int n);

// Raises a kernel's dynamic shared-memory limit, once per device, to all that one
// block may opt in to (`done` holds one bit per device).  The limit belongs to
// the function and is shared by every host thread: set per launch to that
// launch's own size, one thread could lower it between another thread's set and
// that thread's launch.  Occupancy still follows the size each launch asks for.
void raise_smem_limit(const void* func, std::atomic<uint32_t>& done);

// Row chunk of one tree node: rows [r0, r1) of node `node`.
struct Chunk {
  int32_t node;
  int32_t pad;
  int64_t r0;
  int64_t r1;
};

// TSQR task: Householder QR of up to two stacked sources.
//  kind 0: rows [r0, r1) of the panel;  kind 1: an R slot (c x c, row-major).
// rows of one leaf block of the TSQR (and the shared-memory tile of its QR)
constexpr int kTsqrRows = 128;

struct TsqrTask {
  int32_t node;      // heap id (for bookkeeping)
  int32_t nsrc;      // 1 or 2
  int32_t kind[2];
  int32_t out_slot;  // R slot written
  int32_t slot[2];   // source slots for kind 1
  int64_t r0[2];
  int64_t r1[2];
};

// One node's work item of a level-wide launch that spans several operators'
// compressions (hm_compress_batched): the block reads its pointers and panel
// width here instead of from the launch arguments, so that one launch covers
// every operator's nodes of a level with the same per-node arithmetic as the
// one-operator launches.
struct NodeJob {
  const TsqrTask* task;  // TSQR: the block's task (device memory)
  const double* P;       // TSQR first round: the panel (column-major, ld = ldp)
  double* R;             // TSQR: base of the R slots; SVD: the node's c x c R
  double* W;             // SVD: the node's c x c W slot
  double* sigma;         // SVD: the node's c singular values
  int64_t ldp;
  int32_t c;             // panel width
  int32_t pad;
};

// ------------------------------------------------------- launchers --------
// All launchers enqueue on `st` and return cudaSuccess-style status via
// check_launch; T is float (mixed) or double (FP64).

template <typename T>
void launch_gauss_fill(T* X, int64_t ldx, int64_t n, int r, int level, uint64_t seed,
                       bool bf16, const int64_t* d_start, int L, cudaStream_t st);

template <typename T>
void launch_identity_probe(T* X, int64_t ldx, int64_t n, int nmax, const int64_t* d_start,
                           int L, cudaStream_t st);

template <typename T>
void launch_dense_gemm(const T* A, int64_t lda, int trans, int64_t n, int64_t ncols,
                       const T* X, int64_t ldx, T* Y, int64_t ldy, uint8_t* flags,
                       cudaStream_t st);

size_t gemm_tc_smem_bytes();
int64_t gemm_tc_xs_elems(int64_t n, int64_t ncols);
bool gemm_tc_supported(const float* A, int64_t lda, int64_t n);
// FP32 operator x FP64 block on the tensor cores with exact integer accumulation
size_t gemm_esg_smem_bytes();
int64_t gemm_esg_work_bytes(int64_t n, int64_t ncols);
// row exponents then column exponents of A (2 n ints), taken once per operator
// Exponents of A per row and per column, each per window of 256 (n * nw ints
// each, nw = ceil(n / 256)): gemm_esg_exp_count(n) row entries, then as many
// column entries.
int64_t gemm_esg_exp_count(int64_t n);
void launch_esg_scales(const float* A, int64_t lda, int64_t n, int* aexp, cudaStream_t st);
int launch_gemm_esg(const float* A, int64_t lda, int trans, int64_t n, int64_t ncols,
                    const double* X, int64_t ldx, double* Y, int64_t ldy, void* work,
                    const int* aexp, uint8_t* flags, int* err, cudaStream_t st);
// 0: launched; 1: layout not supported (see gemm_tc_supported); 2: TMA map failed
int launch_gemm_tc(const float* A, int64_t lda, int trans, int64_t n, int64_t ncols,
                   const float* X, int64_t ldx, float* Y, int64_t ldy, void* xs_work,
                   uint8_t* flags, int* err, cudaStream_t st);

// Matrix-free log kernel of the ellipse (hm_log_kernel_operator_create): row
// exponents, a block of entries, and the sampling GEMM that forms the entries in
// registers from the tables S (n float pairs) and P (2n - 1 float pairs), high
// parts first.
void launch_logtab_rowexp(const float* S, const float* P, int64_t n, int* e_row, cudaStream_t st);
void launch_logtab_block(const float* S, const float* P, int64_t n, int64_t r0, int64_t r1,
                         int64_t c0, int64_t c1, float* out, int64_t ld, cudaStream_t st);
int launch_gemm_esg_gen(const float* S, const float* P, const int* rowexp, int64_t n,
                        int64_t ncols, const double* X, int64_t ldx, double* Y, int64_t ldy,
                        void* work, uint8_t* flags, int* err, cudaStream_t st);

void launch_dense_gemm_a32(const float* A, int64_t lda, int trans, int64_t n, int64_t ncols,
                           const double* X, int64_t ldx, double* Y, int64_t ldy, uint8_t* flags,
                           cudaStream_t st);

// Gram-like reduction: for every chunk, partial = A(rows, 0:ka)^T B(rows, 0:kb)
// (column offsets chosen by node parity), then per node sum of its chunks:
// out[node - node0] (ka x kb, column-major, ld ka) = sum.  df (T = double only): the
// products in double-float arithmetic on the FP32 pipe, inputs cut to 48 bits
// (~1e-14 relative; for HM_A32, whose operator is FP32, not for HM_FP64).
template <typename T>
void launch_seg_tn(const Chunk* chunks, int nchunks, const int32_t* chunk_begin, int nnodes,
                   int node0, const T* A, int64_t lda, int aoff_even, int aoff_odd, int ka,
                   const T* B, int64_t ldb, int boff_even, int boff_odd, int kb,
                   double* partial, T* out, cudaStream_t st, bool df = false);

// Expansion: Y(rows, yoff(node) + 0:kout) = alpha * P(rows, poff(node) + 0:kin) *
// C[(node ^ cflip) - node0] + beta * Y(...).  C is kin x kout column-major with
// stride cstride per node.  P may alias Y (rows are staged before writing).
template <typename T>
void launch_seg_nn(const Chunk* chunks, int nchunks, int node0, const T* P, int64_t ldp,
                   int poff_even, int poff_odd, int kin, const T* C, int64_t cstride, int cld,
                   int cflip, T* Y, int64_t ldy, int yoff_even, int yoff_odd, int kout, T alpha,
                   T beta, cudaStream_t st, bool df = false);

template <typename T>
void launch_tsqr(const TsqrTask* tasks, int ntasks, int merge, const T* P, int64_t ldp,
                 int c, T* R, cudaStream_t st);

// One-sided Jacobi SVD of the final R of every node: W (c x c col-major, sorted
// by descending sigma), sigma (c).  node_slot[i] = R slot of node node0 + i.
template <typename T>
void launch_jacobi(const int32_t* node_slot, int nnodes, const T* R, int c, T* W, T* sigma,
                   cudaStream_t st);

// The FP64-accurate SVD of k_jacobi_mp with its FP64 phases in double-float
// (HM_A32): same outputs, ~2^-46 relative accuracy.
// A TSQR round of an FP64 panel in double-float arithmetic (HM_A32): the row
// blocks (merge = 0) or the pairwise merges of the R factors (merge = 1).
void launch_tsqr_df(const TsqrTask* tasks, int ntasks, int merge, const double* P, int64_t ldp,
                    int c, double* R, cudaStream_t st);
void launch_jacobi_df(const int32_t* node_slot, int nnodes, const double* R, int c, double* W,
                      double* sigma, cudaStream_t st);
// The same two kernels over a list of node jobs (one block per job, each with
// its own panel, R slots and width; cmax = the largest width, which sizes the
// shared memory).
void launch_tsqr_df_jobs(const NodeJob* jobs, int njobs, int merge, int cmax, cudaStream_t st);
void launch_jacobi_df_jobs(const NodeJob* jobs, int njobs, int cmax, cudaStream_t st);

// Rank decision + T1 = W(:, :k) diag(1/sigma) (c x kcap, zero padded).
// mode 0: numerical range (sigma > floor * sigma1), at most kcap.
// mode 1: tolerance (sigma > eps_abs, with eps_abs computed at the first level
//         from the largest sigma1 as eps_scale * tol * nu), at most kcap.
// mode 2: fixed rank kfix (<= kcap).
template <typename T>
void launch_truncate(int nnodes, const T* W, const T* sigma, int c, int kcap, int mode,
                     int kfix, double tol_scaled, double* eps_abs, int set_eps, double floor_rel,
                     int32_t* rank, T* T1, int32_t* saturated, cudaStream_t st);

// CholQR pass: from G (k x k per node, Gram of Q1) compute R2 = chol(G) with
// dead-pivot guard, T2 = R2^{-1}; and M = T1-side coefficient W_k Sigma_k R2^T
// (c x kcap) when want_m != 0.
template <typename T>
void launch_cholqr(int nnodes, const T* G, int kcap, const int32_t* rank, T* T2,
                   const T* W, const T* sigma, int c, T* M, int want_m, cudaStream_t st);

// X'(i, probe(node) + j) = U(i, j) for j < r; the other r columns zero.
template <typename T>
void launch_scatter_probe(const T* U, int64_t ldu, T* X, int64_t ldx, int64_t n, int r,
                          int level_nodes, const int64_t* d_start, int L, cudaStream_t st);

// P(i, j) = Y(i, sample(node) + j), j < r.
template <typename T>
void launch_gather_sample(const T* Y, int64_t ldy, T* P, int64_t ldp, int64_t n, int r,
                          int level_nodes, const int64_t* d_start, int L, cudaStream_t st);

// D_t = Y(I_t, 0:n_t) for every leaf (D: one nmax x nmax col-major block per leaf).
template <typename T>
void launch_extract_diag(const T* Y, int64_t ldy, T* D, int nmax, const int64_t* d_start,
                         const int64_t* d_size, int L, cudaStream_t st);

// Y(I_t, :) += op(D_t) X(I_t, :) for every leaf.
template <typename T>
void launch_blockdiag_apply(const T* D, int nmax, int trans, const T* X, int64_t ldx, T* Y,
                            int64_t ldy, int64_t ncols, const int64_t* d_start,
                            const int64_t* d_size, int L, cudaStream_t st);

template <typename T>
void launch_fill(T* p, int64_t count, T v, cudaStream_t st);

// HODLR solver: inverses of a batch of n x n matrices held as [A | I] (n x 2n,
// column-major) in `work`, by Gauss-Jordan with partial pivoting.
template <typename T>
void launch_gauss_jordan(T* work, int batch, int n, T* out, int* singular, cudaStream_t st);
template <typename T>
void launch_gj_load_leaves(const T* D, int nmax, const int64_t* d_size, int L, T* work,
                           cudaStream_t st);
template <typename T>
void launch_gj_load_woodbury(const T* P, int r, int nparents, T* work, cudaStream_t st);
// Y = alpha A + beta B (column-major n x ncols; B unread when beta == 0)
template <typename T>
void launch_axpby(T* Y, int64_t ldy, T alpha, const T* A, int64_t lda, T beta, const T* B,
                  int64_t ldb, int64_t n, int64_t ncols, cudaStream_t st);

template <typename T>
void launch_copy_cols(const T* src, int64_t lds, T* dst, int64_t ldd, int64_t rows,
                      int64_t cols, cudaStream_t st);

// Y(:, j) = e_{c0 + j} restricted to rows (identity columns), n x w.
template <typename T>
void launch_identity_cols(T* Y, int64_t ldy, int64_t n, int64_t c0, int64_t w, cudaStream_t st);

// sum over tile of (A(i, c0 + j) - Ac(i, j))^2 and A^2 -> acc[0], acc[1] (atomic FP64)
template <typename T>
void launch_frob_tile(const T* A, int64_t lda, const T* Ac, int64_t ldc, int64_t n,
                      int64_t c0, int64_t w, double* acc, cudaStream_t st);

void launch_frob_tile_a32(const float* A, int64_t lda, const double* Ac, int64_t ldc, int64_t n,
                          int64_t c0, int64_t w, double* acc, cudaStream_t st);

int32_t nonfinite_check_launch(const void* p, int64_t count, int is_double, int32_t* flag,
                               cudaStream_t st);

void launch_gen_log_kernel(float* A, int64_t n, int64_t lda, cudaStream_t st);

struct FactChunk {
  int32_t level;
  int32_t node;
  int64_t r0;
  int64_t r1;
};

}  // namespace hm
struct hm_tree;
namespace hm {
size_t factored_scratch_bytes(const hm_tree* t, int k);
// Checks that the per-leaf kernels' shared memory fits the device (HM_EINVAL
// naming the sizes otherwise) and raises their limit once per device.
hm_status factored_check(const hm_tree* t, bool adjoint);
void launch_factored_apply(const hm_tree* t, int k, const float* U, const float* V,
                           const float* D, int trans, const float* x, float* y, float* scratch,
                           cudaStream_t st);
void launch_factored_adjoint(const hm_tree* t, int k, const float* U, const float* V,
                             const float* D, const float* x, const float* res, float scale,
                             float* gx, float* gU, float* gV, float* gD, float* scratch,
                             cudaStream_t st);
size_t factored_loss_grad_scratch_bytes(const hm_tree* t, int k);
void launch_factored_loss_grad(const hm_tree* t, int k, const float* U, const float* V,
                               const float* D, const float* x, const float* b, float scale,
                               float* y, float* res, float* gx, float* gU, float* gV, float* gD,
                               float* scratch, cudaStream_t st);

}  // namespace hm

namespace hm {
// Device work plan of one node level: row chunks for the segmented kernels and
// the TSQR merge schedule (row blocks first, then pairwise R merges).
struct LevelPlan {
  int nnodes = 0, node0 = 0;
  int n_tn = 0, n_nn = 0;
  std::vector<std::vector<TsqrTask>> tsqr_rounds;
  std::vector<int32_t> final_slot;
  int nslots = 0;
  std::vector<Chunk> tn, nn;
  std::vector<int32_t> tn_begin;
  void* dev = nullptr;
  const Chunk* d_tn = nullptr;
  const int32_t* d_tn_begin = nullptr;
  const Chunk* d_nn = nullptr;
  std::vector<const TsqrTask*> d_rounds;
  const int32_t* d_final_slot = nullptr;
};
int64_t dense_flags_bytes(int64_t n, int64_t ncols, int is_double);
}  // namespace hm

// ----------------------------------------------------------- objects --------
struct hm_tree {
  int64_t n = 0;
  int32_t leaf = 0;
  int32_t L = 0;
  std::vector<int64_t> start, size;  // indexed by heap id, length 2^(L+1)
  int64_t* d_start = nullptr;        // device copies
  int64_t* d_size = nullptr;
  int64_t nmax = 0;
  int32_t dev = -1;                  // device the tables were uploaded to
  std::vector<hm::LevelPlan> plans;  // index = node level (1..L)
  // 256-row chunks of every node of levels 1..L, level-major (heap-id order),
  // and the first chunk of every heap id (fbegin[2^(L+1)] = n_fchunks)
  std::vector<hm::FactChunk> fchunks;
  std::vector<int32_t> fbegin;
  void* fdev = nullptr;
  const hm::FactChunk* d_fchunks = nullptr;
  const int32_t* d_fbegin = nullptr;
  int n_fchunks = 0;
};

struct hm_dense_ctx {
  const void* A = nullptr;
  int64_t n = 0, lda = 0;
  int32_t dtype = 0;
  // Per-call scratch, one set per slot: slot 0 serves hm_dense_apply and the
  // callback, slot 1 the look-ahead stream of a compression, so that the two
  // products of one compression that overlap on the GPU never share scratch.
  uint8_t* flags = nullptr;  // zero-tile flags scratch
  int64_t flags_bytes = 0;
  void* xs = nullptr;        // split copy of X for the tensor-core engine
  int64_t xs_bytes = 0;
  uint8_t* flags1 = nullptr;  // slot 1 (allocated on its first use)
  void* xs1 = nullptr;
  int64_t xs1_bytes = 0;
  int* err = nullptr;        // device flag raised by a kernel that gave up waiting
  int* aexp = nullptr;       // dtype 4 / 5: row (then column) exponents of A per 256-wide window
  float* tabS = nullptr;     // dtype 5 (matrix-free log kernel): S[|i - j|] and P[i + j]
  float* tabP = nullptr;
};

struct hm_handle {
  int32_t format = 0;
  int32_t prec = 0;
  int64_t n = 0;
  int32_t L = 0;
  int32_t r = 0;
  hm_tree tree;  // own copy (device node table owned too)
  // HODLR factors (element type by prec): level j in [1, L] at offset (j-1)*n*r
  void* U = nullptr;  // U_j B_j (absorbed sibling matrix), n x r per level
  void* V = nullptr;  // V_j, n x r per level
  void* D = nullptr;  // leaves x nmax x nmax
  std::vector<int32_t> rank;  // per heap id
  // HBS-ID factors (host-built offsets into device arrays)
  void* hbs_store = nullptr;
  int64_t hbs_bytes = 0;
  std::vector<int64_t> tin_off, tout_off, bsk_off;  // element offsets per heap id
  std::vector<int32_t> kin, kout;                   // ranks per heap id
  std::vector<int64_t> iin_off, iout_off;            // skeleton index offsets
  int64_t* skel = nullptr;                           // device skeleton indices
  hm_info_t info{};
  std::vector<hm_phase_t> prof;                      // phase profile (hm_profile)
  // HODLR solver (hm_hodlr_factorize): leaf inverses, W_j = (A^(j))^{-1} U_j per
  // level, Woodbury matrices M per parent; one device block
  void* solv = nullptr;
  int64_t solv_dinv = 0, solv_w = 0, solv_m = 0;  // element offsets
};
