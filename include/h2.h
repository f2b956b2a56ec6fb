/*
 * h2.h -- C ABI of the GB300 (sm_103a) library for adaptive H^2-matrix
 * multiplication with block-relative error control.
 *
 * Method: S. Boerm, "Adaptive multiplication of H^2-matrices with
 * block-relative error control" (arXiv 2403.01566).  Given H^2-matrices
 * X (I x J) and Y (J x K) that share the cluster tree of J, h2_mul builds an
 * H^2-matrix C ~ X*Y with adaptively chosen isometric cluster bases such that
 * every admissible block b of C satisfies
 *     ||C_b - (XY)_b||_2 <= eps * ||(XY)_b||_2            (Sections 5.1-5.3)
 * and every inadmissible block is exact up to rounding.
 *
 * Conventions for every entry point:
 *   - All matrices handled by the library are FP64.
 *   - Vectors and dense matrices exchanged with the caller are in the caller's
 *     ORIGINAL point ordering; the library permutes internally.
 *   - Dense matrices are column-major n x n.
 *   - Handles are opaque, owned by the library, device resident, and released
 *     only by h2_free.  Inputs are never modified; one handle may be used by
 *     several concurrent h2_mul / h2_matvec calls.
 *   - Every call returns 0 (H2_OK) or a negative error code; no exception
 *     crosses the ABI.  A failed call leaves any output handle set to NULL.
 *   - All device work of a call runs on opts->stream when given, else on the
 *     library's own stream; calls with sync = 1 return after the work is done.
 */
#ifndef H2_GB300_H
#define H2_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define H2_OK 0
#define H2_EINVAL (-1)    /* invalid argument (n <= 0, dim not in 1..3, eps < 0, NaN, ...) */
#define H2_ETREE (-2)     /* X's column cluster tree differs from Y's row cluster tree */
#define H2_ENOMEM (-3)    /* device or host allocation failed */
#define H2_ETIMEOUT (-4)  /* a bounded device wait gave up */
#define H2_ENOCONV (-5)   /* a Jacobi SVD hit its sweep cap without converging */
#define H2_ECUDA (-6)     /* a CUDA runtime call failed (see h2_last_cuda_error) */
#define H2_ERANK (-7)     /* an adaptive rank exceeded h2_mul_opts.max_rank */
#define H2_ENOTREADY (-8) /* no CUDA device is available */

/* Kernel functions g(x,y) of the Nystroem matrices (Section 6 stand-ins):
 * kparam = {scale, diagonal value (entry i == j), width, unused}. */
#define H2_KERNEL_LOG 0   /* -scale * log|x-y|            */
#define H2_KERNEL_INV 1   /*  scale / |x-y|               */
#define H2_KERNEL_GAUSS 2 /*  scale * exp(-|x-y|^2/width) */
#define H2_KERNEL_EXP 3   /*  scale * exp(-|x-y|/width)   */

typedef struct h2_matrix h2_matrix;

/* Parameters of h2_build (Section 2).
 *   eta        admissibility  max(diam Omega_t, diam Omega_s) <= eta * dist(Omega_t, Omega_s)
 *              (eq. (2) of the paper with eta = 2*eta_paper), eta > 0
 *   leaf_size  maximal cluster size of a leaf, >= 2
 *   order      Chebyshev points per axis (eq. (3)); rank k = order^dim, 1..8
 *   kernel     H2_KERNEL_*;  kparam as above
 *   dim        spatial dimension of the points, 1..3 */
typedef struct {
  double eta;
  int leaf_size;
  int order;
  int kernel;
  double kparam[4];
  int dim;
} h2_build_opts;

/* Parameters of h2_mul (Sections 5.1-5.3).
 *   theta      weight factor of the block-relative error control, 0 < theta < 1/2
 *              (binary trees); 0 selects 1/4
 *   max_rank   cap on the adaptive ranks (storage padding of C), <= 64; 0 selects
 *              min(64, max(32, 2k))
 *   precision  0 = FP64 throughout;
 *              1 = FP32 contractions: the accumulation phases (basis products,
 *                  coupling and nearfield products, splits and pushes; Sections
 *                  3-4) and the coupling projection (Section 5.2) compute FP32
 *                  products with FP32 sums from the FP64 data; agglomeration,
 *                  condensation, QR, SVD, rank decisions and norms stay FP64.
 *                  Adds about 1e-7 relative rounding to each block; the bound
 *                  eps still holds for eps >= 1e-6, but the rounding sits above
 *                  the agglomeration tolerance and raises ranks.
 *              2 = compensated FP32 contractions in every GEMM stage: operands
 *                  split into FP32 hi + lo parts, error-free products and
 *                  compensated sums (about 1e-13 relative); QR, SVD, rank
 *                  decisions and norms stay FP64.
 *              3 = every GEMM stage on the tensor cores (mma BF16 operands,
 *                  FP32 accumulation) with 5 slices of 8 bits per operand
 *                  (row and column scaled per k chunk of 32; exact FP32 sums
 *                  of the slice products; compensated accumulation): 40 bits
 *                  relative to the chunk's row and column maxima.
 *              4 = the GEMM stages of 64 x 64 tiles on the tensor cores with
 *                  7 slices (56 bits: about FP64 accuracy), the smaller ones
 *                  as compensated FP32 (form 2); QR, SVD, rank decisions and
 *                  norms FP64 in forms 1-4.
 *              Forms 2-4 need the scaled operands within FP32's exponent
 *              range (about 1e-30 to 1e30).  Other values: H2_EINVAL.
 *   sync       1 = return after the product is complete and report device errors;
 *              0 = return after enqueueing (errors are reported by h2_check)
 *   stream     cudaStream_t to run on, or NULL for the library stream
 *   svd_max_sweeps  sweep cap of every Jacobi SVD of the product; 0 selects 60.
 *              A job that reaches the cap still completes (its singular values
 *              are those of the last sweep) and the product reports H2_ENOCONV. */
typedef struct {
  double theta;
  int max_rank;
  int precision;
  int sync;
  void* stream;
  int svd_max_sweeps;
} h2_mul_opts;

typedef struct {
  int64_t n;
  int dim;
  int depth;          /* leaves are on level `depth` */
  int nclusters;      /* clusters per tree */
  int nadm;           /* admissible leaves of the block tree */
  int ninadm;         /* inadmissible leaves */
  int kpad;           /* padded rank used for storage */
  int row_rank_min, row_rank_max, col_rank_min, col_rank_max;
  int nagglomerated;  /* admissible blocks of a product that needed agglomeration */
  int64_t device_bytes;
  int launches;       /* kernel launches of the product that made this matrix (0 for inputs) */
  int64_t workspace_bytes; /* device workspace of that product */
} h2_stats;

/* Build the H^2 approximation of the Nystroem matrix g(x_i, x_j) on `points`
 * (row-major n x dim, host memory, copied) by cardinality-balanced bisection
 * cluster trees, the admissibility block tree and tensor Chebyshev
 * interpolation (Def. 1-4, eq. (2)-(5)).  Row and column trees/bases coincide. */
int h2_build(const double* points, int64_t n, const h2_build_opts* opts, h2_matrix** out);

/* C ~ A*B with block-relative error eps in every admissible block (Sections 3-5).
 * A's column cluster tree must equal B's row cluster tree (H2_ETREE).
 * eps = 0 keeps every singular value (exact product up to rounding).
 * The result is a new handle; C's block tree is the admissibility block tree of
 * (A's row tree, B's column tree) with A's eta. */
int h2_mul(const h2_matrix* A, const h2_matrix* B, double eps, const h2_mul_opts* opts,
           h2_matrix** C);

/* Measurement helper (not part of the method): per kernel kind, the launches,
 * summed device time (CUDA events around every stage on the product's stream)
 * and the algorithmic work of one product computed like h2_mul.  Kinds:
 * 0 batched GEMM (every arithmetic mode), 1 copy, 2 Householder QR, 3 Q
 * application, 4 Jacobi SVD, 5 rank prefix sums, 6 finalize, 7 block norms,
 * 8 the tensor-core GEMM stages again (a subset of kind 0).  flops count the
 * FP64 operations of the algorithm with the ranks the device decided
 * (Householder QR 2mn^2 - 2n^3/3; one-sided Jacobi m n (n-1) + 2mn per
 * executed sweep plus 6m per applied rotation); for kind 8 they count the
 * multiply-adds issued to the tensor cores instead (2 x 16 x 8 x 16 per BF16
 * slice product of mma.sync m16n8k16, S(S+1)/2 of them per tile and k step,
 * padding included).  bytes are the algorithmic reads and writes of each job.
 * The stages run one by one (no graph).  `out` must hold H2_PROFILE_KINDS
 * entries.  The product is returned in *C. */
#define H2_PROFILE_KINDS 9
typedef struct {
  int launches;
  int jobs;
  double ms;
  double flops;
  double bytes;
} h2_kernel_prof;

int h2_mul_profile(const h2_matrix* A, const h2_matrix* B, double eps, const h2_mul_opts* opts,
                   h2_kernel_prof* out, h2_matrix** C);

/* Device error state of a product computed with sync = 0 (waits for it). */
int h2_check(const h2_matrix* C);

/* y = A x by the H^2 matrix-vector product of Section 2 (complexity O(nk)
 * stated there for Def. 4's representation): forward transform
 * x^_s = W_s^* x|_s up the column tree through the transfer matrices,
 * couplings y^_t += S_ts x^_s over the admissible leaves, backward transform
 * down the row tree, leaf bases, and the dense nearfield blocks.
 * x, y of length n (caller ordering); on_device = 1: both are device
 * pointers, else host pointers.  Runs on the library stream and synchronizes. */
int h2_matvec(const h2_matrix* A, const double* x, double* y, int on_device);

/* Y = A X for nrhs right-hand sides at once (Section 2: forward transform
 * x^_s = W_s^* x|_s up the column tree, couplings y^_t = sum_s S_ts x^_s,
 * backward transform down the row tree, leaf bases and nearfield), as
 * level-wise batched GEMMs with nrhs columns.
 *   X        n_cols x nrhs, column-major (vector j at X + j * n_cols), caller ordering
 *   Y        n_rows x nrhs, column-major, caller ordering (written)
 *   nrhs     1 .. 4096
 *   on_device  1: X and Y are device pointers; 0: host pointers (staged through
 *            the device; the call returns when Y is written)
 *   stream   cudaStream_t for the work, or NULL for the library stream (device
 *            pointers and a NULL stream: the call returns when Y is written;
 *            with a stream it returns after enqueueing)
 * Plans are cached per (matrix structure, nrhs).  Returns H2_EINVAL for null
 * pointers or nrhs out of range. */
int h2_matvec_batch(const h2_matrix* A, const double* X, double* Y, int nrhs, int on_device, void* stream);

/* ---- H-matrix output variant -------------------------------------------
 * C ~ A*B as a standard H-matrix (Section 5.1): the product is accumulated
 * and, where the induced block structure is finer than the target block tree,
 * agglomerated with the coarsening error control (eps_c = eps/3 per block),
 * exactly as in h2_mul; the nested-basis recompression (Sections 5.2-5.3) is
 * skipped.  Every admissible block keeps its own low-rank factors
 * C_b = L_b R_b^T (accumulated blocks rank 2k, agglomerated blocks the
 * truncated rank); inadmissible leaves are dense.  Same operands, options and
 * errors as h2_mul (opts->precision must be 0). */
typedef struct h2_hmatrix h2_hmatrix;
int h2_mul_h(const h2_matrix* A, const h2_matrix* B, double eps, const h2_mul_opts* opts, h2_hmatrix** C);

/* Dense n_rows x n_cols column-major expansion (caller ordering) into `out`
 * (host, or device when on_device = 1). */
int h2_hmatrix_to_dense(const h2_hmatrix* C, double* out, int on_device);

/* Ranks of the admissible blocks in block-tree leaf order (`ranks` holds
 * nadm ints); nadm, the largest rank and the device bytes are optional
 * outputs (NULL to skip). */
int h2_hmatrix_ranks(const h2_hmatrix* C, int* ranks, int* nadm, int* rank_max, int64_t* device_bytes);

void h2_hmatrix_free(h2_hmatrix* C);

/* ---- Serving: continuous batching of products ---------------------------
 * A server runs products C = A*B (h2_mul semantics) over operands the caller
 * keeps resident.  Requests queue in arrival order; a dispatcher thread admits
 * the oldest as soon as one of `slots` streams is free and the device memory
 * the request needs fits `mem_budget`: a further instance of its plan
 * (workspace, control block, graph) when all instances are busy, plus the
 * output.  Admitted products run concurrently, so requests that arrive while
 * others are on the GPU overlap with them.  Results are bitwise the same as
 * the same products run alone (same plan, same kernels).
 *   h2_server_create  slots 1..64; mem_budget in bytes (0: 90% of the free
 *                     device memory at creation)
 *   h2_server_submit  enqueues; opts->stream and opts->sync are ignored; A and
 *                     B must stay alive until the request is collected
 *   h2_server_wait    blocks until the request is done; returns C (free with
 *                     h2_free) and optionally the milliseconds from submit to
 *                     start and from submit to completion
 *   h2_server_destroy drops requests not yet started, waits for running ones,
 *                     frees uncollected results */
typedef struct h2_server h2_server;
int h2_server_create(int slots, int64_t mem_budget, h2_server** out);
int h2_server_submit(h2_server* s, const h2_matrix* A, const h2_matrix* B, double eps, const h2_mul_opts* opts,
                     int64_t* ticket);
int h2_server_wait(h2_server* s, int64_t ticket, h2_matrix** C, double* queued_ms, double* total_ms);
void h2_server_destroy(h2_server* s);

/* ---- Batching: many products in merged launches --------------------------
 * A batch holds nprod products C_i = A_i * B_i (h2_mul semantics, with the
 * shared opts and eps[i]; A_i, B_i must stay alive as long as the batch).  The
 * stage lists of all products (the level-by-level work of Sections 3-5) are
 * interleaved into one launch sequence: a launch serves the matching stage of
 * every product whose next stage it is, whatever the products' sizes, ranks
 * and block counts; runs of consecutive GEMM stages (the tree levels of the
 * basis products, of the accumulation and of the projections) become one
 * persistent launch whose CTAs take jobs of all products from a device work
 * queue, a job waiting (at most about a second, then H2_ETIMEOUT) until its
 * product's previous level is complete; the whole sequence is captured in one
 * CUDA graph.  Each product keeps its own workspace and plan, so every result
 * is bitwise the one h2_mul gives alone.
 *   h2_batch_create   plans, workspaces and results allocated, graph captured
 *   h2_batch_run      replays the batch on `stream` (NULL: library stream);
 *                     sync = 1 waits and returns the first error of a product
 *   h2_batch_result   the i-th result, owned by the batch: valid until the
 *                     batch is freed, overwritten by the next run
 *   h2_batch_info     launches per run (scans counted per product), persistent
 *                     chains among them, kernel launches of the last enqueue
 *   h2_batch_autotune times every GEMM launch of the batch with each kernel
 *                     variant (outputs per thread, tiles per warp) and, for
 *                     chains, CTAs per SM, pins the fastest per shape class in
 *                     a process-wide table used by batches created afterwards,
 *                     and re-captures this batch; the choices never change a
 *                     result (the arithmetic of a job does not depend on them)
 *   h2_tuning_table   the pinned table as text (returns its length)
 * h2_batch_opts.test_unreachable_wait = 1 makes the first chained job wait on
 * a counter nothing sets (tests of the bounded wait: the run returns
 * H2_ETIMEOUT after about a second and the batch remains usable). */
typedef struct h2_batch h2_batch;
typedef struct {
  int test_unreachable_wait;
} h2_batch_opts;
int h2_batch_create(int nprod, const h2_matrix* const* A, const h2_matrix* const* B, const double* eps,
                    const h2_mul_opts* opts, const h2_batch_opts* bopts, h2_batch** out);
int h2_batch_run(h2_batch* b, void* stream, int sync);
int h2_batch_result(const h2_batch* b, int i, const h2_matrix** C);
int h2_batch_info(const h2_batch* b, int* launches, int* chains, int* kernel_launches);
int h2_batch_autotune(h2_batch* b, int* ntuned);
int h2_tuning_table(char* buf, int len);
void h2_batch_free(h2_batch* b);

/* Dense n x n column-major expansion (caller ordering) into `out` (host or device). */
int h2_to_dense(const h2_matrix* A, double* out, int on_device);

/* Statistics; synchronizes. */
int h2_info(const h2_matrix* A, h2_stats* out);

/* Ranks of the row and column cluster bases per cluster, clusters in level
 * order (root first, children in order); each array holds nclusters ints. */
int h2_ranks(const h2_matrix* A, int* row_ranks, int* col_ranks);

/* Cluster-order permutation: perm[i] = original index of the i-th point. */
int h2_permutation(const h2_matrix* A, int64_t* perm);

/* y = A x without any allocation, for callers that cannot call cudaMalloc:
 * latency-critical loops that must stay out of the allocator (an allocation
 * can synchronise the device), and processes whose device memory is
 * partitioned up front (owned by another allocator, or a fixed budget with no
 * room left).  The paper has no counterpart: this is a convenience of the
 * library.
 *   x, y    DEVICE vectors of length n in the library's CLUSTER ordering
 *           (h2_permutation maps it to the caller's ordering) on the current
 *           device, like A's storage (else H2_EINVAL); y is overwritten
 *   stream  cudaStream_t to enqueue on (NULL: legacy default stream).  The
 *           call returns without waiting for the GPU; when A is a product
 *           still being computed, the stream waits for it on the device.
 * Scratch: one static device array of 2^20 doubles (8 MiB) in every process and
 * on every GPU that loads the library, held until exit.  A call needs
 * 2 * nclusters * kpad doubles of it and returns H2_ENOMEM beyond that.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress).  All calls share the array, which keeps the last
 * call's contents (each call clears what must start at zero): calls that
 * overlap on the GPU race, so serialise them (host threads are serialised by
 * the call itself). */
int h2_matvec_noalloc(const h2_matrix* A, const double* x, double* y, void* stream);

void h2_free(h2_matrix* A);

const char* h2_strerror(int code);

/* Text of the last CUDA error seen by the library (thread local). */
const char* h2_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* H2_GB300_H */
