// Batched-operation descriptors shared by the host planner (h2_plan.cpp) and
// the sm_103a kernels (h2_kernels.cu).
//
// A product is compiled on the host into a list of stages; every stage is one
// kernel launch over a list of independent jobs of one kind (small GEMM chains,
// strided copies, Householder QR, Q application, one-sided Jacobi SVD with a
// rank decision, prefix sums of ranks).  Matrix sizes that the method decides
// on the device (adaptive ranks) are "dims" that read integer slots written by
// earlier stages, so the whole stage list is fixed per (X, Y) structure, runs
// without host synchronisation and can be captured in one CUDA graph.
//
// All matrices are FP64.  Unless a job says otherwise a matrix is row-major:
// element (i, j) of a matrix with leading dimension ld is at p[i*ld + j].
#pragma once
#include <stdint.h>

namespace h2 {

// AR_WS per-product workspace, AR_X / AR_Y the factors, AR_C the product,
// AR_K constants of the plan (identity matrices), AR_F the explicit factors of
// the terminal blocks (kept while the workspace of the accumulation phases is
// reused by the recompression phases).
enum Arena : int { AR_WS = 0, AR_X = 1, AR_Y = 2, AR_C = 3, AR_K = 4, AR_F = 5, AR_NONE = -1, AR_COUNT = 6 };

// value = c + slot[s1] + slot[s2] (s1/s2 < 0: absent), then, if mc >= 0,
// min(value, mc + slot[ms]) (ms < 0: absent).
struct Dim {
  int c, s1, s2;
  int mc = -1, ms = -1;
};

// address = base[arena] + off + slot[ds] * dm + slot[ds2] * dm2  (ds < 0: absent)
struct Ptr {
  int64_t off;
  int arena;
  int ds, dm;
  int ds2, dm2;
};

// out(m x n) = beta*out + sum_terms alpha * op(A)(m x k1) op(B)(k1 x k2) op(C)(k2 x n)
// (two-factor term when c.arena < 0: op(A)(m x k1) op(B)(k1 x n);
//  plain add when b.arena < 0: op(A)(m x n)).
struct GemmOut {
  Ptr o;
  int ldo;
  Dim m, n;
  int beta;   // 0: overwrite, 1: accumulate
  int t0, t1; // term range
  int clampn; // 1: n = min(n, 64) (a wider output is covered by further tiles)
};

struct GemmTerm {
  Ptr a, b, c;
  int lda, ldb, ldc;
  Dim k1, k2;
  int ta, tb, tc;
  double alpha;
  int scale_idx;  // >= 0: alpha *= scal[scale_idx]
};

// dst(i,j) = alpha*scal*(trans ? src(j,i) : src(i,j)), i < rows, j < cols
// (src.arena < 0: writes zeros).  Elements with rows <= i < zrows or
// cols <= j < zcols are set to zero.
struct CopyJob {
  Ptr src, dst;
  int lds, ldd;
  Dim rows, cols;
  Dim zrows, zcols;
  int trans;
  double alpha;
  int scale_idx;
};

// In-place Householder QR of the COLUMN-major matrix a (rows x cols, leading
// dimension lda): on exit the upper triangle holds R, the part below the
// diagonal the reflectors v (v_0 = 1 implicit) and tau[j] the factors.
// If r.arena >= 0 the cols x cols upper-triangular R is also written row-major
// to r (ldr); rows i >= q = min(rows, cols) are zero.
// keep = 0: only R is needed (the reflectors may be left unwritten, and R may
// differ from the full Householder R by the signs of its rows).
struct QrJob {
  Ptr a, tau, r;
  int lda, ldr;
  Dim rows, cols;
  int keep;
  // Column pivoting (largest remaining column norm first) when piv is set:
  // a P = Q R with P[:, j] = e_{piv[j]}; piv holds cols int32 (cols <= 256,
  // else the factorisation is unpivoted and piv the identity).  Used where an
  // SVD of R^T follows: its one-sided Jacobi then needs about half the sweeps.
  Ptr piv;
  // Layout of the R output (bits): 1 = columns back in the original order
  // (R P^T, with pivoting); 2 = transposed (r[c * ldr + i] = R(i, c)).
  int rmode;
  // Truncation of a pivoted QR at a noise floor (trunc_idx >= 0): the
  // factorisation stops at the first step j whose trailing columns hold a
  // squared Frobenius norm <= scal[trunc_idx] * ||a||_F^2; R keeps rows < j
  // (the rest zero), tau[j..] = 0, and j is written to slot[rank_slot]
  // (rank_slot >= 0; min(rows, cols) when the QR runs to the end).
  int trunc_idx;
  int rank_slot;
};

// out(rows x ncols) = H_0 H_1 ... H_{q-1} [Y; 0]  with the reflectors of a QrJob
// (Y is q x ncols row-major), i.e. the thin Q factor applied to Y.
struct QApplyJob {
  Ptr a, tau, y, out;
  int lda, ldy, ldo;
  Dim rows, q, ncols;
};

// One-sided Jacobi on the columns of M (rows x cols); M = src if !trans (src is
// row-major rows x cols) else M = src^T (src row-major cols x rows).
// Writes the singular values sorted descending (sig, cols entries), the left
// singular vectors U (rows x cols row-major, column j = u_j, zero for sigma_j=0)
// if u.arena >= 0, and a rank decision into slot[rank_slot]:
//   mode 0: none, 1: count(sigma > tol), 2: count(sigma > tol*sigma_0),
//   4: norm only.
// With norm_idx >= 0 (any mode) it also writes sigma_0 to nrm[norm_idx] and
// 1/sigma_0 (0 if sigma_0 == 0) to scal[norm_idx].
// The threshold is tol * scal[tol_idx] (tol alone if tol_idx < 0).
// A rank above cap sets the error flag (H2_ERANK) and is clamped to cap.
struct SvdJob {
  Ptr src, u, sig;
  int lds, ldu;
  Dim rows, cols;
  int trans;
  int mode;
  double tol;
  int tol_idx;
  int rank_slot;
  int cap;
  int norm_idx;
  // Row permutation of U (int32, rows entries, or none): row r of M's left
  // singular vectors is written to row piv[r] of U.  With M = R^T from a
  // pivoted QR of A (A P = Q R), this yields the singular vectors for A's
  // column order.
  Ptr piv;
};

// Spectral norm of the square matrix N (n x n, row-major): lambda_max(N^T N)
// by Householder tridiagonalisation and Sturm-sequence bisection (accurate to
// rounding relative to ||N||^2, unaffected by sign or rotation freedom of N's
// factors).  Writes sqrt(lambda_max) to nrm[norm_idx], its inverse (0 for a
// zero matrix) to scal[norm_idx].
struct NormJob {
  Ptr src;
  int lds;
  Dim n;
  int norm_idx;
};

// slot[out + i] = sum_{j < i} slot[in[j]] for i = 0..count (count+1 outputs);
// in[] lists slot indices (in the int index table at idx_off).
struct ScanJob {
  int idx_off;
  int count;
  int out;
};

enum StageKind : int { ST_GEMM = 0, ST_COPY = 1, ST_QR = 2, ST_QAPPLY = 3, ST_SVD = 4, ST_SCAN = 5, ST_NORM = 6 };

struct Stage {
  int kind;
  int64_t first;  // first job index in the kind's job array
  int count;      // number of jobs
  int tag;        // phase id, for profiling
  int smem;       // dynamic shared memory of the launch (SVD stages: largest job)
  int aux;        // GEMM stages: (largest m << 16) | largest n or inner width (0: 64, 64)
};

// Indices into the per-product parameter block (ExecCtx::scal[0..]).
// PARAM_SVD_FLOOR: squared relative noise floor of the Jacobi SVD (columns
// with ||m||^2 below it times ||M||_F^2 count as rounding noise: sigma = 0,
// never rotated); set per product from eps and the contraction precision.
// PARAM_SVD_SWEEPS: sweep cap of the Jacobi SVDs (values < 1: the default of
// 60); a job that reaches it sets the error flag -5 (H2_ENOCONV).
enum ParamIdx : int { PARAM_TOL_BASIS = 0, PARAM_TOL_AGG = 1, PARAM_SVD_FLOOR = 2, PARAM_SVD_SWEEPS = 3, PARAM_COUNT = 4 };

// Kernel parameters common to all stages.
// It lives in device memory (one control block per plan) so that a captured
// CUDA graph of the stage list can be replayed with new operand pointers.
struct ExecCtx {
  double* base[AR_COUNT];
  int* slot;
  double* scal;   // [0, PARAM_COUNT): parameters; then per-block 1/||G||
  double* nrm;    // per-block ||G||
  int* err;       // device error flag
  const int* idx; // int index table (scan inputs)
  int* out_int;   // product: ranks (rows, then columns) and error flag
  const int* rank_src;
  int nrank;
  int pad;
  int* svd_sweeps;  // per SVD job: sweeps executed (profiling)
};

// A segment of a batched launch (one launch over the jobs of several
// products): blocks / queue indices [start, start + count) run the jobs
// jobs[0 .. count) of the product whose control block is ctx.  In a chained
// GEMM launch (consecutive GEMM stages of many products in one persistent
// kernel fed by a work queue) a job first waits until counter wait_idx
// reaches wait_target (its product's previous stage is complete; -1: no
// wait) and, when done, increments counter done_idx (-1: none).  first = the
// segment's first job index in the product's job arrays.
struct BatchSeg {
  const ExecCtx* ctx;
  const void* jobs;
  const GemmTerm* terms;
  int start, count;
  int wait_idx, wait_target, done_idx;
  int first;
};

}  // namespace h2
