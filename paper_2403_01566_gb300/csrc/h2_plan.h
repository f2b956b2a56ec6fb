// Host planner: compiles one H^2 x H^2 product (or a matrix-vector product,
// a dense expansion, the explicit level bases) into a list of batched stages
// (see h2_ops.h).  Pure C++; the device upload and execution live in h2_api.cu.
#pragma once
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "h2_internal.h"
#include "h2_ops.h"

namespace h2 {

// What the planner needs to know about an operand: its trees, block tree,
// padded rank and the offsets (in doubles) of its arrays inside its arena.
struct MatDesc {
  const Tree* rows = nullptr;
  const Tree* cols = nullptr;
  const BlockTree* blocks = nullptr;
  int k = 0;
  int64_t off_V = 0, off_E = 0, off_W = 0, off_F = 0, off_S = 0, off_N = 0;
  int64_t off_VF = -1, off_WF = -1;
};

struct MulOptions {
  double eta = 2.0;      // admissibility of the target block tree
  double theta = 0.25;   // weight factor (Section 5.3)
  int max_rank = 0;      // cap of the adaptive ranks (storage padding of C)
  int precision = 0;     // 0 FP64 throughout; 1 FP32 contractions (accumulation and couplings);
                         // 2 compensated FP32 contractions (all GEMM stages);
                         // 3 tensor-core 5-slice contractions (all GEMM stages);
                         // 4 tensor-core 7-slice contractions on 64 x 64 stages,
                         //   compensated FP32 on the others
  bool hmatrix = false;  // H-matrix output: stop after agglomeration (no nested-basis recompression)
};

// Indices into the per-product parameter block (ExecCtx::scal[0..]).
// Indices of the per-product parameters: see ParamIdx in h2_ops.h.

struct Plan {
  std::vector<Stage> stages;
  std::vector<GemmOut> gout;
  std::vector<GemmTerm> gterm;
  std::vector<CopyJob> copy;
  std::vector<QrJob> qr;
  std::vector<QApplyJob> qap;
  std::vector<SvdJob> svd;
  std::vector<ScanJob> scan;
  std::vector<NormJob> norm;
  std::vector<int> idx;
  std::vector<int> slot_init;
  std::vector<double> konst;     // AR_K contents
  int64_t ws_len = 0;            // doubles
  int64_t fac_len = 0;           // doubles of the terminal-factor arena (placed after the workspace)
  int64_t mv_ox = 0, mv_oy = 0;  // matrix-vector plans: X and Y in the workspace
  // H-matrix output (MulOptions::hmatrix): per admissible leaf of the target
  // block tree (adm_list order) the factors L (|t| x w) and R (|r| x w) in the
  // product arena, zero-padded to the width cap w; their ranks go to the
  // product's integer array through rank_row_slot
  std::vector<int64_t> hm_off_L, hm_off_R;
  std::vector<int> hm_w;
  int nscal = PARAM_COUNT;       // scal/nrm entries (first PARAM_COUNT are parameters)
  int svd_maxrows = 1, svd_maxcols = 1;
  // product layout (valid for product plans)
  std::shared_ptr<BlockTree> cblocks;
  int kpad = 0;
  int64_t c_off_V = 0, c_off_E = 0, c_off_W = 0, c_off_F = 0, c_off_S = 0, c_off_N = 0, c_len = 0;
  std::vector<int> rank_row_slot, rank_col_slot;
  int nagg = 0;
  std::map<std::string, int64_t> stats;
  // device copies (h2_api.cu)
  void* d_blob = nullptr;
  DeviceJobs dj;
  int* d_slot_init = nullptr;
  int* d_idx = nullptr;
  double* d_konst = nullptr;
  ~Plan();
};

std::shared_ptr<Plan> make_product_plan(const MatDesc& X, const MatDesc& Y, const MulOptions& o);

// Explicit level bases: out[l][i] = V_t(i, :) of the level-l cluster t that
// contains row i, for l = 0..depth (arena `ar`, (depth+1) x n x k).
std::shared_ptr<Plan> make_levelbasis_plan(const Tree& T, int k, int ar, int64_t off_leaf,
                                           int64_t off_trans, int64_t off_out);

// Y = A X for nrhs right-hand sides: X (cluster order, row-major n x nrhs)
// at ws[mv_ox..), Y likewise at ws[mv_oy..).
std::shared_ptr<Plan> make_matvec_plan(const MatDesc& A, int nrhs = 1);

// Dense expansion in cluster order (row-major n_rows x n_cols) at ws[0..).
std::shared_ptr<Plan> make_dense_plan(const MatDesc& A);

// Dense expansion (cluster order, row-major, at ws[0..)) of an H-matrix
// product whose arena (AR_X) holds the nearfield at off_N (near_off layout)
// and the admissible factors at off_L / off_R (width w, row-major).
std::shared_ptr<Plan> make_hmatrix_dense_plan(const Tree& rows, const Tree& cols, const BlockTree& blocks,
                                              int64_t off_N, const std::vector<int64_t>& off_L,
                                              const std::vector<int64_t>& off_R, const std::vector<int>& w);

}  // namespace h2
