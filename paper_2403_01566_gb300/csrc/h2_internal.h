// Internal host-side data structures of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "h2_ops.h"
#include "h2_kernels.h"

namespace h2 {

// Cluster tree (Def. 1) built by cardinality-balanced bisection: a complete
// binary tree of depth `depth`, clusters numbered in level order (root 0,
// children of c are 2c+1 and 2c+2), leaves on level `depth`.
struct Tree {
  int n = 0, dim = 0, depth = 0, ncl = 0;
  std::vector<int64_t> perm;       // cluster order -> original index
  std::vector<int> off, size, level;
  std::vector<double> lo, hi;      // ncl x dim tight bounding boxes
  uint64_t hash = 0;               // structure hash (H2_ETREE check)
  static int first(int l) { return (1 << l) - 1; }
  static int child(int c, int i) { return 2 * c + 1 + i; }
  static int parent(int c) { return (c - 1) / 2; }
  bool leaf(int c) const { return level[c] == depth; }
  int count(int l) const { return 1 << l; }
};

// Block tree (Def. 2) of two trees of equal depth: every non-leaf block has the
// four children chil(t) x chil(s) (eq. (4) for same-level clusters).
struct BlockTree {
  std::vector<int> t, s;
  std::vector<signed char> adm;   // 1: admissible leaf, 0: inadmissible leaf, -1: inner
  std::vector<int> child0;        // first of four children, -1 for leaves
  std::vector<int> leafidx;       // leaves: index into adm_list / inadm_list
  std::vector<int> adm_list, inadm_list;
  std::vector<int64_t> near_off;  // inadmissible leaf -> offset of its dense block
  int64_t near_total = 0;
  std::unordered_map<int64_t, int> index;   // key(t, s) -> block
  uint64_t sig = 0;                         // structure hash of (t, s, adm) (FNV-1a)
  static int64_t key(int a, int b) { return ((int64_t)a << 32) | (uint32_t)b; }
  int find(int a, int b) const {
    auto it = index.find(key(a, b));
    return it == index.end() ? -1 : it->second;
  }
  bool is_leaf(int b) const { return child0[b] < 0; }
  bool is_adm(int b) const { return adm[b] == 1; }
  int child(int b, int i, int j) const { return child0[b] + 2 * i + j; }
};

void build_block_tree(const Tree& rows, const Tree& cols, double eta, BlockTree& out);
void build_cluster_tree(const double* points, int64_t n, int dim, int leaf_size, Tree& out);

struct Plan;

}  // namespace h2

// The opaque handle of the C ABI.
struct h2_matrix {
  int dim = 0;
  double eta = 0;
  int kpad = 0;                              // rank used for storage (input: k; product: max_rank)
  std::shared_ptr<h2::Tree> rows, cols;
  std::shared_ptr<h2::BlockTree> blocks;
  // One device arena with all numeric arrays (offsets in doubles).
  double* d_arena = nullptr;
  int64_t arena_len = 0;
  int64_t off_V = 0, off_E = 0, off_W = 0, off_F = 0, off_S = 0, off_N = 0;
  int64_t off_VF = -1, off_WF = -1;          // explicit level bases (depth+1) x n x kpad
  int* d_int = nullptr;                      // [rank_row ncl][rank_col ncl][err 1]
  int* d_perm = nullptr;                     // [rows perm n][cols perm n], made on first use
  bool same_basis = false;                   // W == V, F == E (Nystroem builds)
  int nagglomerated = 0;
  int launches = 0;
  int64_t workspace_bytes = 0;
  cudaEvent_t done = nullptr;                // completion of the product that made it
  cudaStream_t stream = nullptr;
  std::mutex mu;
  bool levels_ready = false;                 // explicit level bases computed
  uint64_t uid = 0;
};
