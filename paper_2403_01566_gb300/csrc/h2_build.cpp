// Host-side construction of cluster trees, block trees and the Chebyshev
// H^2 approximation of a Nystroem kernel matrix (Section 2 of the paper:
// Def. 1-4, eq. (2)-(5)).  This is the boundary of the library (inputs are
// assembled once per matrix); the product itself runs on the GPU.
//
// Readings of the points the paper leaves open (also used by the oracle):
//   * Omega_t = tight axis-parallel bounding box of the cluster's points;
//     diam = box diagonal, dist = Euclidean box distance.
//   * Cardinality-balanced bisection along the longest box edge (stable sort
//     by that coordinate, first child floor(|t|/2) points); all clusters above
//     depth D = min{d : ceil(n/2^d) <= leaf} are split, so the tree is complete.
//   * admissible iff max(diam_t, diam_s) <= eta * dist(t, s).
//   * First-kind Chebyshev points per box axis (x fastest in the tensor index);
//     axes narrower than 1e-6 * root diagonal are widened for interpolation.
// Host code is compiled with -ffp-contract=off so that the geometric
// comparisons are bit-identical to the reference computation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "h2_build.h"
#include "h2_internal.h"

namespace h2 {

static double box_diam(const Tree& T, int c) {
  double acc = 0.0;
  for (int a = 0; a < T.dim; ++a) {
    const double g = T.hi[c * T.dim + a] - T.lo[c * T.dim + a];
    acc += g * g;
  }
  return std::sqrt(acc);
}

static double box_dist(const Tree& A, int t, const Tree& B, int s) {
  double acc = 0.0;
  for (int a = 0; a < A.dim; ++a) {
    const double g1 = B.lo[s * B.dim + a] - A.hi[t * A.dim + a];
    const double g2 = A.lo[t * A.dim + a] - B.hi[s * B.dim + a];
    const double g = std::max(0.0, std::max(g1, g2));
    acc += g * g;
  }
  return std::sqrt(acc);
}

int tree_depth(int64_t n, int leaf) {
  int d = 0;
  while (((n + (int64_t(1) << d) - 1) >> d) > leaf) ++d;
  return d;
}

void build_cluster_tree(const double* pts, int64_t n, int dim, int leaf, Tree& T) {
  T.n = (int)n;
  T.dim = dim;
  T.depth = tree_depth(n, leaf);
  T.ncl = (1 << (T.depth + 1)) - 1;
  T.perm.resize(n);
  for (int64_t i = 0; i < n; ++i) T.perm[i] = i;
  T.off.assign(T.ncl, 0);
  T.size.assign(T.ncl, 0);
  T.level.assign(T.ncl, 0);
  T.lo.assign((size_t)T.ncl * dim, 0.0);
  T.hi.assign((size_t)T.ncl * dim, 0.0);
  struct Item { int c, level; int64_t b, e; };
  std::vector<Item> stack{{0, 0, 0, n}};
  while (!stack.empty()) {
    Item it = stack.back();
    stack.pop_back();
    const int c = it.c;
    T.off[c] = (int)it.b;
    T.size[c] = (int)(it.e - it.b);
    T.level[c] = it.level;
    for (int a = 0; a < dim; ++a) {
      double lo = pts[T.perm[it.b] * dim + a], hi = lo;
      for (int64_t i = it.b; i < it.e; ++i) {
        const double v = pts[T.perm[i] * dim + a];
        lo = std::min(lo, v);
        hi = std::max(hi, v);
      }
      T.lo[c * dim + a] = lo;
      T.hi[c * dim + a] = hi;
    }
    if (it.level < T.depth) {
      int axis = 0;
      double best = T.hi[c * dim] - T.lo[c * dim];
      for (int a = 1; a < dim; ++a) {
        const double ext = T.hi[c * dim + a] - T.lo[c * dim + a];
        if (ext > best) {
          best = ext;
          axis = a;
        }
      }
      std::stable_sort(T.perm.begin() + it.b, T.perm.begin() + it.e,
                       [&](int64_t x, int64_t y) { return pts[x * dim + axis] < pts[y * dim + axis]; });
      const int64_t h = (it.e - it.b) / 2;
      // push second child first so that the first child is processed first
      stack.push_back({Tree::child(c, 1), it.level + 1, it.b + h, it.e});
      stack.push_back({Tree::child(c, 0), it.level + 1, it.b, it.b + h});
    }
  }
  // structure hash: permutation and sizes (FNV-1a)
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  mix((uint64_t)n);
  mix((uint64_t)T.depth);
  for (int64_t i = 0; i < n; ++i) mix((uint64_t)T.perm[i]);
  for (int c = 0; c < T.ncl; ++c) mix((uint64_t)T.size[c]);
  T.hash = h;
}

void build_block_tree(const Tree& R, const Tree& C, double eta, BlockTree& B) {
  B = BlockTree();
  struct Item { int b; };
  auto add = [&](int t, int s) {
    const int id = (int)B.t.size();
    B.t.push_back(t);
    B.s.push_back(s);
    B.adm.push_back(-1);
    B.child0.push_back(-1);
    B.leafidx.push_back(-1);
    B.index[BlockTree::key(t, s)] = id;
    return id;
  };
  std::vector<int> stack{add(0, 0)};
  while (!stack.empty()) {
    const int b = stack.back();
    stack.pop_back();
    const int t = B.t[b], s = B.s[b];
    const double dm = std::max(box_diam(R, t), box_diam(C, s));
    if (dm <= eta * box_dist(R, t, C, s)) {
      B.adm[b] = 1;
      B.leafidx[b] = (int)B.adm_list.size();
      B.adm_list.push_back(b);
      continue;
    }
    if (R.leaf(t) || C.leaf(s)) {  // trees of equal depth: both are leaves
      B.adm[b] = 0;
      B.leafidx[b] = (int)B.inadm_list.size();
      B.inadm_list.push_back(b);
      B.near_off.push_back(B.near_total);
      B.near_total += (int64_t)R.size[t] * C.size[s];
      continue;
    }
    const int c0 = add(Tree::child(t, 0), Tree::child(s, 0));
    add(Tree::child(t, 0), Tree::child(s, 1));
    add(Tree::child(t, 1), Tree::child(s, 0));
    add(Tree::child(t, 1), Tree::child(s, 1));
    B.child0[b] = c0;
    for (int i = 3; i >= 0; --i) stack.push_back(c0 + i);
  }
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  for (size_t b = 0; b < B.t.size(); ++b) {
    mix((uint64_t)B.t[b]);
    mix((uint64_t)B.s[b]);
    mix((uint64_t)(B.adm[b] + 1));
  }
  B.sig = h;
}

// ------------------------------------------------------------ Chebyshev ----
std::vector<double> chebyshev_nodes(const Tree& T, int order) {
  std::vector<double> nodes((size_t)T.ncl * T.dim * order, 0.0);
  const double rootdiag = box_diam(T, 0);
  const double minw = rootdiag > 0.0 ? 1e-6 * rootdiag : 1e-6;
  const double pi = 3.14159265358979323846;
  for (int c = 0; c < T.ncl; ++c)
    for (int a = 0; a < T.dim; ++a) {
      double lo = T.lo[c * T.dim + a], hi = T.hi[c * T.dim + a];
      if (hi - lo < minw) {
        const double mid = 0.5 * (lo + hi);
        lo = mid - 0.5 * minw;
        hi = mid + 0.5 * minw;
      }
      double* x = &nodes[((size_t)c * T.dim + a) * order];
      for (int nu = 0; nu < order; ++nu)
        x[nu] = 0.5 * (lo + hi) + 0.5 * (hi - lo) * std::cos((2.0 * nu + 1.0) * pi / (2.0 * order));
    }
  return nodes;
}

}  // namespace h2
