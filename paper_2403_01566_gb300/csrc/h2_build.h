// Host assembly of the input H^2-matrices (boundary of the library).
#pragma once
#include <stdint.h>

#include <vector>

namespace h2 {

struct Tree;
struct BlockTree;

// Numeric arrays of a Chebyshev H^2-matrix on the host (row-major):
//   V  n x k       leaf matrices stacked in cluster order (row and column basis)
//   E  ncl x k x k transfer matrices E_c (E_0 unused)
//   S  nadm x k x k coupling matrices in admissible-leaf order
//   N  dense nearfield blocks of the inadmissible leaves (BlockTree::near_off)
struct HostH2 {
  int k = 0;
  std::vector<double> V, E, S, N;
};

int tree_depth(int64_t n, int leaf);
double kernel_value(int kind, const double* kparam, const double* x, const double* y, int dim);
void assemble_chebyshev(const double* points, const Tree& T, const BlockTree& B, int order, int kind,
                        const double* kparam, HostH2& out);

// First-kind Chebyshev points of every cluster box (ncl x dim x order, axes
// narrower than 1e-6 of the root diagonal widened), shared by the host and the
// device assembly.
std::vector<double> chebyshev_nodes(const Tree& T, int order);

}  // namespace h2
