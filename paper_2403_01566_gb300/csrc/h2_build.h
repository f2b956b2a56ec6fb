// Host construction of the cluster and block trees and the Chebyshev points
// of every cluster box (boundary of the library; the numeric assembly runs on
// the device, h2_assemble.cu).
#pragma once
#include <stdint.h>

#include <vector>

namespace h2 {

struct Tree;
struct BlockTree;

int tree_depth(int64_t n, int leaf);

// First-kind Chebyshev points of every cluster box (ncl x dim x order, axes
// narrower than 1e-6 of the root diagonal widened), shared by the host and the
// device assembly.
std::vector<double> chebyshev_nodes(const Tree& T, int order);

}  // namespace h2
