// Device assembly of a Chebyshev H^2-matrix (h2_assemble.cu).
#pragma once
#include <cuda_runtime.h>

#include <string>

namespace h2 {

struct Tree;
struct BlockTree;

// Evaluates the leaf bases V (n x k), transfer matrices E (ncl x k x k),
// couplings S (nadm x k x k) and nearfield blocks N (BlockTree::near_off) of
// the Nystroem matrix of `points` (host, n x dim, original order) into device
// memory, in the layout of the host assembly.  Returns an H2_* code (err
// names the failing step); on return the stream has finished the work.
int assemble_device(const double* points, const Tree& T, const BlockTree& B, int order, int kind,
                    const double* kparam, double* d_V, double* d_E, double* d_S, double* d_N, cudaStream_t st,
                    std::string& err);

}  // namespace h2
