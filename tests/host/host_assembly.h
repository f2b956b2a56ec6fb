// Host FP64 assembly of a Chebyshev H^2-matrix (eq. (3): leaf bases, transfer
// matrices, couplings and dense nearfield blocks).  Test infrastructure for the
// CPU stage interpreter only: the library assembles its inputs on the device.
#pragma once
#include <stdint.h>

#include <vector>

#include "../../paper_2403_01566_gb300/csrc/h2_build.h"
#include "../../paper_2403_01566_gb300/csrc/h2_internal.h"

namespace h2host {

// Numeric arrays of a Chebyshev H^2-matrix on the host (row-major):
//   V  n x k       leaf matrices stacked in cluster order (row and column basis)
//   E  ncl x k x k transfer matrices E_c (E_0 unused)
//   S  nadm x k x k coupling matrices in admissible-leaf order
//   N  dense nearfield blocks of the inadmissible leaves (BlockTree::near_off)
struct HostH2 {
  int k = 0;
  std::vector<double> V, E, S, N;
};

double kernel_value(int kind, const double* kparam, const double* x, const double* y, int dim);
void assemble_chebyshev(const double* points, const h2::Tree& T, const h2::BlockTree& B, int order, int kind,
                        const double* kparam, HostH2& out);

}  // namespace h2host
