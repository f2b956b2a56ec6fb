// Host-side declarations of the batched kernels (h2_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "h2_ops.h"

namespace h2 {

constexpr int SVD_MAXDIM = 128;  // largest Jacobi SVD (rows and columns)
constexpr int GEMM_MAXTILE = 64; // largest GEMM output tile (rows and columns)

// Device copies of the job arrays of a stage list.
struct DeviceJobs {
  const GemmOut* gemm_out = nullptr;
  const GemmTerm* gemm_term = nullptr;
  const CopyJob* copy = nullptr;
  const QrJob* qr = nullptr;
  const QApplyJob* qapply = nullptr;
  const SvdJob* svd = nullptr;
  const ScanJob* scan = nullptr;
  const NormJob* norm = nullptr;
};

cudaError_t kernels_init();
size_t gemm_smem_bytes();
size_t svd_smem_bytes(int rows, int cols);
void launch_stage(const Stage& st, const ExecCtx* x, const DeviceJobs& j, size_t svd_smem, cudaStream_t s);
void launch_finalize(const ExecCtx* x, int nrank, cudaStream_t s);

}  // namespace h2
