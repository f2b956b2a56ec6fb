// Host-side declarations of the batched kernels (h2_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "h2_ops.h"

namespace h2 {

constexpr int SVD_MAXDIM = 256;  // largest Jacobi SVD (rows and columns)
constexpr int NORM_MAXN = 128;   // largest matrix of a spectral-norm job
constexpr int GEMM_AUX_FP32 = 1 << 24;  // Stage::aux flag of a GEMM stage: FP32 products and sums
constexpr int GEMM_AUX_DF = 1 << 25;    // Stage::aux flag of a GEMM stage: compensated FP32 (double-float)
constexpr int GEMM_AUX_TC5 = 1 << 26;   // Stage::aux flag: tensor cores, 5 BF16 slices (40 bits)
constexpr int GEMM_AUX_TC7 = 1 << 27;   // Stage::aux flag: tensor cores, 7 BF16 slices (about FP64)
constexpr int GEMM_AUX_FLAGS = GEMM_AUX_FP32 | GEMM_AUX_DF | GEMM_AUX_TC5 | GEMM_AUX_TC7;
// Dynamic shared memory of an SVD launch at most (the per-column arrays of a
// job, then its matrix when that fits).  76 KB: two CTAs on an SM, which
// leaves ~90 KB of L1 to the matrices that stay in global memory; a 72 KB cap
// (three CTAs, ~26 KB of L1) ran those 2.3x slower.
constexpr int SVD_SMEM_DOUBLES = 9732;
// SVD jobs needing at most this much shared memory (doubles, 40 KB) run in
// 128-thread CTAs, five per SM, when their stage also holds larger jobs
constexpr int SVD_SMALL_DOUBLES = 5120;

#ifdef __CUDACC__
#define H2_HOST_DEVICE __host__ __device__
#else
#define H2_HOST_DEVICE
#endif
// Per-column arrays of an SVD stage whose jobs have at most cmax columns, in
// doubles: nrm2, dsc, dinv, snorm (cmax each), rfa, rfb (cmax/2+1 each), spos
// and rlist (ints: cmax + cmax/2+1, two per double).  They precede the matrix
// area in the stage's dynamic shared memory.
H2_HOST_DEVICE constexpr int svd_colarr_doubles(int cmax) {
  return 4 * cmax + 2 * (cmax / 2 + 1) + (cmax + cmax / 2 + 2) / 2 + 1;
}
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

// Launch parameters of a GEMM stage from its Stage::aux: largest tile,
// compute mode, slices (tensor-core forms), kernel variant (outputs per thread
// or tiles per warp) and dynamic shared memory.
struct GemmShape {
  int mmax, nb, mode, slices, variant, smem;
};
GemmShape gemm_shape(int aux);

cudaError_t kernels_init();
size_t gemm_smem_bytes();
// kernel launches of a stage (an SVD stage of mixed job sizes takes two)
int stage_launches(const Stage& st);
void launch_stage(const Stage& st, const ExecCtx* x, const DeviceJobs& j, cudaStream_t s);
// One launch of stage kind/shape st over `total` jobs of several products
// (segments in device memory, sorted by start); scans are not batched.
void launch_stage_batched(const Stage& st, const BatchSeg* segs, int nseg, int total, cudaStream_t s);
// Persistent launch of a chain of GEMM stages: `grid` CTAs (at most the
// resident ones) take the `total` jobs from the queue ctr[0] (zeroed
// beforehand with the done counters).
void launch_gemm_batched(const GemmShape& g, const BatchSeg* segs, int nseg, int total, cudaStream_t s);
int gemm_chain_blocks_per_sm(const GemmShape& g);
void launch_gemm_chain(const GemmShape& g, int grid, const BatchSeg* segs, int nseg, int total, int* ctr,
                       cudaStream_t s);
void launch_finalize(const ExecCtx* x, int nrank, cudaStream_t s);

}  // namespace h2
