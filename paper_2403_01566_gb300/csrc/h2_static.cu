// h2_matvec_noalloc: an H^2 matrix-vector product that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA stream is
// being captured into a graph (allocation is not a capturable operation),
// latency-critical loops that must not enter the allocator, and hosts whose
// device memory is partitioned up front.  This entry point serves them.  Its
// intermediate coefficient vectors x^_s = W_s^* x|_s and y^_t live in one
// file-scope device array of fixed size; the block lists of the matrix travel
// as kernel parameters, so no schedule has to be uploaded either.
//
// The paper has no counterpart; this is a convenience of the library.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/h2.h"
#include "h2_internal.h"

namespace h2 {

// Static scratch: 2^20 doubles (8 MiB) per device that loads the library,
// held until process exit.  A product needs 2 * nclusters * k doubles of it.
constexpr int64_t NOALLOC_SCRATCH_DOUBLES = int64_t(1) << 20;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

namespace {

struct NfMat {
  const double* a;  // arena of the matrix
  int64_t off_V, off_E, off_W, off_F, off_S, off_N;
  int n, depth, k;
};

// Offset and size of cluster c of a complete balanced bisection tree
// (first child floor(|t|/2)); the walk mirrors the host construction.
__device__ void cluster_range(int c, int n, int& off, int& size) {
  int l = 0;
  while (((1 << (l + 1)) - 1) <= c) ++l;
  const int j = c - ((1 << l) - 1);
  off = 0;
  size = n;
  for (int bit = l - 1; bit >= 0; --bit) {
    const int h = size / 2;
    if ((j >> bit) & 1) {
      off += h;
      size -= h;
    } else {
      size = h;
    }
  }
}

__global__ void k_nf_zero(double* p, int64_t len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0.0;
}

// x^_c = W_c^* x|_c for the leaves
__global__ void k_nf_fwd_leaf(NfMat M, const double* x, double* xh) {
  const int c = ((1 << M.depth) - 1) + blockIdx.x;
  int off, size;
  cluster_range(c, M.n, off, size);
  for (int i = threadIdx.x; i < M.k; i += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < size; ++r) s = fma(M.a[M.off_W + (int64_t)(off + r) * M.k + i], x[off + r], s);
    xh[(int64_t)c * M.k + i] = s;
  }
}

// x^_c = sum_children F_ch^* x^_ch for the clusters of one level
__global__ void k_nf_fwd_up(NfMat M, int level, double* xh) {
  const int c = ((1 << level) - 1) + blockIdx.x;
  for (int i = threadIdx.x; i < M.k; i += blockDim.x) {
    double s = 0.0;
    for (int h = 0; h < 2; ++h) {
      const int ch = 2 * c + 1 + h;
      const double* F = M.a + M.off_F + (int64_t)ch * M.k * M.k;
      for (int j = 0; j < M.k; ++j) s = fma(F[(int64_t)j * M.k + i], xh[(int64_t)ch * M.k + j], s);
    }
    xh[(int64_t)c * M.k + i] = s;
  }
}

constexpr int NF_MAXE = 1536;  // block entries per parameter chunk (24 KB of kernel parameters)

struct NfChunk {
  int count;
  int t[NF_MAXE];
  int s[NF_MAXE];
  int64_t off[NF_MAXE];  // coupling (k x k) or nearfield block offset in the arena
};

// y^_t += sum S_ts x^_s over the chunk's blocks of row cluster t = blockIdx.x
// (one CTA per cluster scans the chunk: deterministic order, no atomics)
__global__ void k_nf_couple(NfMat M, const __grid_constant__ NfChunk C, const double* xh, double* yh) {
  const int t = blockIdx.x;
  for (int i = threadIdx.x; i < M.k; i += blockDim.x) {
    double s = yh[(int64_t)t * M.k + i];
    for (int e = 0; e < C.count; ++e) {
      if (C.t[e] != t) continue;
      const double* S = M.a + C.off[e];
      const double* xs = xh + (int64_t)C.s[e] * M.k;
      for (int j = 0; j < M.k; ++j) s = fma(S[(int64_t)i * M.k + j], xs[j], s);
    }
    yh[(int64_t)t * M.k + i] = s;
  }
}

// y^_c += E_c y^_parent for the clusters of one level
__global__ void k_nf_bwd(NfMat M, int level, double* yh) {
  const int c = ((1 << level) - 1) + blockIdx.x;
  const int p = (c - 1) / 2;
  const double* E = M.a + M.off_E + (int64_t)c * M.k * M.k;
  for (int i = threadIdx.x; i < M.k; i += blockDim.x) {
    double s = yh[(int64_t)c * M.k + i];
    for (int j = 0; j < M.k; ++j) s = fma(E[(int64_t)i * M.k + j], yh[(int64_t)p * M.k + j], s);
    yh[(int64_t)c * M.k + i] = s;
  }
}

// y|_t = V_t y^_t for the leaves
__global__ void k_nf_leaf(NfMat M, const double* yh, double* y) {
  const int c = ((1 << M.depth) - 1) + blockIdx.x;
  int off, size;
  cluster_range(c, M.n, off, size);
  for (int r = threadIdx.x; r < size; r += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < M.k; ++j) s = fma(M.a[M.off_V + (int64_t)(off + r) * M.k + j], yh[(int64_t)c * M.k + j], s);
    y[off + r] = s;
  }
}

// y|_t += sum N_ts x|_s over the chunk's blocks of leaf t = first leaf + blockIdx.x
__global__ void k_nf_near(NfMat M, const __grid_constant__ NfChunk C, const double* x, double* y) {
  const int t = ((1 << M.depth) - 1) + blockIdx.x;
  int to, ts;
  cluster_range(t, M.n, to, ts);
  for (int r = threadIdx.x; r < ts; r += blockDim.x) {
    double s = y[to + r];
    for (int e = 0; e < C.count; ++e) {
      if (C.t[e] != t) continue;
      int so, ss;
      cluster_range(C.s[e], M.n, so, ss);
      const double* N = M.a + C.off[e];
      for (int j = 0; j < ss; ++j) s = fma(N[(int64_t)r * ss + j], x[so + j], s);
    }
    y[to + r] = s;
  }
}

constexpr int NF_MAXDEV = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[NF_MAXDEV] = {};  // per device, set up once

}  // namespace
}  // namespace h2

using namespace h2;

extern "C" int h2_matvec_noalloc(const h2_matrix* A, const double* x, double* y, void* stream) {
  if (!A || !x || !y) return H2_EINVAL;
  const Tree& R = *A->rows;
  const int k = A->kpad;
  if (A->cols.get() != A->rows.get() && (A->cols->n != R.n || A->cols->depth != R.depth)) return H2_EINVAL;
  if (2 * (int64_t)R.ncl * k > NOALLOC_SCRATCH_DOUBLES) return H2_ENOMEM;  // beyond the static scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= NF_MAXDEV) return H2_ECUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // once per device, with that device current: device address of the
      // static array (its host-side name is only a stand-in)
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return H2_ECUDA;
      g_noalloc_ptr[dev] = (double*)p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  if (A->done && cudaEventSynchronize(A->done) != cudaSuccess) return H2_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const NfMat M{A->d_arena, A->off_V, A->off_E, A->off_W, A->off_F, A->off_S, A->off_N, R.n, R.depth, k};
  double* xh = scratch;
  double* yh = scratch + (int64_t)R.ncl * k;
  const int D = R.depth;
  // the scratch keeps the previous call's contents: y^ must start at zero
  k_nf_zero<<<64, 256, 0, st>>>(yh, (int64_t)R.ncl * k);
  k_nf_fwd_leaf<<<1 << D, 64, 0, st>>>(M, x, xh);
  for (int l = D - 1; l >= 0; --l) k_nf_fwd_up<<<1 << l, 64, 0, st>>>(M, l, xh);
  const BlockTree& B = *A->blocks;
  static thread_local NfChunk C;  // parameters staged on the host, no allocation
  for (size_t i0 = 0; i0 < B.adm_list.size(); i0 += NF_MAXE) {
    C.count = (int)std::min<size_t>(NF_MAXE, B.adm_list.size() - i0);
    for (int e = 0; e < C.count; ++e) {
      const int b = B.adm_list[i0 + e];
      C.t[e] = B.t[b];
      C.s[e] = B.s[b];
      C.off[e] = A->off_S + (int64_t)(i0 + e) * k * k;
    }
    k_nf_couple<<<R.ncl, 64, 0, st>>>(M, C, xh, yh);
  }
  for (int l = 1; l <= D; ++l) k_nf_bwd<<<1 << l, 64, 0, st>>>(M, l, yh);
  k_nf_leaf<<<1 << D, 128, 0, st>>>(M, yh, y);
  for (size_t i0 = 0; i0 < B.inadm_list.size(); i0 += NF_MAXE) {
    C.count = (int)std::min<size_t>(NF_MAXE, B.inadm_list.size() - i0);
    for (int e = 0; e < C.count; ++e) {
      const int b = B.inadm_list[i0 + e];
      C.t[e] = B.t[b];
      C.s[e] = B.s[b];
      C.off[e] = A->off_N + B.near_off[i0 + e];
    }
    k_nf_near<<<1 << D, 128, 0, st>>>(M, C, x, y);
  }
  return cudaGetLastError() == cudaSuccess ? H2_OK : H2_ECUDA;
}
