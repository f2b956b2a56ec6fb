// h2_matvec_noalloc: an H^2 matrix-vector product that allocates nothing.
//
// Some callers cannot call cudaMalloc: latency-critical loops that must not
// enter the allocator (an allocation can synchronise the device or wait on
// the driver), and processes whose device memory is partitioned up front
// (an allocator owned by another component, or a fixed memory budget that
// leaves no room for further allocations).  This entry point serves them.
// Its intermediate coefficient vectors x^_s = W_s^* x|_s and y^_t live in one
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

// Block entries of one launch, sorted by row cluster t (stable, so the
// entries of one t keep the order of the matrix's block lists).
struct NfChunk {
  int count;
  int t[NF_MAXE];
  int s[NF_MAXE];
  int64_t off[NF_MAXE];  // coupling (k x k) or nearfield block offset in the arena
};

// CTA e handles the run of entries that starts at e (entries e' >= e with the
// same t); CTAs whose entry is not the first of its run return at once.  The
// work is proportional to the blocks, the order fixed, and no atomics.
__device__ __forceinline__ bool nf_run_start(const NfChunk& C, int e) {
  return e < C.count && (e == 0 || C.t[e - 1] != C.t[e]);
}

// y^_t += sum S_ts x^_s over the chunk's run of blocks of row cluster t
__global__ void k_nf_couple(NfMat M, const __grid_constant__ NfChunk C, const double* xh, double* yh) {
  const int e0 = blockIdx.x;
  if (!nf_run_start(C, e0)) return;
  const int t = C.t[e0];
  for (int i = threadIdx.x; i < M.k; i += blockDim.x) {
    double s = yh[(int64_t)t * M.k + i];
    for (int e = e0; e < C.count && C.t[e] == t; ++e) {
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

// y|_t += sum N_ts x|_s over the chunk's run of blocks of leaf t
__global__ void k_nf_near(NfMat M, const __grid_constant__ NfChunk C, const double* x, double* y) {
  const int e0 = blockIdx.x;
  if (!nf_run_start(C, e0)) return;
  const int t = C.t[e0];
  int to, ts;
  cluster_range(t, M.n, to, ts);
  for (int r = threadIdx.x; r < ts; r += blockDim.x) {
    double s = y[to + r];
    for (int e = e0; e < C.count && C.t[e] == t; ++e) {
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

// True when p is device (or managed) memory that device dev can address as
// its own.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

// Host staging of the kernel parameters: static storage (no allocation, not
// thread-local), used under g_noalloc_mu.  Kernel parameters are copied at
// launch, so the buffers are free again once a launch call returns.
NfChunk g_chunk, g_sorted;
uint64_t g_keys[NF_MAXE];

// Entries of g_chunk sorted by row cluster into g_sorted, insertion order kept
// within a cluster: an in-place sort of the keys (t, position).
void sort_chunk() {
  const NfChunk& C = g_chunk;
  for (int e = 0; e < C.count; ++e) g_keys[e] = ((uint64_t)(uint32_t)C.t[e] << 32) | (uint32_t)e;
  std::sort(g_keys, g_keys + C.count);
  g_sorted.count = C.count;
  for (int e = 0; e < C.count; ++e) {
    const int i = (int)(g_keys[e] & 0xffffffffu);
    g_sorted.t[e] = C.t[i];
    g_sorted.s[e] = C.s[i];
    g_sorted.off[e] = C.off[i];
  }
}

}  // namespace
}  // namespace h2

using namespace h2;

extern "C" int h2_matvec_noalloc(const h2_matrix* A, const double* x, double* y, void* stream) {
  if (!A || !x || !y) return H2_EINVAL;
  const Tree& R = *A->rows;
  const int k = A->kpad;
  if (A->cols.get() != A->rows.get() && (A->cols->n != R.n || A->cols->depth != R.depth)) return H2_EINVAL;
  if (2 * (int64_t)R.ncl * k > NOALLOC_SCRATCH_DOUBLES) return H2_ENOMEM;  // beyond the static scratch
  cudaGetLastError();  // an error left by an earlier, unrelated call is not this call's
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= NF_MAXDEV) return H2_ECUDA;
  // the matrix and both vectors must live on the current device
  if (!on_device(A->d_arena, dev) || !on_device(x, dev) || !on_device(y, dev)) return H2_EINVAL;
  // one caller at a time on the host: the parameter staging buffers are shared
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    // once per device, with that device current: device address of the
    // static array (its host-side name is only a stand-in)
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return H2_ECUDA;
    g_noalloc_ptr[dev] = (double*)p;
  }
  double* scratch = g_noalloc_ptr[dev];
  cudaStream_t st = (cudaStream_t)stream;
  // a product still in flight: order the reads after it on the device (no host wait)
  if (A->done && cudaStreamWaitEvent(st, A->done, 0) != cudaSuccess) return H2_ECUDA;
#define NF_CHECK()                                          \
  do {                                                      \
    if (cudaGetLastError() != cudaSuccess) return H2_ECUDA; \
  } while (0)
  const NfMat M{A->d_arena, A->off_V, A->off_E, A->off_W, A->off_F, A->off_S, A->off_N, R.n, R.depth, k};
  double* xh = scratch;
  double* yh = scratch + (int64_t)R.ncl * k;
  const int D = R.depth;
  // the scratch keeps the previous call's contents: y^ must start at zero
  k_nf_zero<<<64, 256, 0, st>>>(yh, (int64_t)R.ncl * k);
  NF_CHECK();
  k_nf_fwd_leaf<<<1 << D, 64, 0, st>>>(M, x, xh);
  NF_CHECK();
  for (int l = D - 1; l >= 0; --l) {
    k_nf_fwd_up<<<1 << l, 64, 0, st>>>(M, l, xh);
    NF_CHECK();
  }
  const BlockTree& B = *A->blocks;
  NfChunk& C = g_chunk;
  for (size_t i0 = 0; i0 < B.adm_list.size(); i0 += NF_MAXE) {
    C.count = (int)std::min<size_t>(NF_MAXE, B.adm_list.size() - i0);
    for (int e = 0; e < C.count; ++e) {
      const int b = B.adm_list[i0 + e];
      C.t[e] = B.t[b];
      C.s[e] = B.s[b];
      C.off[e] = A->off_S + (int64_t)(i0 + e) * k * k;
    }
    sort_chunk();
    k_nf_couple<<<C.count, 64, 0, st>>>(M, g_sorted, xh, yh);
    NF_CHECK();
  }
  for (int l = 1; l <= D; ++l) {
    k_nf_bwd<<<1 << l, 64, 0, st>>>(M, l, yh);
    NF_CHECK();
  }
  k_nf_leaf<<<1 << D, 128, 0, st>>>(M, yh, y);
  NF_CHECK();
  for (size_t i0 = 0; i0 < B.inadm_list.size(); i0 += NF_MAXE) {
    C.count = (int)std::min<size_t>(NF_MAXE, B.inadm_list.size() - i0);
    for (int e = 0; e < C.count; ++e) {
      const int b = B.inadm_list[i0 + e];
      C.t[e] = B.t[b];
      C.s[e] = B.s[b];
      C.off[e] = A->off_N + B.near_off[i0 + e];
    }
    sort_chunk();
    k_nf_near<<<C.count, 128, 0, st>>>(M, g_sorted, x, y);
    NF_CHECK();
  }
#undef NF_CHECK
  return H2_OK;
}
