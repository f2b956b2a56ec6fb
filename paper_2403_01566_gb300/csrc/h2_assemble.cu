// Device assembly of a Chebyshev H^2-matrix (the numeric part of h2_build).
//
// A Nystroem matrix g(x_i, x_j) with tensor Chebyshev interpolation on the
// cluster boxes (Section 2, eq. (3)):
//   V_t(i, nu)   = ell_{t,nu}(x_i)                 leaf bases
//   E_t'(nu',nu) = ell_{t,nu}(xi_{t',nu'})          transfer matrices, t = parent of t'
//   S_b(nu, mu)  = g(xi_{t,nu}, xi_{s,mu})          couplings of admissible leaves b = (t, s)
//   N_b(i, j)    = g(x_i, x_j)  (prescribed value on i = j)   inadmissible leaves
// with ell the tensor Lagrange polynomials of the first-kind Chebyshev points
// xi of each box.  The host builds the trees, the block tree and the
// Chebyshev points (shared with the host assembly); these kernels evaluate the
// entries straight into the matrix's device arena.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/h2.h"
#include "h2_assemble.h"
#include "h2_build.h"
#include "h2_internal.h"

namespace h2 {
namespace {

constexpr int ASM_MAXM = 8;  // interpolation order limit of h2_build

struct AsmGeom {
  const double* pts;    // points in cluster order (n x dim)
  const double* nodes;  // Chebyshev points (ncl x dim x m)
  const int* off;       // cluster offsets
  const int* size;      // cluster sizes
  int dim, m, k;
};

__device__ double kernel_eval(int kind, double scale, double width, const double* x, const double* y, int dim) {
  double r2 = 0.0;
  for (int a = 0; a < dim; ++a) {
    const double d = x[a] - y[a];
    r2 += d * d;
  }
  switch (kind) {
    case 0: return -scale * 0.5 * log(r2);
    case 1: return scale / sqrt(r2);
    case 2: return scale * exp(-r2 / width);
    default: return scale * exp(-sqrt(r2) / width);
  }
}

// one-dimensional Lagrange polynomial j of the m points x at p
__device__ double lagrange1(const double* x, int m, int j, double p) {
  double v = 1.0;
  for (int i = 0; i < m; ++i)
    if (i != j) v *= (p - x[i]) / (x[j] - x[i]);
  return v;
}

// V: one CTA per leaf, one thread per point, k values per point
__global__ void k_asm_leaf(AsmGeom G, int first_leaf, double* V) {
  const int c = first_leaf + blockIdx.x;
  const int off = G.off[c], sz = G.size[c];
  for (int i = threadIdx.x; i < sz; i += blockDim.x) {
    const double* p = G.pts + (int64_t)(off + i) * G.dim;
    double l1[3][ASM_MAXM];
    for (int a = 0; a < G.dim; ++a) {
      const double* x = G.nodes + ((int64_t)c * G.dim + a) * G.m;
      for (int j = 0; j < G.m; ++j) l1[a][j] = lagrange1(x, G.m, j, p[a]);
    }
    double* out = V + (int64_t)(off + i) * G.k;
    for (int nu = 0; nu < G.k; ++nu) {
      int r = nu;
      double v = 1.0;
      for (int a = 0; a < G.dim; ++a) {
        v *= l1[a][r % G.m];
        r /= G.m;
      }
      out[nu] = v;
    }
  }
}

// E: one CTA per cluster c >= 1, one thread per entry (nu', nu)
__global__ void k_asm_transfer(AsmGeom G, double* E) {
  const int c = 1 + blockIdx.x;
  const int par = (c - 1) / 2;
  for (int e = threadIdx.x; e < G.k * G.k; e += blockDim.x) {
    const int nu2 = e / G.k, nu = e % G.k;
    int r2 = nu2, r = nu;
    double v = 1.0;
    for (int a = 0; a < G.dim; ++a) {
      const double p = G.nodes[((int64_t)c * G.dim + a) * G.m + r2 % G.m];
      v *= lagrange1(G.nodes + ((int64_t)par * G.dim + a) * G.m, G.m, r % G.m, p);
      r2 /= G.m;
      r /= G.m;
    }
    E[((int64_t)c * G.k + nu2) * G.k + nu] = v;
  }
}

// S: one CTA per admissible leaf, one thread per entry (nu, mu)
__global__ void k_asm_coupling(AsmGeom G, const int* __restrict__ ts, int kind, double scale, double width,
                               double* S) {
  const int t = ts[2 * blockIdx.x], s = ts[2 * blockIdx.x + 1];
  double* out = S + (int64_t)blockIdx.x * G.k * G.k;
  for (int e = threadIdx.x; e < G.k * G.k; e += blockDim.x) {
    const int nu = e / G.k, mu = e % G.k;
    double p[3], q[3];
    int r = nu, u = mu;
    for (int a = 0; a < G.dim; ++a) {
      p[a] = G.nodes[((int64_t)t * G.dim + a) * G.m + r % G.m];
      q[a] = G.nodes[((int64_t)s * G.dim + a) * G.m + u % G.m];
      r /= G.m;
      u /= G.m;
    }
    out[e] = kernel_eval(kind, scale, width, p, q, G.dim);
  }
}

// N: one CTA per inadmissible leaf, one thread per entry (i, j)
__global__ void k_asm_near(AsmGeom G, const int* __restrict__ ts, const int64_t* __restrict__ noff, int kind,
                           double scale, double diag, double width, double* N) {
  const int t = ts[2 * blockIdx.x], s = ts[2 * blockIdx.x + 1];
  const int ot = G.off[t], st = G.size[t], os = G.off[s], ss = G.size[s];
  double* out = N + noff[blockIdx.x];
  for (int e = threadIdx.x; e < st * ss; e += blockDim.x) {
    const int i = e / ss, j = e % ss;
    out[e] = (ot + i == os + j) ? diag
                                : kernel_eval(kind, scale, width, G.pts + (int64_t)(ot + i) * G.dim,
                                              G.pts + (int64_t)(os + j) * G.dim, G.dim);
  }
}

}  // namespace

int assemble_device(const double* points, const Tree& T, const BlockTree& B, int order, int kind,
                    const double* kparam, double* d_V, double* d_E, double* d_S, double* d_N, cudaStream_t st,
                    std::string& err) {
  int k = 1;
  for (int a = 0; a < T.dim; ++a) k *= order;
  if (order > ASM_MAXM || T.dim > 3) {
    err = "assembly: order or dimension out of range";
    return H2_EINVAL;
  }
  // host side: points in cluster order, Chebyshev points, cluster and block lists
  const int dim = T.dim;
  std::vector<double> pts((size_t)T.n * dim);
  for (int64_t r = 0; r < T.n; ++r)
    for (int a = 0; a < dim; ++a) pts[(size_t)r * dim + a] = points[(size_t)T.perm[r] * dim + a];
  const std::vector<double> nodes = chebyshev_nodes(T, order);
  std::vector<int> adm(2 * B.adm_list.size()), inadm(2 * B.inadm_list.size());
  for (size_t a = 0; a < B.adm_list.size(); ++a) {
    adm[2 * a] = B.t[B.adm_list[a]];
    adm[2 * a + 1] = B.s[B.adm_list[a]];
  }
  for (size_t a = 0; a < B.inadm_list.size(); ++a) {
    inadm[2 * a] = B.t[B.inadm_list[a]];
    inadm[2 * a + 1] = B.s[B.inadm_list[a]];
  }
  // one staging buffer for all inputs of the kernels
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t o_pts = 0, o_nodes = o_pts + al(pts.size() * 8), o_off = o_nodes + al(nodes.size() * 8),
               o_size = o_off + al(T.off.size() * 4), o_adm = o_size + al(T.size.size() * 4),
               o_inadm = o_adm + al(adm.size() * 4 + 8), o_noff = o_inadm + al(inadm.size() * 4 + 8),
               total = o_noff + al(B.near_off.size() * 8 + 8);
  std::vector<char> blob(total);
  auto put = [&](size_t o, const void* p, size_t n) {
    if (n) std::memcpy(blob.data() + o, p, n);
  };
  put(o_pts, pts.data(), pts.size() * 8);
  put(o_nodes, nodes.data(), nodes.size() * 8);
  put(o_off, T.off.data(), T.off.size() * 4);
  put(o_size, T.size.data(), T.size.size() * 4);
  put(o_adm, adm.data(), adm.size() * 4);
  put(o_inadm, inadm.data(), inadm.size() * 4);
  put(o_noff, B.near_off.data(), B.near_off.size() * 8);
  char* d = nullptr;
  if (cudaMalloc(&d, total) != cudaSuccess) {
    cudaGetLastError();
    err = "assembly: staging allocation";
    return H2_ENOMEM;
  }
  cudaMemcpyAsync(d, blob.data(), total, cudaMemcpyHostToDevice, st);
  AsmGeom G{reinterpret_cast<const double*>(d + o_pts), reinterpret_cast<const double*>(d + o_nodes),
            reinterpret_cast<const int*>(d + o_off), reinterpret_cast<const int*>(d + o_size), dim, order, k};
  const int nleaf = T.count(T.depth);
  if (nleaf > 0) k_asm_leaf<<<nleaf, 128, 0, st>>>(G, Tree::first(T.depth), d_V);
  if (T.ncl > 1) k_asm_transfer<<<T.ncl - 1, 256, 0, st>>>(G, d_E);
  if (!B.adm_list.empty())
    k_asm_coupling<<<(unsigned)B.adm_list.size(), 256, 0, st>>>(G, reinterpret_cast<const int*>(d + o_adm), kind,
                                                                  kparam[0], kparam[2], d_S);
  if (!B.inadm_list.empty())
    k_asm_near<<<(unsigned)B.inadm_list.size(), 256, 0, st>>>(
        G, reinterpret_cast<const int*>(d + o_inadm), reinterpret_cast<const int64_t*>(d + o_noff), kind, kparam[0],
        kparam[1], kparam[2], d_N);
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaStreamSynchronize(st);  // the staging buffer is freed below
  cudaFree(d);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    err = std::string("assembly kernels: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2);
    return H2_ECUDA;
  }
  return H2_OK;
}

}  // namespace h2
