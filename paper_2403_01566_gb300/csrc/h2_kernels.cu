// Batched FP64 kernels for sm_103a that execute the stage lists built by the
// planner (see h2_ops.h):
//   k_gemm    grouped small GEMM chains with index gathers (out = sum A B [C])
//   k_copy    strided copies / transposes / scalings with zero padding
//   k_qr      Householder QR (the thin QR factorizations of Sections 5.1-5.2)
//   k_qapply  application of the thin Q factor to a small matrix
//   k_svd     one-sided Jacobi SVD (Hestenes) with the truncation rule
//   k_scan    prefix sums of adaptive ranks (panel column offsets)
// One CTA processes one job; FP64 arithmetic throughout.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "h2_ops.h"
#include "h2_kernels.h"

namespace h2 {

__device__ __forceinline__ int dimv(const Dim& d, const int* slot) {
  int v = d.c;
  if (d.s1 >= 0) v += slot[d.s1];
  if (d.s2 >= 0) v += slot[d.s2];
  return v;
}

__device__ __forceinline__ double* ptrv(const Ptr& p, const ExecCtx& x) {
  if (p.arena < 0) return nullptr;
  double* b = x.base[p.arena] + p.off;
  if (p.ds >= 0) b += (int64_t)x.slot[p.ds] * p.dm;
  if (p.ds2 >= 0) b += (int64_t)x.slot[p.ds2] * p.dm2;
  return b;
}

__device__ __forceinline__ void set_err(const ExecCtx& x, int code) {
  if (x.err) atomicCAS(x.err, 0, code);
}

// ------------------------------------------------------------------ GEMM ----
// Output tile up to GT x GT, 256 threads, each thread 4x4 outputs.
constexpr int GT = 64;
constexpr int GK = 32;

__device__ __forceinline__ double ld_op(const double* p, int ld, int t, int i, int j) {
  return t ? p[(int64_t)j * ld + i] : p[(int64_t)i * ld + j];
}

__global__ void __launch_bounds__(256) k_gemm(const ExecCtx* __restrict__ px, const GemmOut* __restrict__ outs,
                                              const GemmTerm* __restrict__ terms) {
  const ExecCtx& x = *px;
  extern __shared__ double sm[];
  double* As = sm;                      // GT x (GK+1)
  double* Bs = As + GT * (GK + 1);      // GK x (GT+1)
  double* Ts = Bs + GK * (GT + 1);      // GT x (GT+1)
  const GemmOut& O = outs[blockIdx.x];
  const int m = dimv(O.m, x.slot);
  const int n = O.clampn ? min(dimv(O.n, x.slot), GT) : dimv(O.n, x.slot);
  if (m <= 0 || n <= 0) return;
  if (m > GT || n > GT) {
    if (threadIdx.x == 0) set_err(x, -9);
    return;
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int ti = O.t0; ti < O.t1; ++ti) {
    const GemmTerm& T = terms[ti];
    double alpha = T.alpha;
    if (T.scale_idx >= 0) alpha *= x.scal[T.scale_idx];
    const double* A = ptrv(T.a, x);
    const double* B = ptrv(T.b, x);
    const double* C = ptrv(T.c, x);
    if (B == nullptr) {  // plain add of op(A) (m x n)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int r = ty + 16 * i, c = tx + 16 * j;
          if (r < m && c < n) acc[i][j] += alpha * ld_op(A, T.lda, T.ta, r, c);
        }
      continue;
    }
    const int k1 = dimv(T.k1, x.slot);
    const int nn = C ? dimv(T.k2, x.slot) : n;  // columns of op(A)op(B)
    if (C && nn > GT) {
      if (threadIdx.x == 0) set_err(x, -9);
      return;
    }
    double tacc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) tacc[i][j] = 0.0;
    for (int kk = 0; kk < k1; kk += GK) {
      const int kc = min(GK, k1 - kk);
      for (int e = threadIdx.x; e < GT * GK; e += 256) {
        int r = e / GK, l = e % GK;
        As[r * (GK + 1) + l] = (r < m && l < kc) ? ld_op(A, T.lda, T.ta, r, kk + l) : 0.0;
      }
      for (int e = threadIdx.x; e < GK * GT; e += 256) {
        int l = e / GT, c = e % GT;
        Bs[l * (GT + 1) + c] = (l < kc && c < nn) ? ld_op(B, T.ldb, T.tb, kk + l, c) : 0.0;
      }
      __syncthreads();
      for (int l = 0; l < kc; ++l) {
        double av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[(ty + 16 * i) * (GK + 1) + l];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[l * (GT + 1) + tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) tacc[i][j] = fma(av[i], bv[j], tacc[i][j]);
      }
      __syncthreads();
    }
    if (C == nullptr) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += alpha * tacc[i][j];
      continue;
    }
    // three-factor term: Ts = op(A)op(B) (m x nn), then acc += alpha * Ts op(C)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) Ts[(ty + 16 * i) * (GT + 1) + tx + 16 * j] = tacc[i][j];
    __syncthreads();
    for (int kk = 0; kk < nn; kk += GK) {
      const int kc = min(GK, nn - kk);
      for (int e = threadIdx.x; e < GK * GT; e += 256) {
        int l = e / GT, c = e % GT;
        Bs[l * (GT + 1) + c] = (l < kc && c < n) ? ld_op(C, T.ldc, T.tc, kk + l, c) : 0.0;
      }
      __syncthreads();
      for (int l = 0; l < kc; ++l) {
        double av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = Ts[(ty + 16 * i) * (GT + 1) + kk + l];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[l * (GT + 1) + tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(alpha * av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  double* out = ptrv(O.o, x);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = ty + 16 * i, c = tx + 16 * j;
      if (r < m && c < n) {
        double* p = out + (int64_t)r * O.ldo + c;
        *p = O.beta ? (*p + acc[i][j]) : acc[i][j];
      }
    }
}

// ------------------------------------------------------------------ copy ----
__global__ void __launch_bounds__(256) k_copy(const ExecCtx* __restrict__ px, const CopyJob* __restrict__ jobs) {
  const ExecCtx& x = *px;
  const CopyJob& J = jobs[blockIdx.x];
  const int rows = dimv(J.rows, x.slot), cols = dimv(J.cols, x.slot);
  const int zr = max(rows, dimv(J.zrows, x.slot)), zc = max(cols, dimv(J.zcols, x.slot));
  const double* S = ptrv(J.src, x);
  double* D = ptrv(J.dst, x);
  double alpha = J.alpha;
  if (J.scale_idx >= 0) alpha *= x.scal[J.scale_idx];
  const int64_t total = (int64_t)zr * zc;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    int i = (int)(e / zc), j = (int)(e % zc);
    double v = 0.0;
    if (S && i < rows && j < cols) v = alpha * (J.trans ? S[(int64_t)j * J.lds + i] : S[(int64_t)i * J.lds + j]);
    D[(int64_t)i * J.ldd + j] = v;
  }
}

// -------------------------------------------------------------------- QR ----
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    s = warp_sum(s);
    if (l == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  return s;
}

__global__ void __launch_bounds__(256) k_qr(const ExecCtx* __restrict__ px, const QrJob* __restrict__ jobs) {
  const ExecCtx& x = *px;
  __shared__ double red[32];
  __shared__ double sh_tau;
  const QrJob& J = jobs[blockIdx.x];
  const int rows = dimv(J.rows, x.slot), cols = dimv(J.cols, x.slot);
  double* a = ptrv(J.a, x);
  double* tau = ptrv(J.tau, x);
  const int lda = J.lda;
  const int q = min(rows, cols);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = 0; j < q; ++j) {
    double* col = a + (int64_t)j * lda;
    double s2 = 0.0;
    for (int i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) s2 += col[i] * col[i];
    s2 = block_sum(s2, red);
    if (threadIdx.x == 0) {
      const double alpha = col[j];
      double t = 0.0;
      if (s2 > 0.0) {
        const double beta = -copysign(sqrt(alpha * alpha + s2), alpha);
        t = (beta - alpha) / beta;
        red[1] = 1.0 / (alpha - beta);
        col[j] = beta;
      } else {
        red[1] = 0.0;
      }
      sh_tau = t;
      if (tau) tau[j] = t;
    }
    __syncthreads();
    const double t = sh_tau, sc = red[1];
    if (t != 0.0)
      for (int i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) col[i] *= sc;
    __syncthreads();
    if (t != 0.0) {
      for (int c = j + 1 + warp; c < cols; c += nw) {
        double* cc = a + (int64_t)c * lda;
        double p = 0.0;
        for (int i = j + 1 + lane; i < rows; i += 32) p += col[i] * cc[i];
        p = warp_sum(p);
        const double w = t * (cc[j] + p);
        if (lane == 0) cc[j] -= w;
        for (int i = j + 1 + lane; i < rows; i += 32) cc[i] -= w * col[i];
      }
    }
    __syncthreads();
  }
  double* r = ptrv(J.r, x);
  if (r) {
    for (int e = threadIdx.x; e < cols * cols; e += blockDim.x) {
      int i = e / cols, c = e % cols;
      r[(int64_t)i * J.ldr + c] = (c >= i && i < q) ? a[(int64_t)c * lda + i] : 0.0;
    }
  }
}

__global__ void __launch_bounds__(256) k_qapply(const ExecCtx* __restrict__ px, const QApplyJob* __restrict__ jobs) {
  const ExecCtx& x = *px;
  const QApplyJob& J = jobs[blockIdx.x];
  const int rows = dimv(J.rows, x.slot), q = dimv(J.q, x.slot), nc = dimv(J.ncols, x.slot);
  const double* a = ptrv(J.a, x);
  const double* tau = ptrv(J.tau, x);
  const double* y = ptrv(J.y, x);
  double* out = ptrv(J.out, x);
  const int ldo = J.ldo;
  for (int64_t e = threadIdx.x; e < (int64_t)rows * nc; e += blockDim.x) {
    int i = (int)(e / nc), c = (int)(e % nc);
    out[(int64_t)i * ldo + c] = (i < q) ? y[(int64_t)i * J.ldy + c] : 0.0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = min(q, rows) - 1; j >= 0; --j) {
    const double t = tau[j];
    if (t != 0.0) {
      const double* v = a + (int64_t)j * J.lda;
      for (int c = warp; c < nc; c += nw) {
        double p = 0.0;
        for (int i = j + 1 + lane; i < rows; i += 32) p += v[i] * out[(int64_t)i * ldo + c];
        p = warp_sum(p);
        const double w = t * (out[(int64_t)j * ldo + c] + p);
        if (lane == 0) out[(int64_t)j * ldo + c] -= w;
        for (int i = j + 1 + lane; i < rows; i += 32) out[(int64_t)i * ldo + c] -= w * v[i];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------- SVD ----
constexpr int SVD_MAXSWEEP = 60;

__global__ void __launch_bounds__(256) k_svd(const ExecCtx* __restrict__ px, const SvdJob* __restrict__ jobs,
                                             int64_t first) {
  const ExecCtx& x = *px;
  extern __shared__ double sm[];
  __shared__ int rotated;
  __shared__ double snorm[SVD_MAXDIM];
  __shared__ int spos[SVD_MAXDIM];
  const SvdJob& J = jobs[blockIdx.x];
  const int rows = dimv(J.rows, x.slot), cols = dimv(J.cols, x.slot);
  int* rank_out = (J.rank_slot >= 0) ? x.slot + J.rank_slot : nullptr;
  if (rows <= 0 || cols <= 0) {
    if (threadIdx.x == 0) {
      if (rank_out) *rank_out = 0;
      if (J.mode == 4) {
        x.nrm[J.norm_idx] = 0.0;
        x.scal[J.norm_idx] = 0.0;
      }
    }
    return;
  }
  if (rows > SVD_MAXDIM || cols > SVD_MAXDIM) {
    if (threadIdx.x == 0) {
      set_err(x, -9);
      if (rank_out) *rank_out = 0;
    }
    return;
  }
  const int ldm = rows + 1;
  double* M = sm;  // column c at M + c*ldm
  const double* S = ptrv(J.src, x);
  for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
    int r = e / cols, c = e % cols;
    M[c * ldm + r] = J.trans ? S[(int64_t)c * J.lds + r] : S[(int64_t)r * J.lds + c];
  }
  __syncthreads();
  // Frobenius norm (invariant under the rotations); columns whose norm falls
  // below 2^-50 ||M||_F are rounding noise: they are not rotated and count as
  // sigma = 0 (otherwise noise re-created by neighbouring rotations keeps the
  // sweeps from converging and yields non-orthogonal vectors).
  __shared__ double s_fro;
  {
    double p = 0.0;
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int r = e / cols, c = e % cols;
      const double v = M[c * ldm + r];
      p = fma(v, v, p);
    }
    p = block_sum(p, snorm);
    if (threadIdx.x == 0) s_fro = p;
    __syncthreads();
  }
  const double tiny2 = s_fro * 7.888609052210118e-31;  // (2^-50)^2 ||M||_F^2
  const int ce = cols + (cols & 1);
  const int npairs = ce / 2;
  int ts = 32;
  while (ts > 1 && ts * npairs > (int)blockDim.x) ts >>= 1;
  const int team = threadIdx.x / ts, tl = threadIdx.x % ts;
  const double tol = 2.5e-15;
  int sweep = 0;
  for (; sweep < SVD_MAXSWEEP; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < ce - 1; ++rnd) {
      int i = -1, j = -1;
      if (team < npairs) {
        if (team == 0) {
          i = rnd;
          j = ce - 1;
        } else {
          i = (rnd + team) % (ce - 1);
          j = (rnd - team + ce - 1) % (ce - 1);
        }
        if (i > j) {
          int t = i;
          i = j;
          j = t;
        }
      }
      const bool valid = team < npairs && j < cols;
      double al = 0.0, be = 0.0, ga = 0.0;
      if (valid) {
        const double* mi = M + i * ldm;
        const double* mj = M + j * ldm;
        for (int r = tl; r < rows; r += ts) {
          const double u = mi[r], v = mj[r];
          al = fma(u, u, al);
          be = fma(v, v, be);
          ga = fma(u, v, ga);
        }
      }
      for (int o = ts >> 1; o > 0; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
      }
      if (valid && ga != 0.0 && al > tiny2 && be > tiny2 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
        const double zeta = (be - al) / (2.0 * ga);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double s = c * t;
        double* mi = M + i * ldm;
        double* mj = M + j * ldm;
        for (int r = tl; r < rows; r += ts) {
          const double u = mi[r], v = mj[r];
          mi[r] = c * u - s * v;
          mj[r] = s * u + c * v;
        }
        if (tl == 0) rotated = 1;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (sweep >= SVD_MAXSWEEP) set_err(x, -5);
    if (x.svd_sweeps) x.svd_sweeps[first + blockIdx.x] = sweep + 1;
  }
  // column norms = singular values
  for (int c = threadIdx.x >> 5; c < cols; c += blockDim.x >> 5) {
    double s = 0.0;
    for (int r = threadIdx.x & 31; r < rows; r += 32) s = fma(M[c * ldm + r], M[c * ldm + r], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) snorm[c] = (s > tiny2) ? sqrt(s) : 0.0;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    const double v = snorm[c];
    int p = 0;
    for (int l = 0; l < cols; ++l) {
      const double w = snorm[l];
      p += (w > v) || (w == v && l < c);
    }
    spos[c] = p;
  }
  __syncthreads();
  double* sig = ptrv(J.sig, x);
  if (sig)
    for (int c = threadIdx.x; c < cols; c += blockDim.x) sig[spos[c]] = snorm[c];
  double* U = ptrv(J.u, x);
  if (U) {
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      int r = e / cols, c = e % cols;
      const double s = snorm[c];
      U[(int64_t)r * J.ldu + spos[c]] = s > 0.0 ? M[c * ldm + r] / s : 0.0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0;
    for (int c = 0; c < cols; ++c) s0 = fmax(s0, snorm[c]);
    const double tol = J.tol_idx >= 0 ? J.tol * x.scal[J.tol_idx] : J.tol;
    int k = 0;
    if (J.mode == 1) {
      for (int c = 0; c < cols; ++c) k += snorm[c] > tol;
    } else if (J.mode == 2) {
      if (s0 > 0.0)
        for (int c = 0; c < cols; ++c) k += snorm[c] > tol * s0;
    } else if (J.mode == 4) {
      x.nrm[J.norm_idx] = s0;
      x.scal[J.norm_idx] = s0 > 0.0 ? 1.0 / s0 : 0.0;
    }
    if (J.mode == 1 || J.mode == 2) {
      if (k > J.cap) {
        set_err(x, -7);
        k = J.cap;
      }
      if (rank_out) *rank_out = k;
    }
  }
}

// ------------------------------------------------------------------ scan ----
__global__ void k_scan(const ExecCtx* __restrict__ px, const ScanJob* __restrict__ jobs, int count) {
  const ExecCtx& x = *px;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  const ScanJob& J = jobs[j];
  int s = 0;
  for (int i = 0; i < J.count; ++i) {
    x.slot[J.out + i] = s;
    s += x.slot[x.idx[J.idx_off + i]];
  }
  x.slot[J.out + J.count] = s;
}

// Copies the adaptive ranks and the error flag of a product into the
// product's own integer array (last kernel of a product's stage list).
__global__ void k_finalize(const ExecCtx* __restrict__ px) {
  const ExecCtx& x = *px;
  if (x.out_int == nullptr) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < x.nrank; i += gridDim.x * blockDim.x)
    x.out_int[i] = x.slot[x.rank_src[i]];
  if (blockIdx.x == 0 && threadIdx.x == 0) x.out_int[x.nrank] = *x.err;
}

// ------------------------------------------------------------- launchers ----
size_t gemm_smem_bytes() { return sizeof(double) * (GT * (GK + 1) + GK * (GT + 1) + GT * (GT + 1)); }
size_t svd_smem_bytes(int rows, int cols) { return sizeof(double) * (size_t)(rows + 1) * cols; }

static bool g_attr_done = false;

cudaError_t kernels_init() {
  if (g_attr_done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem_bytes());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_svd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)svd_smem_bytes(SVD_MAXDIM, SVD_MAXDIM));
  if (e != cudaSuccess) return e;
  g_attr_done = true;
  return cudaSuccess;
}

void launch_finalize(const ExecCtx* x, int nrank, cudaStream_t s) {
  k_finalize<<<(nrank + 255) / 256 + 1, 256, 0, s>>>(x);
}

void launch_stage(const Stage& st, const ExecCtx* x, const DeviceJobs& j, size_t svd_smem, cudaStream_t s) {
  if (st.count <= 0) return;
  switch (st.kind) {
    case ST_GEMM:
      k_gemm<<<st.count, 256, gemm_smem_bytes(), s>>>(x, j.gemm_out + st.first, j.gemm_term);
      break;
    case ST_COPY:
      k_copy<<<st.count, 256, 0, s>>>(x, j.copy + st.first);
      break;
    case ST_QR:
      k_qr<<<st.count, 256, 0, s>>>(x, j.qr + st.first);
      break;
    case ST_QAPPLY:
      k_qapply<<<st.count, 256, 0, s>>>(x, j.qapply + st.first);
      break;
    case ST_SVD:
      k_svd<<<st.count, 256, svd_smem, s>>>(x, j.svd + st.first, st.first);
      break;
    case ST_SCAN:
      k_scan<<<(st.count + 127) / 128, 128, 0, s>>>(x, j.scan + st.first, st.count);
      break;
  }
}

}  // namespace h2
