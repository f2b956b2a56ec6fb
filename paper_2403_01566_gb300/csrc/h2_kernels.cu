// Batched FP64 kernels for sm_103a that execute the stage lists built by the
// planner (see h2_ops.h):
//   k_gemm    grouped small GEMM chains with index gathers (out = sum A B [C]),
//             in FP64, FP32 or compensated FP32 (the precision forms)
//   k_gemm_tc the same chains on the tensor cores (mma.sync BF16, FP32
//             accumulation) with 8-bit operand slices: about FP64 accuracy
//             with 7 slices, 40 bits with 5
//   k_copy    strided copies / transposes / scalings with zero padding
//   k_qr      Householder QR (the thin QR factorizations of Sections 5.1-5.2),
//             column-pivoted where an SVD follows, optionally stopped at a
//             noise floor
//   k_qapply  application of the thin Q factor to a small matrix
//   k_svd     one-sided Jacobi SVD (Hestenes) with the truncation rule
//   k_norm    spectral norms (Section 5.3)
//   k_scan    prefix sums of adaptive ranks (panel column offsets)
// One CTA processes one job; everything but the contractions of the FP32 and
// compensated forms is FP64 arithmetic.
#include <cuda_runtime.h>
#include <climits>
#include <cstdint>
#include <math.h>
#include <stdint.h>

#include "h2_ops.h"
#include "h2_kernels.h"

namespace h2 {

__device__ __forceinline__ int dimv(const Dim& d, const int* slot) {
  int v = d.c;
  if (d.s1 >= 0) v += slot[d.s1];
  if (d.s2 >= 0) v += slot[d.s2];
  if (d.mc >= 0) v = min(v, d.mc + (d.ms >= 0 ? slot[d.ms] : 0));
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
// Output tile up to GT x GT; the 256 threads are mapped onto the actual output
// elements (see out_map), so small outputs (16 x 16 coupling and transfer
// products) waste no FP64 FMA.  Operand chunks of GK columns are staged in
// shared memory; each output is a dot product over the chunk.
constexpr int GT = 64;
constexpr int GK = 32;
constexpr int GQ = (GT * GT) / 256;  // outputs per thread at most

__device__ __forceinline__ double ld_op(const double* p, int ld, int t, int i, int j) {
  return t ? p[(int64_t)j * ld + i] : p[(int64_t)i * ld + j];
}

// Compute modes of the grouped GEMM.  Operands are FP64 arrays; each inner
// product over k runs in the mode's arithmetic, its result is combined in
// FP64 (alpha, further terms, beta).
//   GM_F64  FP64 products and sums
//   GM_F32  operands rounded to FP32, FP32 products and sums (~1e-7)
//   GM_DF   compensated: operands split into FP32 hi + lo parts (a = hi + lo
//           to ~2^-48), the hi*hi product error-free via FMA, sums by TwoSum
//           (Knuth), the hi*lo and lo*hi cross terms and all error terms in a
//           second FP32 word (Ogita, Rump and Oishi, "Accurate sum and dot
//           product", SIAM J. Sci. Comput. 26, 2005); ~1e-13 relative at FP32
//           issue rates.  The error-free steps use the non-contracting
//           __fmul_rn / __fadd_rn / __fsub_rn intrinsics.
enum GemmMode : int { GM_F64 = 0, GM_F32 = 1, GM_DF = 2 };

struct DF {
  float s, c;
};

template <int MODE>
struct GemmPol;

// Policy members: S staged operand, A inner (k-loop) accumulator, O outer
// accumulator over the terms of an output; stage() converts a loaded
// operand, restage() an inner result that becomes an operand again (the
// middle product of a three-factor term), oadd(o, alpha, a) does
// o += alpha * a, oadd_plain(o, alpha, v) does o += alpha * v, result()
// returns the output value.
template <>
struct GemmPol<GM_F64> {
  using S = double;
  using A = double;
  using O = double;
  __device__ static S stage(double v) { return v; }
  __device__ static S restage(const A& a) { return a; }
  __device__ static A zero() { return 0.0; }
  __device__ static O ozero() { return 0.0; }
  __device__ static void fma_acc(A& a, S x, S y) { a = fma(x, y, a); }
  using Alpha = double;
  __device__ static Alpha alpha_of(double alpha) { return alpha; }
  __device__ static void oadd(O& o, Alpha alpha, const A& a) { o = fma(alpha, a, o); }
  __device__ static void oadd_plain(O& o, double alpha, double v) { o = fma(alpha, v, o); }
  __device__ static double result(const O& o) { return o; }
};

template <>
struct GemmPol<GM_F32> {
  using S = float;
  using A = float;
  using O = double;
  __device__ static S stage(double v) { return (float)v; }
  __device__ static S restage(const A& a) { return a; }
  __device__ static A zero() { return 0.0f; }
  __device__ static O ozero() { return 0.0; }
  __device__ static void fma_acc(A& a, S x, S y) { a = fmaf(x, y, a); }
  using Alpha = double;
  __device__ static Alpha alpha_of(double alpha) { return alpha; }
  __device__ static void oadd(O& o, Alpha alpha, const A& a) { o = fma(alpha, (double)a, o); }
  __device__ static void oadd_plain(O& o, double alpha, double v) { o = fma(alpha, v, o); }
  __device__ static double result(const O& o) { return o; }
};

// FP32 value of an integer 0 <= m < 2^29 rounded to nearest even, by integer
// operations only (on this GPU int-to-float conversions issue on the FP64
// pipe, 16 cycles a warp instruction; the same bits as __uint2float_rn).
__device__ __forceinline__ float f32_of_u29_rn(uint32_t m) {
  if (m == 0u) return 0.0f;
  const int p = 31 - __clz(m);  // leading bit
  uint32_t mant;
  int e = p;
  if (p <= 23) {
    mant = m << (23 - p);
  } else {
    const int sh = p - 23;  // 1..5
    mant = m >> sh;
    const uint32_t rem = m & ((1u << sh) - 1u), half = 1u << (sh - 1);
    if (rem > half || (rem == half && (mant & 1u))) ++mant;
    if (mant == (1u << 24)) {
      mant >>= 1;
      ++e;
    }
  }
  return __uint_as_float(((uint32_t)(e + 127) << 23) | (mant & 0x7fffffu));
}

// Split of an FP64 value into FP32 hi + lo without FP64-pipe instructions
// (on this GPU every FP64 instruction, conversions included, issues at 1/64
// of the FP32 rate).  hi = the value truncated to 24 significant bits (bit
// copy of sign, re-biased exponent and the top 23 fraction bits); lo = the
// remaining 29 fraction bits rounded to FP32 and scaled: |v - hi - lo| <=
// 2^-47 |v|.  Zero and values below FP32's normal range (|v| < 2^-126) give
// (0, 0); |v| >= 2^128, inf and NaN take the plain conversion.
__device__ __forceinline__ float2 split_df(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
  const int e = (int)((hw >> 20) & 0x7ffu) - 1023;
  if (e < -126) return make_float2(0.0f, 0.0f);
  if (e > 127) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  }
  const unsigned sign = hw & 0x80000000u;
  const unsigned ebits = (unsigned)(e + 127) << 23;
  const float hi = __uint_as_float(sign | ebits | ((hw & 0xfffffu) << 3) | (lw >> 29));
  const float rem = __fmul_rn(f32_of_u29_rn(lw & 0x1fffffffu), 0x1p-52f);  // < 2^-23
  const float lo = __fmul_rn(rem, __uint_as_float(ebits));                  // rem * 2^e
  return make_float2(hi, __uint_as_float(__float_as_uint(lo) | sign));
}

// Exact FP64 value of an FP32 value, by bit operations for normal values and
// zero (float-to-double conversions also issue on the FP64 pipe).
__device__ __forceinline__ double f64_of_f32(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t ef = (b >> 23) & 0xffu;
  if (ef == 0u && (b & 0x7fffffu) != 0u) return (double)f;  // subnormal
  if (ef == 0xffu) return (double)f;                        // inf, NaN
  const uint32_t hw = (b & 0x80000000u) | (ef ? ((ef - 127u + 1023u) << 20) : 0u) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hw, (int)((b & 0x7u) << 29));
}

template <>
struct GemmPol<GM_DF> {
  using S = float2;  // (hi, lo)
  using A = DF;
  using O = DF;
  __device__ static S stage(double v) { return split_df(v); }
  // (s, c) renormalised by Fast2Sum (|c| <= |s| for these accumulators)
  __device__ static S restage(const A& a) {
    const float h = __fadd_rn(a.s, a.c);
    return make_float2(h, __fsub_rn(a.c, __fsub_rn(h, a.s)));
  }
  __device__ static A zero() { return DF{0.0f, 0.0f}; }
  __device__ static O ozero() { return DF{0.0f, 0.0f}; }
  // o += (ph + pl) with ph = alpha_hi * a.s exact through an FMA: TwoSum on
  // the leading parts, every error term into o.c (alpha split once per term)
  using Alpha = float2;
  __device__ static Alpha alpha_of(double alpha) { return split_df(alpha); }
  __device__ static void oadd(O& o, Alpha al, const A& a) {
    const float ph = __fmul_rn(al.x, a.s);
    float pl = fmaf(al.x, a.s, -ph);
    pl = fmaf(al.x, a.c, pl);
    pl = fmaf(al.y, a.s, pl);
    add2(o, ph, pl);
  }
  __device__ static void oadd_plain(O& o, double alpha, double v) {
    const float2 p = split_df(alpha * v);
    add2(o, p.x, p.y);
  }
  __device__ static void add2(O& o, float h, float l) {
    const float t = __fadd_rn(o.s, h);
    const float z = __fsub_rn(t, o.s);
    const float err = __fadd_rn(__fsub_rn(o.s, __fsub_rn(t, z)), __fsub_rn(h, z));
    o.s = t;
    o.c = __fadd_rn(__fadd_rn(o.c, err), l);
  }
  __device__ static double result(const O& o) { return f64_of_f32(o.s) + f64_of_f32(o.c); }
  // The error terms of one step are summed first, so that each of a.s and
  // a.c carries a single dependent add from one k step to the next.
  __device__ static void fma_acc(A& a, S x, S y) {
    const float p = __fmul_rn(x.x, y.x);
    const float e = fmaf(x.x, y.x, -p);  // x.hi * y.hi = p + e exactly
    const float t = __fadd_rn(a.s, p);   // TwoSum(a.s, p) = t + err exactly
    const float z = __fsub_rn(t, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, z)), __fsub_rn(p, z));
    a.s = t;
    float u = fmaf(x.x, y.y, e);
    u = fmaf(x.y, y.x, u);
    a.c = __fadd_rn(a.c, __fadd_rn(u, err));
  }
};

// Outputs of this thread in an m x n tile: column c, rows r0 + q * rstep for
// q < nv, where rstep = 256 / n rows are covered per step (threads beyond
// rstep * n idle).  Every output of a thread shares its column, so one staged
// B value serves all of its accumulators, and the Q accumulation chains are
// independent (they interleave in the inner loop).  Requires
// ceil(m / rstep) <= Q.
struct OutMap {
  int r0, c, rstep, nv;
};
__device__ __forceinline__ OutMap out_map(int m, int n) {
  OutMap o;
  o.rstep = 256 / n;
  o.c = threadIdx.x % n;
  o.r0 = threadIdx.x / n;
  o.nv = (o.r0 < o.rstep && o.r0 < m) ? (m - o.r0 + o.rstep - 1) / o.rstep : 0;
  return o;
}

// acc[q] += sum_l a[q * astep + l] b[l * ldb] (l < kc) for q < nv, one
// output at a time (interleaving 2, 4 or 8 outputs measured slower in every
// mode).
template <int Q, int MODE>
__device__ __forceinline__ void mac_rows(typename GemmPol<MODE>::A (&acc)[Q], int nv,
                                         const typename GemmPol<MODE>::S* a, int astep,
                                         const typename GemmPol<MODE>::S* b, int ldb, int kc) {
  using P = GemmPol<MODE>;
#pragma unroll
  for (int q = 0; q < Q; ++q)
    if (q < nv) {
      typename P::A t = acc[q];
      for (int l = 0; l < kc; ++l) P::fma_acc(t, a[q * astep + l], b[l * ldb]);
      acc[q] = t;
    }
}

// dst[i * ldd + j] = stage(op(src)(i0 + i, j0 + j)) for i < R, j < Cc, with
// op(src)(i, j) = src[j * ld + i] if t else src[i * ld + j].  All threads
// share the R x Cc elements; consecutive threads take consecutive source
// addresses in both orientations.
template <int MODE>
__device__ __forceinline__ void stage_tile(typename GemmPol<MODE>::S* dst, int ldd, const double* src, int ld,
                                           int t, int R, int Cc, int i0, int j0) {
  using P = GemmPol<MODE>;
  if (!t) {
    for (int e = threadIdx.x; e < R * Cc; e += blockDim.x) {
      const int i = e / Cc, j = e % Cc;
      dst[i * ldd + j] = P::stage(src[(int64_t)(i0 + i) * ld + j0 + j]);
    }
  } else {
    for (int e = threadIdx.x; e < R * Cc; e += blockDim.x) {
      const int j = e / R, i = e % R;
      dst[i * ldd + j] = P::stage(src[(int64_t)(j0 + j) * ld + i0 + i]);
    }
  }
}

// acc[q] += op(A)(m x k) op(B)(k x n) for the outputs of this thread
template <int Q, int MODE>
__device__ __forceinline__ void gemm_accumulate(typename GemmPol<MODE>::A (&acc)[Q], const OutMap& om, int m, int n,
                                                int k, const double* A, int lda, int ta, const double* B, int ldb,
                                                int tb, typename GemmPol<MODE>::S* As, typename GemmPol<MODE>::S* Bs,
                                                int ldbs) {
  using P = GemmPol<MODE>;
  using S = typename P::S;
  const S* ar = As + om.r0 * (GK + 1);
  const int astep = om.rstep * (GK + 1);
  for (int kk = 0; kk < k; kk += GK) {
    const int kc = min(GK, k - kk);
    stage_tile<MODE>(As, GK + 1, A, lda, ta, m, kc, 0, kk);
    stage_tile<MODE>(Bs, ldbs, B, ldb, tb, kc, n, kk, 0);
    __syncthreads();
    mac_rows<Q, MODE>(acc, om.nv, ar, astep, Bs + om.c, ldbs, kc);
    __syncthreads();
  }
}

// Shared memory of a stage whose outputs are at most mmax rows and whose
// right factors (and inner widths of three-factor terms) at most nb columns:
// As mmax x (GK+1), Bs GK x (nb+1), Ts mmax x (nb+1) staged operands (8 bytes
// each in the FP64 and compensated modes, 4 in the FP32 mode).  Stages of
// small static shapes thus keep many CTAs resident per SM.
__host__ __device__ constexpr int gemm_smem_doubles(int mmax, int nb) {
  return mmax * (GK + 1) + (GK + mmax) * (nb + 1);
}

// Q = outputs per thread (ceil(m / (256 / n)) <= Q, see out_map): small
// stages take a small Q, so fewer registers and more resident CTAs per SM.
// MODE = compute mode (above).
template <int Q, int MODE>
__device__ __forceinline__ void gemm_job(const ExecCtx& x, const GemmOut& O, const GemmTerm* __restrict__ terms,
                                         int mmax, int nb) {
  using P = GemmPol<MODE>;
  using S = typename P::S;
  extern __shared__ double sm_raw[];
  S* sm = reinterpret_cast<S*>(sm_raw);
  const int ldbs = nb + 1;
  S* As = sm;                      // mmax x (GK+1)
  S* Bs = As + mmax * (GK + 1);    // GK x (nb+1)
  S* Ts = Bs + GK * ldbs;          // mmax x (nb+1)
  const int m = dimv(O.m, x.slot);
  const int n = O.clampn ? min(dimv(O.n, x.slot), GT) : dimv(O.n, x.slot);
  if (m <= 0 || n <= 0) return;
  auto fits = [&](int cols) { return (m + 256 / cols - 1) / (256 / cols) <= Q; };
  if (m > mmax || n > nb || !fits(n)) {
    if (threadIdx.x == 0) set_err(x, -9);
    return;
  }
  const OutMap om = out_map(m, n);
  typename P::O acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) acc[q] = P::ozero();

  for (int ti = O.t0; ti < O.t1; ++ti) {
    const GemmTerm& Tm = terms[ti];
    double alpha = Tm.alpha;
    if (Tm.scale_idx >= 0) alpha *= x.scal[Tm.scale_idx];
    const double* A = ptrv(Tm.a, x);
    const double* B = ptrv(Tm.b, x);
    const double* C = ptrv(Tm.c, x);
    if (B == nullptr) {  // plain add of op(A) (m x n)
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (q < om.nv) P::oadd_plain(acc[q], alpha, ld_op(A, Tm.lda, Tm.ta, om.r0 + q * om.rstep, om.c));
      continue;
    }
    const int k1 = dimv(Tm.k1, x.slot);
    typename P::A tacc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) tacc[q] = P::zero();
    if (C == nullptr) {
      gemm_accumulate<Q, MODE>(tacc, om, m, n, k1, A, Tm.lda, Tm.ta, B, Tm.ldb, Tm.tb, As, Bs, ldbs);
      const typename P::Alpha al = P::alpha_of(alpha);
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (q < om.nv) P::oadd(acc[q], al, tacc[q]);
      continue;
    }
    // three-factor term: Ts = op(A)op(B) (m x nn), then acc += alpha * Ts op(C)
    const int nn = dimv(Tm.k2, x.slot);
    if (nn <= 0) continue;
    if (nn > nb || !fits(nn)) {
      if (threadIdx.x == 0) set_err(x, -9);
      return;
    }
    const OutMap om2 = out_map(m, nn);
    gemm_accumulate<Q, MODE>(tacc, om2, m, nn, k1, A, Tm.lda, Tm.ta, B, Tm.ldb, Tm.tb, As, Bs, ldbs);
#pragma unroll
    for (int q = 0; q < Q; ++q)
      if (q < om2.nv) Ts[(om2.r0 + q * om2.rstep) * ldbs + om2.c] = P::restage(tacc[q]);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) tacc[q] = P::zero();
    // Ts (m x nn) times op(C) (nn x n); Ts plays the role of A (already in smem)
    const S* tr = Ts + om.r0 * ldbs;
    const int tstep = om.rstep * ldbs;
    for (int kk = 0; kk < nn; kk += GK) {
      const int kc = min(GK, nn - kk);
      stage_tile<MODE>(Bs, ldbs, C, Tm.ldc, Tm.tc, kc, n, kk, 0);
      __syncthreads();
      mac_rows<Q, MODE>(tacc, om.nv, tr + kk, tstep, Bs + om.c, ldbs, kc);
      __syncthreads();
    }
    const typename P::Alpha al = P::alpha_of(alpha);
#pragma unroll
    for (int q = 0; q < Q; ++q)
      if (q < om.nv) P::oadd(acc[q], al, tacc[q]);
  }
  double* out = ptrv(O.o, x);
#pragma unroll
  for (int q = 0; q < Q; ++q)
    if (q < om.nv) {
      double* p = out + (int64_t)(om.r0 + q * om.rstep) * O.ldo + om.c;
      const double v = P::result(acc[q]);
      *p = O.beta ? (*p + v) : v;
    }
}

// Index of the segment holding block / queue index b (segments sorted by start).
__device__ __forceinline__ int seg_find(const BatchSeg* __restrict__ segs, int nseg, int b) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].start <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One CTA per output tile of a stage (segs == nullptr: the jobs of one
// product; else the segments of a batched launch).
template <int Q, int MODE>
__global__ void __launch_bounds__(256, Q == 1 ? 5 : Q == 4 ? 4 : 2)
    k_gemm(const ExecCtx* __restrict__ px, const GemmOut* __restrict__ outs, const GemmTerm* __restrict__ terms,
           int mmax, int nb, const BatchSeg* __restrict__ segs, int nseg) {
  int b = blockIdx.x;
  if (segs) {
    const BatchSeg& sg = segs[seg_find(segs, nseg, b)];
    px = sg.ctx;
    outs = static_cast<const GemmOut*>(sg.jobs);
    terms = sg.terms;
    b -= sg.start;
  }
  gemm_job<Q, MODE>(*px, outs[b], terms, mmax, nb);
}

// Bounded wait of a chained job for its product's previous stage: about a
// second (2^20 polls, 1 us apart), after which the caller records H2_ETIMEOUT.
constexpr int CHAIN_WAIT_POLLS = 1 << 20;
__device__ __forceinline__ bool chain_wait(const int* p, int target) {
  for (int i = 0; i < CHAIN_WAIT_POLLS; ++i) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    if (v >= target) return true;
    __nanosleep(1000);
  }
  return false;
}

// Persistent launch over a chain of GEMM stages of many products: CTAs take
// jobs from a device work queue (ctr[0]) in stage order; a job waits for its
// product's previous stage (BatchSeg::wait_idx) and counts itself done.  The
// grid never exceeds the CTAs resident at once, so every awaited job is held
// by a running CTA.  A wait that gives up sets H2_ETIMEOUT (-4) on the
// product and the job is skipped; the chain still completes.
template <class JOB>
__device__ __forceinline__ void chain_loop(const BatchSeg* __restrict__ segs, int nseg, int total, int* ctr, JOB job) {
  __shared__ int s_job, s_ok;
  for (;;) {
    if (threadIdx.x == 0) s_job = atomicAdd(&ctr[0], 1);
    __syncthreads();
    const int j = s_job;
    if (j >= total) break;
    const BatchSeg& sg = segs[seg_find(segs, nseg, j)];
    if (threadIdx.x == 0) {
      int ok = 1;
      if (sg.wait_idx >= 0) ok = chain_wait(&ctr[sg.wait_idx], sg.wait_target) ? 1 : 0;
      if (!ok) set_err(*sg.ctx, -4);
      __threadfence();
      s_ok = ok;
    }
    __syncthreads();
    if (s_ok) job(sg, j - sg.start);
    __syncthreads();
    if (threadIdx.x == 0 && sg.done_idx >= 0) {
      __threadfence();
      atomicAdd(&ctr[sg.done_idx], 1);
    }
  }
}

template <int Q, int MODE>
__global__ void __launch_bounds__(256, Q == 1 ? 5 : Q == 4 ? 4 : 2)
    k_gemm_chain(const BatchSeg* __restrict__ segs, int nseg, int total, int* ctr, int mmax, int nb) {
  chain_loop(segs, nseg, total, ctr, [&](const BatchSeg& sg, int i) {
    gemm_job<Q, MODE>(*sg.ctx, static_cast<const GemmOut*>(sg.jobs)[i], sg.terms, mmax, nb);
  });
}

// ------------------------------------------------- tensor-core GEMM (BF16) ----
// Contractions on the tensor cores (mma.sync m16n8k16: BF16 operands, FP32
// accumulation) by operand slicing in the manner of Ozaki, Ogita, Oishi and
// Rump ("Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer. Algorithms
// 59, 2012), with S slices of 8 bits per operand.  The scheme, per k chunk of
// TK = 32:
//   * row i of op(A) gets the exponent e_i with 2^(e_i) > max_k |a_ik|, column
//     j of op(B) the exponent f_j;
//   * a_ik = 2^(e_i) sum_{p=1..S} al_ik^(p) 2^(-8p) + r_ik with integers
//     |al^(p)| <= 255 (the bits of |a_ik| 2^(-e_i), 8 at a time, truncated:
//     |r_ik| < 2^(e_i - 8S)), exact in BF16; b_kj likewise with be^(q);
//   * the diagonal sums D_d = sum_{p+q=d} sum_{k in chunk} al^(p) be^(q),
//     d = 2..S+1, have at most S (p, q) pairs of TK integer products below
//     2^16: |D_d| <= S * 32 * 255^2 < 2^24, so the FP32 accumulation of the
//     tensor cores adds them without rounding;
//   * sum_k a_ik b_kj = 2^(e_i + f_j) sum_d 2^(-8d) D_d up to the dropped
//     products (p + q > S + 1) and the remainders: about (S + 3) 2^(-8S) TK
//     relative to max_k |a_ik| max_k |b_kj|.
// The D_d of a chunk are added to a compensated FP32 pair (TwoSum for d <= 4,
// plain FP32 sums of the smaller rest into the low word).  S = 7 (56 bits,
// 28 products per 16 x 8 x 16 step) reaches about FP64 accuracy (precision
// form 4); S = 5 (40 bits, 15 products) is the reduced form (precision 3).
// The accuracy is relative to the row and column maxima of each chunk: a row
// whose entries span 2^x in magnitude keeps 8S - x bits for its smallest ones.
// Elements below 2^-1022 count as zero; like the compensated FP32 form, the
// scaled partial sums must stay within FP32's exponent range.
constexpr int TK = 32;        // k chunk
constexpr int TKP = TK + 8;   // row length of a slice tile (BF16): conflict-free fragment loads

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// BF16 bits of the integer sg * v, 0 <= v <= 255 (exact: at most 8
// significant bits); v + 2^23 is an FP32 whose low bits hold v.
__device__ __forceinline__ uint32_t bf16_of_small(uint32_t v, uint32_t sg) {
  const float f = __uint_as_float(0x4B000000u | v) - 8388608.0f;
  return (__float_as_uint(f) >> 16) | sg;
}

// 2^E as FP32: 0 below the subnormal range, and 2^127 for E > 127 (outside
// the supported range of these forms; finite, so that a zero sum stays zero)
__device__ __forceinline__ float pow2f(int E) {
  if (E >= -126) return __uint_as_float((uint32_t)(min(E, 127) + 127) << 23);
  return E >= -149 ? __uint_as_float(1u << (E + 149)) : 0.0f;
}

// Fixed-point magnitude floor(|v| 2^(8S - e)) of an FP64 value v with
// biased exponent Ev, e = Emax - 1022 (Emax the largest biased exponent of
// its row or column): shift = 8S - 53 - (Emax - Ev).
template <int S>
__device__ __forceinline__ unsigned long long fixed_of_double(unsigned long long u, int Emax) {
  const int Ev = (int)((u >> 52) & 0x7ff);
  if (Ev == 0) return 0ull;
  const unsigned long long mant = (u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const int sh = 8 * S - 53 - (Emax - Ev);
  if (sh >= 0) return mant << sh;
  return -sh >= 64 ? 0ull : (mant >> -sh);
}

// Same for an FP32 value (a word of a compensated pair), its biased exponent
// mapped to the FP64 bias: shift = 8S - 24 - (Emax - Ev).
template <int S>
__device__ __forceinline__ unsigned long long fixed_of_float(uint32_t u, int Emax) {
  const int Ef = (int)((u >> 23) & 0xff);
  if (Ef == 0) return 0ull;
  const int Ev = Ef - 127 + 1023;
  const unsigned long long mant = (unsigned long long)((u & 0x7FFFFFu) | 0x800000u);
  const int sh = 8 * S - 24 - (Emax - Ev);
  if (sh >= 0) return sh >= 64 ? 0ull : (mant << sh);
  return -sh >= 64 ? 0ull : (mant >> -sh);
}

// Operand element as raw bits: an FP64 value, or a compensated pair (s, c)
// renormalised so that |c| <= ulp(s) / 2 (s in the high word).
struct TcRaw {
  unsigned long long u;
};

__device__ __forceinline__ TcRaw raw_of_double(double v) { return TcRaw{(unsigned long long)__double_as_longlong(v)}; }
__device__ __forceinline__ TcRaw raw_of_pair(float2 p) {
  // TwoSum: h + l = s + c exactly, l within half an ulp of h
  const float h = __fadd_rn(p.x, p.y);
  const float z = __fsub_rn(h, p.x);
  const float l = __fadd_rn(__fsub_rn(p.x, __fsub_rn(h, z)), __fsub_rn(p.y, z));
  return TcRaw{((unsigned long long)__float_as_uint(h) << 32) | __float_as_uint(l)};
}

// Biased FP64-scale exponent of an element (0 for zero): the value's own, or
// that of the pair's leading word.
template <bool PAIR>
__device__ __forceinline__ int raw_exp(TcRaw r) {
  if (!PAIR) return (int)((r.u >> 52) & 0x7ff);
  const int Ef = (int)((r.u >> 55) & 0xff);
  return Ef == 0 ? 0 : Ef - 127 + 1023;
}

// Writes the S slices of an element, scaled by its row or column exponent
// Emax, to dst[p * pstride] (BF16 bits).
template <int S, bool PAIR>
__device__ __forceinline__ void put_raw_slices(uint16_t* dst, int pstride, TcRaw r, int Emax) {
  unsigned long long a;
  bool neg;
  if (!PAIR) {
    a = fixed_of_double<S>(r.u, Emax);
    neg = (r.u >> 63) != 0ull;
  } else {
    const uint32_t us = (uint32_t)(r.u >> 32), uc = (uint32_t)r.u;
    long long f = (long long)fixed_of_float<S>(us, Emax);
    if (us >> 31) f = -f;
    const long long fc = (long long)fixed_of_float<S>(uc, Emax);
    f += (uc >> 31) ? -fc : fc;
    neg = f < 0;
    a = (unsigned long long)(neg ? -f : f);
  }
  const uint32_t sg = neg ? 0x8000u : 0u;
#pragma unroll
  for (int p = 1; p <= S; ++p) {
    const uint32_t v = (uint32_t)(a >> (8 * (S - p))) & 0xffu;
    dst[(p - 1) * pstride] = (uint16_t)bf16_of_small(v, sg);
  }
}

// Operand source of a chunk: global FP64 op(X) or the compensated pairs of a
// three-factor intermediate in shared memory (row-major, ld; never transposed).
struct TcSrc {
  const double* g;  // global matrix (nullptr: use s)
  const float2* s;  // shared pairs
  int ld, t;
};

constexpr int TC_NE = (64 * TK) / 256;  // elements of an operand chunk per thread at most

// Stages the slices of a chunk of an operand: rows 0..R16 (R16 = rows rounded
// up to 16 or 8) by k = k0..k0+TK, element (r, k) = X(r, k0 + k) where
// X(r, k) = g[r * ld + k] (along = true: consecutive k consecutive in memory)
// or g[k * ld + r] (along = false), or the shared pairs s[r * ld + k].
// Slices go to dst[p][r][k] (row length TKP), the exponents to rexp[r].
// along: a warp holds one row (lane = k), its maximum is a warp reduction;
// otherwise the maxima meet in shared memory (zeroed by the caller) and a
// second pass slices.  Each thread issues all of its loads before it slices
// (8 in flight instead of one; the GEMM stages of a product 21.8 -> 19.5 ms).
template <int S, bool PAIR>
__device__ __forceinline__ void tc_stage(uint16_t* dst, int R16, int* rexp, const TcSrc& X, bool along, int rows,
                                         int k0, int kc) {
  const int total = R16 * TK;
  const int pstride = R16 * TKP;
  if (along) {
    // all of this thread's loads first (independent, in flight together)
    TcRaw v[TC_NE];
#pragma unroll
    for (int it = 0; it < TC_NE; ++it) {
      const int e = threadIdx.x + 256 * it;
      const int r = e / TK, k = e % TK;
      v[it] = TcRaw{0ull};
      if (e < total && r < rows && k < kc) {
        if (PAIR) v[it] = raw_of_pair(X.s[r * X.ld + k0 + k]);
        else v[it] = raw_of_double(X.g[(int64_t)r * X.ld + k0 + k]);
      }
    }
#pragma unroll
    for (int it = 0; it < TC_NE; ++it) {
      const int e = threadIdx.x + 256 * it;
      if (e >= total) break;
      const int r = e / TK, k = e % TK;
      const TcRaw vi = v[it];
      const int Emax = __reduce_max_sync(0xffffffffu, raw_exp<PAIR>(vi));
      if ((threadIdx.x & 31) == 0) rexp[r] = Emax;
      put_raw_slices<S, PAIR>(dst + r * TKP + k, pstride, vi, Emax);
    }
    return;
  }
  // two passes over the elements held in registers.  A warp takes a block of
  // 8 rows x 4 k: 64-byte runs of consecutive r in memory, and slice stores
  // into 16 distinct banks (row length TKP = 20 words).
  const int nrb = R16 >> 3;
  TcRaw v[TC_NE];
#pragma unroll
  for (int it = 0; it < TC_NE; ++it) {
    const int e = threadIdx.x + 256 * it;
    const int b = e >> 5, ln = e & 31;
    const int r = (b % nrb) * 8 + (ln & 7), k = (b / nrb) * 4 + (ln >> 3);
    v[it] = (e < total && r < rows && k < kc) ? raw_of_double(X.g[(int64_t)(k0 + k) * X.ld + r]) : TcRaw{0ull};
  }
#pragma unroll
  for (int it = 0; it < TC_NE; ++it) {
    const int e = threadIdx.x + 256 * it;
    if (e >= total) break;
    const int b = e >> 5, ln = e & 31;
    const int r = (b % nrb) * 8 + (ln & 7);
    const int E = raw_exp<false>(v[it]);
    if (E) atomicMax(&rexp[r], E);
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < TC_NE; ++it) {
    const int e = threadIdx.x + 256 * it;
    if (e >= total) break;
    const int b = e >> 5, ln = e & 31;
    const int r = (b % nrb) * 8 + (ln & 7), k = (b / nrb) * 4 + (ln >> 3);
    put_raw_slices<S, false>(dst + r * TKP + k, pstride, v[it], rexp[r]);
  }
}

// Adds the diagonal sums D (d = j + 2) of fragment element (r, c), scaled by
// 2^(e_r + f_c - 8d) and alpha = ah + al, to the compensated pair (s, c):
// TwoSum for d <= 4, the smaller rest summed in FP32 into the low word.
template <int S>
__device__ __forceinline__ void tc_flush(float& ss, float& cc, const float (&D)[S][4], int e, int E0, float ah,
                                         float al) {
  float sc = pow2f(E0 - 16);
  float low = 0.0f;
#pragma unroll
  for (int j = 0; j < S; ++j) {
    const float v = D[j][e] * sc;  // exact (a power-of-two scaling of an integer below 2^24)
    sc *= 0.00390625f;             // 2^-8
    if (j < 3) {
      const float ph = __fmul_rn(ah, v);
      const float pl = fmaf(al, v, fmaf(ah, v, -ph));  // ah v = ph + exact error, plus al v
      const float t = __fadd_rn(ss, ph);
      const float z = __fsub_rn(t, ss);
      const float err = __fadd_rn(__fsub_rn(ss, __fsub_rn(t, z)), __fsub_rn(ph, z));
      ss = t;
      cc = __fadd_rn(cc, __fadd_rn(err, pl));
    } else {
      low = fmaf(ah, v, low);
    }
  }
  cc = __fadd_rn(cc, low);
}

// Accumulates alpha op(A)(m x K) op(B)(K x n) into this warp's fragment
// elements (tile = warp + 8 ti of the ceil(m/16) x ceil(n/8) tiles; element
// e: row g + 8 (e >> 1), column 2 tq + (e & 1) of the tile): into acc, or,
// with TOSMEM, into the compensated pairs ts[r * ldts + c] in shared memory.
template <int S, int TPW, bool APAIR, bool TOSMEM>
__device__ void tc_product(DF (&acc)[TPW][4], float2* ts, int ldts, const TcSrc& A, const double* B, int ldb,
                           int tb, int m, int n, int K, double alpha, uint16_t* As, uint16_t* Bs, int* rexp,
                           int* cexp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
  const int m16 = (m + 15) & ~15, n8 = (n + 7) & ~7;
  const int nt = n8 >> 3, ntiles = (m16 >> 4) * nt;
  const float2 al2 = split_df(alpha);
  const bool a_along = APAIR || !A.t, b_along = tb != 0;
  const TcSrc Bsrc{B, nullptr, ldb, tb};
  for (int k0 = 0; k0 < K; k0 += TK) {
    const int kc = min(TK, K - k0);
    __syncthreads();  // the previous chunk's slices and exponents are consumed
    if (!a_along || !b_along) {
      for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        if (!a_along) rexp[i] = 0;
        if (!b_along) cexp[i] = 0;
      }
      __syncthreads();
    }
    tc_stage<S, APAIR>(As, m16, rexp, A, a_along, m, k0, kc);
    tc_stage<S, false>(Bs, n8, cexp, Bsrc, b_along, n, k0, kc);
    __syncthreads();
    const int ksteps = (kc + 15) >> 4;
#pragma unroll
    for (int ti = 0; ti < TPW; ++ti) {
      const int tile = warp + 8 * ti;
      if (tile >= ntiles) break;
      const int tr = (tile / nt) * 16, tcn = (tile % nt) * 8;
      float D[S][4];
#pragma unroll
      for (int d = 0; d < S; ++d) D[d][0] = D[d][1] = D[d][2] = D[d][3] = 0.0f;
      for (int ks = 0; ks < ksteps; ++ks) {
        const int kb = ks * 16 + 2 * tq;
        uint32_t b0[S], b1[S];
#pragma unroll
        for (int q = 0; q < S; ++q) {
          const uint16_t* bp = Bs + q * n8 * TKP + (tcn + g) * TKP + kb;
          b0[q] = *reinterpret_cast<const uint32_t*>(bp);
          b1[q] = *reinterpret_cast<const uint32_t*>(bp + 8);
        }
#pragma unroll
        for (int p = 0; p < S; ++p) {
          const uint16_t* ap = As + p * m16 * TKP + (tr + g) * TKP + kb;
          const uint32_t a0 = *reinterpret_cast<const uint32_t*>(ap);
          const uint32_t a1 = *reinterpret_cast<const uint32_t*>(ap + 8 * TKP);
          const uint32_t a2 = *reinterpret_cast<const uint32_t*>(ap + 8);
          const uint32_t a3 = *reinterpret_cast<const uint32_t*>(ap + 8 * TKP + 8);
#pragma unroll
          for (int q = 0; q < S - p; ++q) mma_bf16(D[p + q], a0, a1, a2, a3, b0[q], b1[q]);
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = tr + g + 8 * (e >> 1), c = tcn + 2 * tq + (e & 1);
        if (r >= m || c >= n) continue;
        const int er = rexp[r], fc = cexp[c];
        if (er == 0 || fc == 0) continue;
        const int E0 = (er - 1022) + (fc - 1022);
        if (TOSMEM) {
          float2 v = ts[r * ldts + c];
          tc_flush<S>(v.x, v.y, D, e, E0, al2.x, al2.y);
          ts[r * ldts + c] = v;
        } else {
          tc_flush<S>(acc[ti][e].s, acc[ti][e].c, D, e, E0, al2.x, al2.y);
        }
      }
    }
  }
}

// One CTA per output tile (<= 64 x 64) of a GemmOut with its terms, as k_gemm,
// with every contraction on the tensor cores.  S slices (see above); TPW =
// tiles per warp of the stage's largest tile (1, 2 or 4).  A three-factor
// term alpha op(A) op(B) op(C) forms Ts = op(A) op(B) as compensated pairs in
// shared memory (when the stage has such terms: shared memory for them is
// part of the launch), then adds alpha Ts op(C).
template <int S, int TPW>
__device__ __forceinline__ void gemm_tc_job(const ExecCtx& x, const GemmOut& O, const GemmTerm* __restrict__ terms,
                                            int mmax, int nb) {
  extern __shared__ __align__(16) unsigned char tc_raw[];
  const int m16max = (mmax + 15) & ~15, n8max = (nb + 7) & ~7;
  uint16_t* As = reinterpret_cast<uint16_t*>(tc_raw);
  uint16_t* Bs = As + S * m16max * TKP;
  int* rexp = reinterpret_cast<int*>(Bs + S * n8max * TKP);
  int* cexp = rexp + 64;
  float2* Ts = reinterpret_cast<float2*>(cexp + 64);
  const int ldts = nb + 1;
  const int m = dimv(O.m, x.slot);
  const int n = O.clampn ? min(dimv(O.n, x.slot), GT) : dimv(O.n, x.slot);
  if (m <= 0 || n <= 0) return;
  if (m > mmax || n > nb || ((m + 15) / 16) * ((n + 7) / 8) > 8 * TPW) {
    if (threadIdx.x == 0) set_err(x, -9);
    return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
  const int nt = (n + 7) >> 3, ntiles = ((m + 15) >> 4) * nt;
  DF acc[TPW][4];
#pragma unroll
  for (int ti = 0; ti < TPW; ++ti)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[ti][e] = DF{0.0f, 0.0f};

  for (int tix = O.t0; tix < O.t1; ++tix) {
    const GemmTerm& Tm = terms[tix];
    double alpha = Tm.alpha;
    if (Tm.scale_idx >= 0) alpha *= x.scal[Tm.scale_idx];
    const double* A = ptrv(Tm.a, x);
    const double* B = ptrv(Tm.b, x);
    const double* C = ptrv(Tm.c, x);
    if (B == nullptr) {  // plain add of op(A) (m x n)
#pragma unroll
      for (int ti = 0; ti < TPW; ++ti) {
        const int tile = warp + 8 * ti;
        if (tile >= ntiles) break;
        const int tr = (tile / nt) * 16, tcn = (tile % nt) * 8;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = tr + g + 8 * (e >> 1), c = tcn + 2 * tq + (e & 1);
          if (r < m && c < n) GemmPol<GM_DF>::oadd_plain(acc[ti][e], alpha, ld_op(A, Tm.lda, Tm.ta, r, c));
        }
      }
      continue;
    }
    const int k1 = dimv(Tm.k1, x.slot);
    if (C == nullptr) {
      tc_product<S, TPW, false, false>(acc, nullptr, 0, TcSrc{A, nullptr, Tm.lda, Tm.ta}, B, Tm.ldb, Tm.tb, m, n,
                                       k1, alpha, As, Bs, rexp, cexp);
      continue;
    }
    // three-factor term: Ts = op(A) op(B) (m x nn), then alpha Ts op(C)
    const int nn = dimv(Tm.k2, x.slot);
    if (nn <= 0) continue;
    if (nn > nb || ((m + 15) / 16) * ((nn + 7) / 8) > 8 * TPW) {
      if (threadIdx.x == 0) set_err(x, -9);
      return;
    }
    __syncthreads();  // an earlier term's reads of Ts are done
    for (int e = threadIdx.x; e < m * ldts; e += blockDim.x) Ts[e] = make_float2(0.0f, 0.0f);
    tc_product<S, TPW, false, true>(acc, Ts, ldts, TcSrc{A, nullptr, Tm.lda, Tm.ta}, B, Tm.ldb, Tm.tb, m, nn, k1,
                                    1.0, As, Bs, rexp, cexp);
    tc_product<S, TPW, true, false>(acc, nullptr, 0, TcSrc{nullptr, Ts, ldts, 0}, C, Tm.ldc, Tm.tc, m, n, nn, alpha,
                                    As, Bs, rexp, cexp);
  }
  double* out = ptrv(O.o, x);
#pragma unroll
  for (int ti = 0; ti < TPW; ++ti) {
    const int tile = warp + 8 * ti;
    if (tile >= ntiles) break;
    const int tr = (tile / nt) * 16, tcn = (tile % nt) * 8;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = tr + g + 8 * (e >> 1), c = tcn + 2 * tq + (e & 1);
      if (r < m && c < n) {
        double* p = out + (int64_t)r * O.ldo + c;
        const double v = GemmPol<GM_DF>::result(acc[ti][e]);
        *p = O.beta ? (*p + v) : v;
      }
    }
  }
}

template <int S, int TPW>
__global__ void __launch_bounds__(256, 2)
    k_gemm_tc(const ExecCtx* __restrict__ px, const GemmOut* __restrict__ outs, const GemmTerm* __restrict__ terms,
              int mmax, int nb, const BatchSeg* __restrict__ segs, int nseg) {
  int b = blockIdx.x;
  if (segs) {
    const BatchSeg& sg = segs[seg_find(segs, nseg, b)];
    px = sg.ctx;
    outs = static_cast<const GemmOut*>(sg.jobs);
    terms = sg.terms;
    b -= sg.start;
  }
  gemm_tc_job<S, TPW>(*px, outs[b], terms, mmax, nb);
}

template <int S, int TPW>
__global__ void __launch_bounds__(256, 2)
    k_gemm_tc_chain(const BatchSeg* __restrict__ segs, int nseg, int total, int* ctr, int mmax, int nb) {
  chain_loop(segs, nseg, total, ctr, [&](const BatchSeg& sg, int i) {
    gemm_tc_job<S, TPW>(*sg.ctx, static_cast<const GemmOut*>(sg.jobs)[i], sg.terms, mmax, nb);
  });
}

// Dynamic shared memory of a tensor-core GEMM stage (bytes).
__host__ __device__ constexpr int gemm_tc_smem_bytes(int S, int mmax, int nb) {
  return 2 * S * (((mmax + 15) & ~15) + ((nb + 7) & ~7)) * TKP + 2 * 64 * 4 + 8 * mmax * (nb + 1);
}

// ------------------------------------------------------------------ copy ----
__global__ void __launch_bounds__(256) k_copy(const ExecCtx* __restrict__ px, const CopyJob* __restrict__ jobs,
                                              const BatchSeg* __restrict__ segs, int nseg) {
  int jb = blockIdx.x;
  if (segs) {
    const BatchSeg& sg = segs[seg_find(segs, nseg, jb)];
    px = sg.ctx;
    jobs = static_cast<const CopyJob*>(sg.jobs);
    jb -= sg.start;
  }
  const ExecCtx& x = *px;
  const CopyJob& J = jobs[jb];
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

// Householder reflector of x = [alpha; x2] with s2 = ||x2||^2 > 0:
// beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta = 1 + |alpha| / ||x||,
// v = [1; x2 / (alpha - beta)].  Written with one reciprocal square root and
// one reciprocal instead of a square root and two divisions: every FP64
// instruction costs a full warp issue on this GPU, and this runs once per
// column on the critical path.
__device__ __forceinline__ void householder_scalars(double alpha, double s2, double& beta, double& tau, double& sc) {
  const double n2 = fma(alpha, alpha, s2);
  const double r = rsqrt(n2);
  const double nrm = n2 * r;
  beta = -copysign(nrm, alpha);
  tau = fma(fabs(alpha), r, 1.0);
  sc = copysign(__drcp_rn(fabs(alpha) + nrm), alpha);
}

constexpr int QR_MAXPIV = 256;  // largest column count of a pivoted QR

// Unpivoted Householder QR of a column-major matrix (rows x cols, leading
// dimension lda, global or shared memory) with one step of look-ahead: while
// warps 1.. apply reflector j to columns j+2.., warp 0 applies it to column
// j+1 and forms reflector j+1 from the result, so a step needs one block
// barrier and the reflector's serial work overlaps the trailing update.
// Reflector scalars alternate between sh[0] and sh[1].  Returns min(rows, cols).
__device__ int householder_cols_la(double* a, int lda, int rows, int cols, double* tau, double* sh) {
  const int q = min(rows, cols);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q <= 0) return 0;
  // warp 0: reflector of column j from its current contents
  auto form = [&](int j) {
    double* col = a + (int64_t)j * lda;
    const double alpha = col[j];
    double s2 = 0.0;
    for (int i = j + 1 + lane; i < rows; i += 32) s2 = fma(col[i], col[i], s2);
    s2 = warp_sum(s2);
    double t = 0.0;
    if (s2 > 0.0) {
      double beta, sc;
      householder_scalars(alpha, s2, beta, t, sc);
      for (int i = j + 1 + lane; i < rows; i += 32) col[i] *= sc;
      __syncwarp();
      if (lane == 0) col[j] = beta;
    }
    if (lane == 0) {
      sh[j & 1] = t;
      if (tau) tau[j] = t;
    }
    __syncwarp();
  };
  // column c -= t v (v^T c), v = [1; col_j below j], by a team of ts lanes of one warp
  auto apply = [&](int j, double t, int c, int tl, int ts) {
    const double* vj = a + (int64_t)j * lda;
    double p = 0.0, cj = 0.0;
    double* cc = a + (int64_t)c * lda;
    if (c < cols) {
      cj = cc[j];
      for (int i = j + 1 + tl; i < rows; i += ts) p = fma(vj[i], cc[i], p);
    }
    for (int o = ts >> 1; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    const double w = t * (cj + p);
    if (c < cols) {
      if (tl == 0) cc[j] -= w;
      for (int i = j + 1 + tl; i < rows; i += ts) cc[i] = fma(-w, vj[i], cc[i]);
    }
  };
  if (warp == 0) form(0);
  __syncthreads();
  for (int j = 0; j < q; ++j) {
    const double t = sh[j & 1];
    if (warp == 0) {
      if (j + 1 < cols) {
        if (t != 0.0) apply(j, t, j + 1, lane, 32);
        __syncwarp();
        if (j + 1 < q) form(j + 1);
      }
    } else if (t != 0.0) {
      const int len = rows - j - 1;
      int ts = 32;
      while (ts > 1 && ts * 16 > len) ts >>= 1;
      const int tid = threadIdx.x - 32, nteam = ((int)blockDim.x - 32) / ts, team = tid / ts, tl = tid % ts;
      for (int c0 = j + 2; c0 < cols; c0 += nteam) apply(j, t, c0 + team, tl, ts);
    }
    __syncthreads();
  }
  return q;
}

// Householder QR on a column-major matrix a (rows x cols, leading dimension
// lda), in place; `a` is global or shared memory.  With piv != nullptr the
// columns are pivoted (column of largest remaining norm first, lowest index on
// ties): cn holds the squared norms of the trailing parts, downdated after each
// step and recomputed exactly where the downdate has cancelled below 2^-26 of
// the value at the last recomputation; cn0 holds 2^-26 times that value.
//
// Each step: warp 0 alone picks the pivot, swaps, forms the reflector and
// scales it (no block barrier inside), then all warps update the trailing
// columns; two block barriers per step.  Without pivoting the look-ahead
// variant above runs instead.
//
// With pivoting and floor2 > 0 the factorisation stops at the first step j
// whose trailing columns hold a squared Frobenius norm (the sum of cn) <=
// floor2 * ||a||_F^2; tau[j..] is then 0.  Returns the number of steps taken.
__device__ int householder_cols(double* a, int lda, int rows, int cols, double* tau, double* sh, int* piv,
                                double* cn, double* cn0, double floor2 = -1.0) {
  if (!piv) return householder_cols_la(a, lda, rows, cols, tau, sh);
  const int q = min(rows, cols);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  constexpr double kRecompute = 1.4901161193847656e-08;  // 2^-26
  double thr = -1.0;  // truncation threshold (warp 0)
  if (piv) {
    for (int c = threadIdx.x; c < cols; c += blockDim.x) piv[c] = c;
    for (int c = warp; c < cols; c += nwarp) {
      const double* cc = a + (int64_t)c * lda;
      double s = 0.0;
      for (int i = lane; i < rows; i += 32) s = fma(cc[i], cc[i], s);
      s = warp_sum(s);
      if (lane == 0) {
        cn[c] = s;
        cn0[c] = s * kRecompute;
      }
    }
    __syncthreads();
    if (floor2 > 0.0 && warp == 0) {
      double s = 0.0;
      for (int c = lane; c < cols; c += 32) s += cn[c];
      thr = floor2 * warp_sum(s);
    }
  }
  int steps = q;
  for (int j = 0; j < q; ++j) {
    double* col = a + (int64_t)j * lda;
    if (warp == 0) {
      bool stop = false;
      if (piv) {
        // largest trailing norm: the norms are never negative, so their
        // FP64 bit patterns order like the values and compare as integers
        // (no FP64 instruction on this serial step)
        long long bv = -1;
        double rs = 0.0;
        int bi = j;
        for (int c = j + lane; c < cols; c += 32) {
          const double v = cn[c];
          if (thr >= 0.0) rs += v;
          const long long vb = __double_as_longlong(v);
          if (vb > bv) {
            bv = vb;
            bi = c;
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ov > bv || (ov == bv && oi < bi)) {
            bv = ov;
            bi = oi;
          }
        }
        if (thr >= 0.0) stop = warp_sum(rs) <= thr;  // the same sum in every lane
        if (!stop && bi != j) {
          double* cp = a + (int64_t)bi * lda;
          for (int i = lane; i < rows; i += 32) {
            const double t = col[i];
            col[i] = cp[i];
            cp[i] = t;
          }
          if (lane == 0) {
            double t = cn[j];
            cn[j] = cn[bi];
            cn[bi] = t;
            t = cn0[j];
            cn0[j] = cn0[bi];
            cn0[bi] = t;
            const int pi = piv[j];
            piv[j] = piv[bi];
            piv[bi] = pi;
          }
          __syncwarp();
        }
      }
      double t = 0.0;
      if (!stop) {
        double s2 = 0.0;
        for (int i = j + 1 + lane; i < rows; i += 32) s2 = fma(col[i], col[i], s2);
        s2 = warp_sum(s2);
        const double alpha = col[j];
        double sc = 0.0;
        if (s2 > 0.0) {
          double beta;
          householder_scalars(alpha, s2, beta, t, sc);
          for (int i = j + 1 + lane; i < rows; i += 32) col[i] *= sc;
          __syncwarp();
          if (lane == 0) col[j] = beta;
        }
      }
      if (lane == 0) {
        sh[0] = t;
        sh[1] = stop ? 1.0 : 0.0;
        if (tau) tau[j] = t;
      }
    }
    __syncthreads();
    if (sh[1] != 0.0) {
      steps = j;
      break;
    }
    const double t = sh[0];
    if (t != 0.0) {
      // trailing columns: teams of ts lanes per column, at least 16 rows per
      // lane (the FP64 shuffle reduction of a team costs log2(ts) full warp
      // issues per column; 8 rows per lane measured 2% slower, 32 rows 20%
      // slower through idle teams)
      const int len = rows - j - 1;
      int ts = 32;
      while (ts > 1 && ts * 16 > len) ts >>= 1;
      const int nteam = blockDim.x / ts, team = threadIdx.x / ts, tl = threadIdx.x % ts;
      for (int c0 = j + 1; c0 < cols; c0 += nteam) {
        const int c = c0 + team;
        double p = 0.0, cj = 0.0;
        double* cc = a + (int64_t)c * lda;
        if (c < cols) {
          cj = cc[j];  // read by every lane before the shuffle (lane 0 writes it below)
          for (int i = j + 1 + tl; i < rows; i += ts) p = fma(col[i], cc[i], p);
        }
        for (int o = ts >> 1; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        const double w = t * (cj + p);
        const double rj = cj - w;  // new row-j entry
        if (c < cols) {
          if (tl == 0) cc[j] = rj;
          for (int i = j + 1 + tl; i < rows; i += ts) cc[i] = fma(-w, col[i], cc[i]);
        }
        if (piv) {
          // downdate the trailing norm by the new row-j entry; recompute on cancellation
          // (cn0 >= 0: a negative or -0 downdate reads as a negative integer)
          const double nd = c < cols ? cn[c] - rj * rj : 0.0;
          const bool need = c < cols && __double_as_longlong(nd) <= __double_as_longlong(cn0[c]);
          if (__any_sync(0xffffffffu, need)) {
            double e = 0.0;
            if (need)
              for (int i = j + 1 + tl; i < rows; i += ts) e = fma(cc[i], cc[i], e);
            for (int o = ts >> 1; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
            if (need && tl == 0) {
              cn[c] = e;
              cn0[c] = e * kRecompute;
            }
          }
          if (c < cols && !need && tl == 0) cn[c] = nd;
        }
      }
    } else if (piv) {
      // no reflection: the trailing parts lose row j only
      for (int c = j + 1 + threadIdx.x; c < cols; c += blockDim.x) {
        const double* cc = a + (int64_t)c * lda;
        const double nd = cn[c] - cc[j] * cc[j];
        if (nd <= cn0[c]) {
          double e = 0.0;
          for (int i = j + 1; i < rows; ++i) e = fma(cc[i], cc[i], e);
          cn[c] = e;
          cn0[c] = e * kRecompute;
        } else {
          cn[c] = nd;
        }
      }
    }
    __syncthreads();
  }
  if (tau)
    for (int c = steps + threadIdx.x; c < q; c += blockDim.x) tau[c] = 0.0;
  return steps;
}

// R factor of a tall column-major matrix a (rows x cols) without its Q:
// row chunks of a stream through shared memory under the triangle accumulated
// so far, W = [R (cols x cols); chunk (ch x cols)], leading dimension ld.  Each
// chunk is annihilated column by column by reflectors that touch row j of R
// and the chunk only (the triangle-on-top step of a tall-skinny QR), so the
// flop count equals that of Householder QR on a and every load of a is one
// coalesced pass.  On return W's upper cols x cols triangle holds R.
__device__ void tsqr_r(const double* __restrict__ a, int lda, int rows, int cols, double* W, int ld, int ch_max,
                       double* sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* C = W + cols;  // chunk rows start below the triangle
  for (int e = threadIdx.x; e < cols * cols; e += blockDim.x) W[(e / cols) * ld + e % cols] = 0.0;
  for (int r0 = 0; r0 < rows; r0 += ch_max) {
    const int ch = min(ch_max, rows - r0);
    for (int e0 = threadIdx.x; e0 < ch * cols; e0 += 8 * blockDim.x) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x;
        v[u] = e < ch * cols ? a[(int64_t)(e / ch) * lda + r0 + e % ch] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < ch * cols) C[(e / ch) * ld + e % ch] = v[u];
      }
    }
    __syncthreads();
    // one step of look-ahead, as in householder_cols_la: while warps 1..
    // apply reflector j to columns j+2.., warp 0 applies it to column j+1 and
    // forms reflector j+1; the scalars alternate between sh[0] and sh[1]
    auto form = [&](int j) {  // warp 0: reflector of [W(j, j); C(:, j)]
      double* cj = C + j * ld;
      double s2 = 0.0;
      for (int i = lane; i < ch; i += 32) s2 = fma(cj[i], cj[i], s2);
      s2 = warp_sum(s2);
      const double alpha = W[j * ld + j];
      double t = 0.0;
      if (s2 > 0.0) {
        double beta, sc;
        householder_scalars(alpha, s2, beta, t, sc);
        for (int i = lane; i < ch; i += 32) cj[i] *= sc;
        __syncwarp();
        if (lane == 0) W[j * ld + j] = beta;
      }
      if (lane == 0) sh[j & 1] = t;
      __syncwarp();
    };
    // [W(j, c); C(:, c)] -= t v (v^T [W(j, c); C(:, c)]), v = [1; C(:, j)], by a
    // team of ts lanes of one warp
    auto apply = [&](int j, double t, int c, int tl, int ts) {
      const double* cj = C + j * ld;
      double p = 0.0, rjc = 0.0;
      double* cc = C + c * ld;
      if (c < cols) {
        rjc = W[c * ld + j];  // read by every lane before the shuffle (lane 0 writes it below)
        for (int i = tl; i < ch; i += ts) p = fma(cj[i], cc[i], p);
      }
      for (int o = ts >> 1; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
      if (c < cols) {
        const double w = t * (rjc + p);
        if (tl == 0) W[c * ld + j] = rjc - w;
        for (int i = tl; i < ch; i += ts) cc[i] = fma(-w, cj[i], cc[i]);
      }
    };
    int ts = 32;
    while (ts > 1 && ts * 16 > ch) ts >>= 1;
    const int tid = threadIdx.x - 32, nteam = ((int)blockDim.x - 32) / ts, team = tid / ts, tl = tid % ts;
    if (warp == 0) form(0);
    __syncthreads();
    for (int j = 0; j < cols; ++j) {
      const double t = sh[j & 1];
      if (warp == 0) {
        if (j + 1 < cols) {
          if (t != 0.0) apply(j, t, j + 1, lane, 32);
          __syncwarp();
          form(j + 1);
        }
      } else if (t != 0.0) {
        for (int c0 = j + 2; c0 < cols; c0 += nteam) apply(j, t, c0 + team, tl, ts);
      }
      __syncthreads();
    }
  }
}

constexpr int QR_TSQR_MAXC = 64;       // widest R-only factorisation that streams row chunks
constexpr int QR_MAX_SMEM_BYTES = 8 * (QR_TSQR_MAXC + 128) * QR_TSQR_MAXC;  // 96 KB

// R output of a QR job (see QrJob::rmode): R(i, c) = src[c * lds + i] above
// the diagonal for i < q, zero elsewhere.  Call after a block barrier (the
// pivot order and src are complete).
__device__ void write_r(const QrJob& J, double* r, const double* src, int64_t lds, int cols, int q, const int* piv) {
  const bool unpiv = (J.rmode & 1) && piv;
  const bool trans = (J.rmode & 2) != 0;
  for (int e = threadIdx.x; e < cols * cols; e += blockDim.x) {
    // consecutive threads write consecutive addresses of r
    const int i = trans ? e % cols : e / cols, c = trans ? e / cols : e % cols;
    const double v = (src && c >= i && i < q) ? src[(int64_t)c * lds + i] : 0.0;
    const int dc = unpiv ? piv[c] : c;
    r[trans ? (int64_t)dc * J.ldr + i : (int64_t)i * J.ldr + dc] = v;
  }
}

__global__ void __launch_bounds__(256) k_qr(const ExecCtx* __restrict__ px, const QrJob* __restrict__ jobs,
                                            int smem_doubles, const BatchSeg* __restrict__ segs, int nseg) {
  int jb = blockIdx.x;
  if (segs) {
    const BatchSeg& sg = segs[seg_find(segs, nseg, jb)];
    px = sg.ctx;
    jobs = static_cast<const QrJob*>(sg.jobs);
    jb -= sg.start;
  }
  const ExecCtx& x = *px;
  extern __shared__ double sm[];
  __shared__ double sh[2];
  __shared__ double cn[QR_MAXPIV], cn0[QR_MAXPIV];
  const QrJob& J = jobs[jb];
  const int rows = dimv(J.rows, x.slot), cols = dimv(J.cols, x.slot);
  double* a = ptrv(J.a, x);
  double* tau = ptrv(J.tau, x);
  double* r = ptrv(J.r, x);
  int* piv = reinterpret_cast<int*>(ptrv(J.piv, x));
  if (piv && cols > QR_MAXPIV) {
    // too wide to pivot: unpivoted factorisation, identity order
    for (int c = threadIdx.x; c < cols; c += blockDim.x) piv[c] = c;
    piv = nullptr;
  }
  const int lda = J.lda;
  const int q = min(rows, cols);
  // truncation at a noise floor (pivoted factorisations only)
  const double floor2 = (piv && J.trunc_idx >= 0) ? x.scal[J.trunc_idx] : -1.0;
  int* rank_out = J.rank_slot >= 0 ? x.slot + J.rank_slot : nullptr;
  if (rows <= 0 || cols <= 0) {
    if (r) write_r(J, r, nullptr, 0, cols, 0, nullptr);
    if (piv)
      for (int c = threadIdx.x; c < cols; c += blockDim.x) piv[c] = c;
    if (rank_out && threadIdx.x == 0) *rank_out = 0;
    return;
  }
  if ((int64_t)rows * cols <= smem_doubles) {
    // whole matrix in shared memory
    {
      const int64_t tot = (int64_t)rows * cols;
      for (int64_t e0 = threadIdx.x; e0 < tot; e0 += 8 * (int64_t)blockDim.x) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int64_t e = e0 + (int64_t)u * blockDim.x;
          v[u] = e < tot ? a[(int64_t)(e / rows) * lda + e % rows] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int64_t e = e0 + (int64_t)u * blockDim.x;
          if (e < tot) sm[e] = v[u];
        }
      }
    }
    __syncthreads();
    const int rk = householder_cols(sm, rows, rows, cols, tau, sh, piv, cn, cn0, floor2);
    if (J.keep)
      for (int64_t e = threadIdx.x; e < (int64_t)rows * cols; e += blockDim.x) {
        const int c = (int)(e / rows), i = (int)(e % rows);
        a[(int64_t)c * lda + i] = sm[e];
      }
    if (r) write_r(J, r, sm, rows, cols, rk, piv);
    if (rank_out && threadIdx.x == 0) *rank_out = rk;
    return;
  }
  if (!J.keep && cols <= QR_TSQR_MAXC && smem_doubles / cols - cols >= 16) {
    // R only, tall: stream row chunks through shared memory, then pivot the
    // (cols x cols) triangle; the reflectors are not kept (no Q application
    // follows an R-only job)
    const int ld = smem_doubles / cols;
    tsqr_r(a, lda, rows, cols, sm, ld, ld - cols, sh);
    // the triangle has the Frobenius norm of a: the same truncation applies
    const int rk = piv ? householder_cols(sm, ld, cols, cols, nullptr, sh, piv, cn, cn0, floor2) : q;
    if (tau)
      for (int c = threadIdx.x; c < q; c += blockDim.x) tau[c] = 0.0;
    if (r) write_r(J, r, sm, ld, cols, rk, piv);
    if (rank_out && threadIdx.x == 0) *rank_out = rk;
    return;
  }
  // general case: in place in global memory
  const int rk = householder_cols(a, lda, rows, cols, tau, sh, piv, cn, cn0, floor2);
  if (r) write_r(J, r, a, lda, cols, rk, piv);
  if (rank_out && threadIdx.x == 0) *rank_out = rk;
}

// out = H_0 ... H_{q-1} [Y; 0], the reflectors applied QB at a time (last
// block first).  For a block H_{j0} ... H_{j1-1} and each column o of out:
//   d_k = v_k^T o (all k of the block, one pass over o),
//   w_k = tau_k (d_k - sum_{m > k} (v_k^T v_m) w_m)   (k = j1-1 down to j0),
//   o  -= sum_k v_k w_k                                (one more pass),
// which equals applying H_{j1-1} first and H_{j0} last.  Threads: column
// c = tid % nc of out, row segment tid / nc; the partial dots meet in shared
// memory and one thread per column sums them (no FP64 shuffle reductions on
// the columns); the block's reflector products v_k^T v_m are one warp each.
// A block reads and writes out once and takes three barriers, not QB times.
constexpr int QB = 4;
__global__ void __launch_bounds__(256) k_qapply(const ExecCtx* __restrict__ px, const QApplyJob* __restrict__ jobs,
                                                const BatchSeg* __restrict__ segs, int nsegs) {
  int jb = blockIdx.x;
  if (segs) {
    const BatchSeg& sg = segs[seg_find(segs, nsegs, jb)];
    px = sg.ctx;
    jobs = static_cast<const QApplyJob*>(sg.jobs);
    jb -= sg.start;
  }
  const ExecCtx& x = *px;
  __shared__ double part[QB][256];
  __shared__ double wsh[QB][256];
  __shared__ double gsh[QB * QB];
  const QApplyJob& J = jobs[jb];
  const int rows = dimv(J.rows, x.slot), q = dimv(J.q, x.slot), nc = dimv(J.ncols, x.slot);
  const double* a = ptrv(J.a, x);
  const double* tau = ptrv(J.tau, x);
  const double* y = ptrv(J.y, x);
  double* out = ptrv(J.out, x);
  const int ldo = J.ldo, lda = J.lda;
  if (nc > (int)blockDim.x) {
    if (threadIdx.x == 0) set_err(x, -9);
    return;
  }
  for (int64_t e = threadIdx.x; e < (int64_t)rows * nc; e += blockDim.x) {
    int i = (int)(e / nc), c = (int)(e % nc);
    out[(int64_t)i * ldo + c] = (i < q) ? y[(int64_t)i * J.ldy + c] : 0.0;
  }
  if (nc <= 0) return;
  __syncthreads();
  const int nseg = blockDim.x / nc;
  const int c = threadIdx.x % nc, sg = threadIdx.x / nc;
  const bool active = sg < nseg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  // v_k[i]: 1 at i = k, the stored reflector below, 0 above
  auto vk = [&](int k, int i) { return i > k ? a[(int64_t)k * lda + i] : (i == k ? 1.0 : 0.0); };
  for (int j1 = min(q, rows); j1 > 0; j1 -= QB) {
    const int j0 = max(0, j1 - QB), nb = j1 - j0;
    // v_u^T v_m for u < m of the block, one warp each
    for (int pr = warp; pr < QB * QB; pr += nwarp) {
      const int u = pr / QB, m = pr % QB;
      if (u < m && m < nb) {
        const int ku = j0 + u, km = j0 + m;
        double sdot = 0.0;
        for (int i = km + 1 + lane; i < rows; i += 32)
          sdot = fma(a[(int64_t)ku * lda + i], a[(int64_t)km * lda + i], sdot);
        sdot = warp_sum(sdot);
        if (lane == 0) gsh[u * QB + m] = a[(int64_t)ku * lda + km] + sdot;
      }
    }
    if (active) {
      double d[QB];
#pragma unroll
      for (int u = 0; u < QB; ++u) d[u] = 0.0;
      for (int i = j0 + sg; i < rows; i += nseg) {
        const double o = out[(int64_t)i * ldo + c];
#pragma unroll
        for (int u = 0; u < QB; ++u)
          if (u < nb) d[u] = fma(vk(j0 + u, i), o, d[u]);
      }
#pragma unroll
      for (int u = 0; u < QB; ++u) part[u][sg * nc + c] = d[u];
    }
    __syncthreads();
    if ((int)threadIdx.x < nc) {
      for (int u = nb - 1; u >= 0; --u) {
        double sum = part[u][threadIdx.x];
        for (int g = 1; g < nseg; ++g) sum += part[u][g * nc + threadIdx.x];
        for (int m = u + 1; m < nb; ++m) sum -= gsh[u * QB + m] * wsh[m][threadIdx.x];
        wsh[u][threadIdx.x] = tau[j0 + u] * sum;
      }
    }
    __syncthreads();
    if (active) {
      double w[QB];
#pragma unroll
      for (int u = 0; u < QB; ++u) w[u] = u < nb ? wsh[u][c] : 0.0;
      for (int i = j0 + sg; i < rows; i += nseg) {
        double o = out[(int64_t)i * ldo + c];
#pragma unroll
        for (int u = 0; u < QB; ++u)
          if (u < nb) o = fma(-vk(j0 + u, i), w[u], o);
        out[(int64_t)i * ldo + c] = o;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------- SVD ----
// One-sided (Hestenes) Jacobi: rotate pairs of columns of M until all pairs are
// orthogonal to relative precision; the column norms are the singular values
// and the normalised columns the left singular vectors.  Pairs follow the
// round-robin (circle) ordering so that cols/2 disjoint pairs rotate at once.
// Squared column norms are kept in shared memory, updated after each rotation
// (alpha' = alpha - t*gamma, beta' = beta + t*gamma) and recomputed exactly at
// the start of every sweep.
//
// The FP64 pipe issues a warp instruction at the same cost however many lanes
// it uses, so the rounds are laid out to issue few of them:
//  - dot products: one lane per pair, the warps splitting the rows; the
//    partial sums meet in shared memory (no shuffle-add chains);
//  - rotations in scaled form: M = Mt diag(d), and the rotation by
//    (c, s = c t) of columns i, j becomes Mt_i -= (t d_j/d_i) Mt_j,
//    Mt_j += (t d_i/d_j) Mt_i (one FMA per element), d_i, d_j *= c; the
//    scales are folded back into M at the start of every sweep, so Mt grows
//    by at most 2^(cols/2) within a sweep (|t| <= 1);
//  - only the pairs that rotate are visited, from a compacted list.
constexpr int SVD_MAXSWEEP = 60;

// v 2^k as FP32 by bit operations (no FP64 instruction): the exponent
// re-biased, the fraction truncated to 23 bits; 0 when v is zero or v 2^k is
// below FP32's normal range.  The callers keep v 2^k below 2^127.
__device__ __forceinline__ float f32_of_scaled(double v, int k) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
  const int eb = (int)((hw >> 20) & 0x7ffu);
  const int e = eb - 1023 + k;
  if (eb == 0 || e < -126) return 0.0f;
  return __uint_as_float((hw & 0x80000000u) | ((unsigned)(e + 127) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
}

// f 2^k as FP64, exactly, by bit operations (f normal or zero)
__device__ __forceinline__ double f64_of_f32_scaled(float f, int k) {
  const unsigned u = __float_as_uint(f);
  const int ef = (int)((u >> 23) & 0xffu);
  if (ef == 0) return 0.0;
  const unsigned hw = (u & 0x80000000u) | ((unsigned)(ef - 127 + 1023 + k) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hw, (int)((u & 0x7u) << 29));
}

// Round-robin (circle method) pairing of ce (even) columns: in round rnd, pair
// p matches columns i < j; over ce-1 rounds every pair meets once.
__device__ __forceinline__ int svd_pair_a(int rnd, int p, int ce) { return p == 0 ? rnd : (rnd + p) % (ce - 1); }
__device__ __forceinline__ int svd_pair_b(int rnd, int p, int ce) {
  return p == 0 ? ce - 1 : (rnd - p + ce - 1) % (ce - 1);
}
__device__ __forceinline__ int svd_pair_i(int rnd, int p, int ce) {
  return min(svd_pair_a(rnd, p, ce), svd_pair_b(rnd, p, ce));
}
__device__ __forceinline__ int svd_pair_j(int rnd, int p, int ce) {
  return max(svd_pair_a(rnd, p, ce), svd_pair_b(rnd, p, ce));
}

// A launch may take only the jobs whose shared-memory need (per-column
// arrays and matrix, in doubles; 0 for an empty job) lies in
// (need_lo, need_hi]: a stage of mixed sizes then runs its small jobs in
// small CTAs, many per SM, and its large ones in a second launch.
__global__ void __launch_bounds__(256, 3) k_svd(const ExecCtx* __restrict__ px, const SvdJob* __restrict__ jobs,
                                                int64_t first, int smem_doubles, int cmax, int need_lo, int need_hi,
                                                const BatchSeg* __restrict__ segs, int nsegs) {
  int jb = blockIdx.x;
  if (segs) {
    const BatchSeg& sg = segs[seg_find(segs, nsegs, jb)];
    px = sg.ctx;
    jobs = static_cast<const SvdJob*>(sg.jobs);
    jb -= sg.start;
    first = sg.first;
  }
  const ExecCtx& x = *px;
  extern __shared__ double sdyn[];
  __shared__ int rotated;
  __shared__ int nrot;
  __shared__ int nround;
  __shared__ double part[256];  // partial dot products (blockDim <= 256)
  __shared__ double s_fro;
  const SvdJob& J = jobs[jb];
  const int rows = dimv(J.rows, x.slot), cols = dimv(J.cols, x.slot);
  {
    const int64_t need = (rows <= 0 || cols <= 0) ? 0 : svd_colarr_doubles(cols) + (int64_t)(rows + 1) * cols;
    if (need <= need_lo || need > need_hi) return;  // the other launch of the stage
  }
  // per-column arrays sized for this job's columns, the matrix behind them
  const int ca = svd_colarr_doubles(cols);
  double* nrm2 = sdyn;                 // squared column norms
  double* dsc = nrm2 + cols;           // column scales d of M = Mt diag(d)
  double* dinv = dsc + cols;           // 1/d
  double* snorm = dinv + cols;         // singular values
  double* rfa = snorm + cols;          // rotation factors of the round's rotating pairs
  double* rfb = rfa + (cols / 2 + 1);
  int* spos = reinterpret_cast<int*>(rfb + (cols / 2 + 1));  // sorted position of each column
  int* rlist = spos + cols;            // rotating pairs of the round: (i << 16) | j
  double* sm = sdyn + ca;
  int* rank_out = (J.rank_slot >= 0) ? x.slot + J.rank_slot : nullptr;
  if (rows <= 0 || cols <= 0) {
    if (threadIdx.x == 0) {
      if (rank_out) *rank_out = 0;
      if (J.norm_idx >= 0) {
        x.nrm[J.norm_idx] = 0.0;
        x.scal[J.norm_idx] = 0.0;
      }
    }
    return;
  }
  const bool fits = ca + (int64_t)(rows + 1) * cols <= smem_doubles;
  if (rows > SVD_MAXDIM || cols > cmax || ca > smem_doubles || (!fits && !J.trans)) {
    if (threadIdx.x == 0) {
      set_err(x, -9);
      if (rank_out) *rank_out = 0;
    }
    return;
  }
  // M in shared memory when it fits the launch, else in place in the source
  // (only for transposed sources, whose rows are M's columns; the planner
  // passes scratch copies that are not needed afterwards)
  double* S = ptrv(J.src, x);
  const bool in_smem = fits || !J.trans;
  const int ldm = in_smem ? rows + 1 : J.lds;
  double* M = in_smem ? sm : S;  // column c at M + c*ldm
  // (consecutive threads read consecutive source addresses)
  if (in_smem && J.trans)
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int c = e / rows, r = e % rows;
      M[c * ldm + r] = S[(int64_t)c * J.lds + r];
    }
  else if (in_smem)
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int r = e / cols, c = e % cols;
      M[c * ldm + r] = S[(int64_t)r * J.lds + c];
    }
  if (threadIdx.x == 0) nrot = 0;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    dsc[c] = 1.0;
    dinv[c] = 1.0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  // fold the scales into M, then exact squared column norms (one warp per column)
  auto col_norms = [&]() {
    for (int c = warp; c < cols; c += nwarp) {
      const double dc = dsc[c];
      double* mc = M + c * ldm;
      double p = 0.0;
      if (dc != 1.0) {
        for (int r = lane; r < rows; r += 32) {
          const double v = mc[r] * dc;
          mc[r] = v;
          p = fma(v, v, p);
        }
      } else {
        for (int r = lane; r < rows; r += 32) p = fma(mc[r], mc[r], p);
      }
      p = warp_sum(p);
      if (lane == 0) {
        nrm2[c] = p;
        dsc[c] = 1.0;
        dinv[c] = 1.0;
      }
    }
    __syncthreads();
  };
  col_norms();
  if (threadIdx.x == 0) {
    double f = 0.0;
    for (int c = 0; c < cols; ++c) f += nrm2[c];
    s_fro = f;
  }
  __syncthreads();
  // columns below the noise floor (2^-50 ||M||_F for FP64 inputs) are
  // rounding noise: never rotated, sigma = 0
  const double tiny2 = s_fro * x.scal[PARAM_SVD_FLOOR];
  const int ce = cols + (cols & 1);
  const int npairs = ce / 2;
  const double tol = 2.5e-15;
  // dot products: thread -> (pair, row segment); at most 4 segments, so that
  // phase B sums few partials (every FP64 add there is a full warp issue;
  // 4 measured 1% faster than 8, 16 and more 3% slower)
  const int nseg = min(4, (int)blockDim.x / npairs);
  const int ap = threadIdx.x % npairs, aseg = threadIdx.x / npairs;
  const int maxsweep = x.scal[PARAM_SVD_SWEEPS] >= 1.0 ? (int)x.scal[PARAM_SVD_SWEEPS] : SVD_MAXSWEEP;
  int sweep = 0;
  for (; sweep < maxsweep; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < ce - 1; ++rnd) {
      // phase A: partial dot products of the round's pairs
      if (aseg < nseg) {
        const int i = svd_pair_i(rnd, ap, ce), j = svd_pair_j(rnd, ap, ce);
        double g = 0.0, h = 0.0;
        if (j < cols) {
          const double* mi = M + i * ldm;
          const double* mj = M + j * ldm;
          int r = aseg;
          for (; r + nseg < rows; r += 2 * nseg) {
            g = fma(mi[r], mj[r], g);
            h = fma(mi[r + nseg], mj[r + nseg], h);
          }
          if (r < rows) g = fma(mi[r], mj[r], g);
        }
        part[aseg * npairs + ap] = g + h;
      }
      if (threadIdx.x == 0) nround = 0;
      __syncthreads();
      // phase B: one thread per pair sums the partials and sets up the rotation
      if (threadIdx.x < npairs) {
        const int p = threadIdx.x;
        const int i = svd_pair_i(rnd, p, ce), j = svd_pair_j(rnd, p, ce);
        if (j < cols) {
          double gt = part[p];
          for (int sg = 1; sg < nseg; ++sg) gt += part[sg * npairs + p];
          const double di = dsc[i], dj = dsc[j];
          const double ga = gt * di * dj, al = nrm2[i], be = nrm2[j];
          // |ga| > tol * sqrt(al * be), in squared form; the squared norms and
          // the floor are never negative, so those tests compare FP64 bit
          // patterns as integers (no FP64 instruction)
          const long long tb = __double_as_longlong(tiny2);
          if ((__double_as_longlong(ga) << 1) != 0 && __double_as_longlong(al) > tb &&
              __double_as_longlong(be) > tb && ga * ga > (tol * tol) * al * be) {
            // t = tan(theta), the smaller root of f(t) = g2 t^2 + 2 d t - g2
            // (d = be - al, g2 = 2 ga): first in FP32 as
            // t = sign(d) g2 / (|d| + sqrt(d^2 + g2^2)) from d and g2 scaled by
            // 2^k into [1, 2), then one Newton step in FP64 (t to ~1e-14; the
            // angle only steers convergence).  The rotation itself is exact:
            // c = 1 / sqrt(1 + t^2) in FP64 from an FP32 seed and two Newton
            // steps, s = c t.  FP64 work on this serial step: 14 instructions
            // instead of about 30 with an FP64 square root and division.
            const double d0 = be - al, g0 = ga + ga;
            const int k = 1023 - max((__double2hiint(d0) >> 20) & 0x7ff, (__double2hiint(g0) >> 20) & 0x7ff);
            const float df = f32_of_scaled(d0, k), gf = f32_of_scaled(g0, k);
            const float tf = copysignf(1.0f, df) * gf / (fabsf(df) + sqrtf(fmaf(df, df, gf * gf)));
            const double t0 = f64_of_f32_scaled(tf, 0);
            const double fp = fma(g0, t0, d0);  // f'(t0) / 2
            const double ft = fma(fma(g0, t0, d0 + d0), t0, -g0);
            const double t = fma(-ft, f64_of_f32_scaled(__frcp_rn(f32_of_scaled(fp, k)), k - 1), t0);
            const double q = fma(t, t, 1.0);
            const double hq = 0.5 * q;
            double c = f64_of_f32_scaled(rsqrtf(f32_of_scaled(q, 0)), 0);
            c *= fma(-hq * c, c, 1.5);
            c *= fma(-hq * c, c, 1.5);
            const double ei = dinv[i], ej = dinv[j];
            nrm2[i] = fmax(al - t * ga, 0.0);
            nrm2[j] = be + t * ga;
            dsc[i] = di * c;
            dsc[j] = dj * c;
            dinv[i] = ei * (q * c);
            dinv[j] = ej * (q * c);
            const int slot = atomicAdd(&nround, 1);
            rlist[slot] = (i << 16) | j;
            rfa[slot] = t * dj * ei;
            rfb[slot] = t * di * ej;
          }
        }
      }
      __syncthreads();
      // phase C: scaled rotations of the pairs that rotate
      const int nr = nround;
      if (nr > 0) {
        for (int e = threadIdx.x; e < nr * rows; e += blockDim.x) {
          const int sl = e % nr, r = e / nr;
          const int ij = rlist[sl];
          double* mi = M + (ij >> 16) * ldm;
          double* mj = M + (ij & 0xffff) * ldm;
          const double u = mi[r], v = mj[r];
          mi[r] = fma(-rfa[sl], v, u);
          mj[r] = fma(rfb[sl], u, v);
        }
        if (threadIdx.x == 0) {
          rotated = 1;
          nrot += nr;
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
    col_norms();
  }
  if (threadIdx.x == 0) {
    if (sweep >= maxsweep) set_err(x, -5);
    if (x.svd_sweeps) {
      x.svd_sweeps[2 * (first + jb)] = sweep + 1;
      x.svd_sweeps[2 * (first + jb) + 1] = nrot;
    }
  }
  // singular values = column norms (exact), sorted descending
  col_norms();
  for (int c = threadIdx.x; c < cols; c += blockDim.x) snorm[c] = nrm2[c] > tiny2 ? sqrt(nrm2[c]) : 0.0;
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
  const int* upiv = reinterpret_cast<const int*>(ptrv(J.piv, x));
  if (U) {
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      int r = e / cols, c = e % cols;
      const double s = snorm[c];
      const int ur = upiv ? upiv[r] : r;
      U[(int64_t)ur * J.ldu + spos[c]] = s > 0.0 ? M[c * ldm + r] / s : 0.0;
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
    }
    if (J.norm_idx >= 0) {
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

// ------------------------------------------------------------------ norm ----
// ||N||_2^2 = lambda_max(G), G = N^T N: Householder tridiagonalisation of G in
// shared memory (symmetric rank-2 updates), then bisection with Sturm counts on
// the tridiagonal matrix for its largest eigenvalue.
// G lives in dynamic shared memory sized for the stage's largest n (nmax x
// (nmax+1) doubles); N is read from global memory (L1-resident).
__global__ void __launch_bounds__(128, 6) k_norm(const ExecCtx* __restrict__ px, const NormJob* __restrict__ jobs,
                                              int nmax, const BatchSeg* __restrict__ segs, int nseg) {
  int jb = blockIdx.x;
  if (segs) {
    const BatchSeg& sg = segs[seg_find(segs, nseg, jb)];
    px = sg.ctx;
    jobs = static_cast<const NormJob*>(sg.jobs);
    jb -= sg.start;
  }
  const ExecCtx& x = *px;
  constexpr int NM = NORM_MAXN;
  extern __shared__ double G[];  // nmax x (nmax+1)
  __shared__ double v[NM], p[NM], w[NM], d[NM], e[NM];
  __shared__ double red[32];
  __shared__ double sh[4];
  const NormJob& J = jobs[jb];
  const int n = dimv(J.n, x.slot);
  if (n <= 0 || n > nmax || n > NM) {
    if (threadIdx.x == 0) {
      if (n > 0) set_err(x, -9);
      x.nrm[J.norm_idx] = 0.0;
      x.scal[J.norm_idx] = 0.0;
    }
    return;
  }
  const double* S = ptrv(J.src, x);
  const int ld = nmax + 1;
  // G = N^T N (symmetric)
  for (int e2 = threadIdx.x; e2 < n * n; e2 += blockDim.x) {
    const int i = e2 / n, j = e2 % n;
    if (j < i) continue;
    double a = 0.0;
    for (int l = 0; l < n; ++l) a = fma(S[(int64_t)l * J.lds + i], S[(int64_t)l * J.lds + j], a);
    G[i * ld + j] = a;
    G[j * ld + i] = a;
  }
  __syncthreads();
  // tridiagonalisation: for column k, reflect rows/cols k+1..n-1.  Four
  // barriers a step: warp 0 forms the reflector (its norm a warp sum) and v;
  // p = tau A v with two threads per row (halves of the row, one shuffle);
  // every warp forms p.v itself (the same value in all) and w; the rank-2
  // update.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k + 2 < n; ++k) {
    if (warp == 0) {
      double s2 = 0.0;
      for (int i = k + 2 + lane; i < n; i += 32) s2 = fma(G[i * ld + k], G[i * ld + k], s2);
      s2 = warp_sum(s2);
      const double alpha = G[(k + 1) * ld + k];
      double tau = 0.0, sc = 0.0, beta = alpha;
      if (s2 > 0.0) householder_scalars(alpha, s2, beta, tau, sc);
      if (lane == 0) {
        sh[k & 1] = tau;  // two slots: a step without reflection has one barrier
        e[k] = beta;
        d[k] = G[k * ld + k];
      }
      if (tau != 0.0)
        for (int i = k + 1 + lane; i < n; i += 32) v[i] = (i == k + 1) ? 1.0 : G[i * ld + k] * sc;
    }
    __syncthreads();
    const double tau = sh[k & 1];
    if (tau == 0.0) continue;
    const int m = n - k - 1, half = (m + 1) >> 1;
    for (int base = 0; base < 2 * m; base += blockDim.x) {
      const int r2 = base + threadIdx.x;
      const int i = k + 1 + (r2 >> 1), h = r2 & 1;
      double a = 0.0;
      if (r2 < 2 * m) {
        const int j0 = k + 1 + h * half, j1 = h ? n : k + 1 + half;
        for (int j = j0; j < j1; ++j) a = fma(G[i * ld + j], v[j], a);
      }
      a += __shfl_xor_sync(0xffffffffu, a, 1);
      if (r2 < 2 * m && h == 0) p[i] = tau * a;
    }
    __syncthreads();
    double pv = 0.0;
    for (int i = k + 1 + lane; i < n; i += 32) pv = fma(p[i], v[i], pv);
    pv = warp_sum(pv);
    const double K = 0.5 * tau * pv;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) w[i] = p[i] - K * v[i];
    __syncthreads();
    for (int e2 = threadIdx.x; e2 < m * m; e2 += blockDim.x) {
      const int i = k + 1 + e2 / m, j = k + 1 + e2 % m;
      G[i * ld + j] -= v[i] * w[j] + w[i] * v[j];
    }
    __syncthreads();
  }
  __syncthreads();  // every warp has read the last step's tau
  if (threadIdx.x == 0) {
    if (n >= 2) {
      d[n - 2] = G[(n - 2) * ld + (n - 2)];
      e[n - 2] = G[(n - 1) * ld + (n - 2)];
    }
    d[n - 1] = G[(n - 1) * ld + (n - 1)];
    // Gershgorin interval of the tridiagonal (d, e)
    double lo = d[0], hi = d[0];
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
      lo = fmin(lo, d[i] - r);
      hi = fmax(hi, d[i] + r);
    }
    for (int i = 0; i + 1 < n; ++i) w[i] = e[i] * e[i];
    double dmax = d[0];
    for (int i = 1; i < n; ++i) dmax = fmax(dmax, d[i]);
    sh[0] = fmax(fmax(lo, dmax), 0.0);  // lambda_max >= every diagonal entry; G is semi-definite
    sh[1] = hi;
    sh[2] = fmax(fabs(lo), fabs(hi));
  }
  __syncthreads();
  // largest eigenvalue by multisection on one warp: each round every lane takes
  // the Sturm count (eigenvalues below its point) at one of 32 equally spaced
  // interior points; the first point with all n below is the new upper end,
  // the point before it the new lower end.  (A warp instruction costs the same
  // however many lanes it uses, so one warp of points beats both single-lane
  // bisection and a block of points.)
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double lo = sh[0], hi = sh[1];
    const double scale = sh[2];
    for (int it = 0; it < 24 && hi - lo > 2.0e-16 * scale; ++it) {
      const double step = (hi - lo) / 33.0;
      const double pt = fma((double)(lane + 1), step, lo);
      int cnt = 0;
      double q = d[0] - pt;
      cnt += q < 0.0;
      for (int i = 1; i < n; ++i) {
        if (q == 0.0) q = 1e-300;
        q = d[i] - pt - w[i - 1] / q;
        cnt += q < 0.0;
      }
      const unsigned all = __ballot_sync(0xffffffffu, cnt == n);
      const int f = all ? __ffs(all) - 1 : 32;  // first point with every eigenvalue below
      const double nlo = f > 0 ? fma((double)f, step, lo) : lo;
      const double nhi = f < 32 ? fma((double)(f + 1), step, lo) : hi;
      lo = nlo;
      hi = nhi;
    }
    if (lane == 0) sh[1] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double s0 = sqrt(fmax(sh[1], 0.0));
    x.nrm[J.norm_idx] = s0;
    x.scal[J.norm_idx] = s0 > 0.0 ? 1.0 / s0 : 0.0;
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
size_t norm_smem_bytes(int nmax) { return sizeof(double) * nmax * (nmax + 1); }
size_t gemm_smem_bytes() { return sizeof(double) * gemm_smem_doubles(GT, GT); }

static bool g_attr_done = false;

cudaError_t kernels_init() {
  if (g_attr_done) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  const int gsm = (int)gemm_smem_bytes();
#define H2_GEMM_ATTR(Q, M) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm<Q, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm);
  H2_GEMM_ATTR(1, GM_F64) H2_GEMM_ATTR(4, GM_F64) H2_GEMM_ATTR(GQ, GM_F64)
  H2_GEMM_ATTR(1, GM_F32) H2_GEMM_ATTR(4, GM_F32) H2_GEMM_ATTR(GQ, GM_F32)
  H2_GEMM_ATTR(1, GM_DF) H2_GEMM_ATTR(4, GM_DF) H2_GEMM_ATTR(GQ, GM_DF)
#undef H2_GEMM_ATTR
#define H2_GEMM_ATTR_CHAIN                                                                          \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_chain<1, GM_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_chain<4, GM_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_chain<GQ, GM_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_chain<1, GM_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_chain<4, GM_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_chain<GQ, GM_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_chain<1, GM_DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_chain<4, GM_DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_chain<GQ, GM_DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, gsm); \
  for (int S_ : {5, 7}) {                                                                            \
    const int tsm = gemm_tc_smem_bytes(S_, GT, GT);                                                  \
    if (S_ == 5) {                                                                                   \
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_tc_chain<5, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm); \
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_tc_chain<5, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm); \
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_tc_chain<5, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm); \
    } else {                                                                                         \
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_tc_chain<7, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm); \
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_tc_chain<7, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm); \
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_tc_chain<7, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm); \
    }                                                                                                \
  }
#define H2_GEMM_TC_ATTR(S, T)                                                                      \
  if (e == cudaSuccess)                                                                            \
    e = cudaFuncSetAttribute(k_gemm_tc<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                             gemm_tc_smem_bytes(S, GT, GT));
  H2_GEMM_TC_ATTR(5, 1) H2_GEMM_TC_ATTR(5, 2) H2_GEMM_TC_ATTR(5, 4)
  H2_GEMM_TC_ATTR(7, 1) H2_GEMM_TC_ATTR(7, 2) H2_GEMM_TC_ATTR(7, 4)
  H2_GEMM_ATTR_CHAIN
#undef H2_GEMM_TC_ATTR
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_norm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)norm_smem_bytes(NORM_MAXN));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, QR_MAX_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_svd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           8 * std::max(SVD_SMEM_DOUBLES, svd_colarr_doubles(SVD_MAXDIM)));
  if (e != cudaSuccess) return e;
  g_attr_done = true;
  return cudaSuccess;
}

void launch_finalize(const ExecCtx* x, int nrank, cudaStream_t s) {
  k_finalize<<<(nrank + 255) / 256 + 1, 256, 0, s>>>(x);
}

// qsteps = ceil(mmax / (256 / nb)): outputs per thread of the stage's largest tile
template <int MODE>
static void launch_gemm_mode(int qsteps, int count, size_t sm, cudaStream_t s, const ExecCtx* x, const GemmOut* go,
                             const GemmTerm* gt, int mmax, int nb, const BatchSeg* segs, int nseg) {
  if (qsteps <= 1)
    k_gemm<1, MODE><<<count, 256, sm, s>>>(x, go, gt, mmax, nb, segs, nseg);
  else if (qsteps <= 4)
    k_gemm<4, MODE><<<count, 256, sm, s>>>(x, go, gt, mmax, nb, segs, nseg);
  else
    k_gemm<GQ, MODE><<<count, 256, sm, s>>>(x, go, gt, mmax, nb, segs, nseg);
}

static void launch_gemm(int mode, int qsteps, int count, size_t sm, cudaStream_t s, const ExecCtx* x,
                        const GemmOut* go, const GemmTerm* gt, int mmax, int nb, const BatchSeg* segs, int nseg) {
  if (mode == GM_DF)
    launch_gemm_mode<GM_DF>(qsteps, count, sm, s, x, go, gt, mmax, nb, segs, nseg);
  else if (mode == GM_F32)
    launch_gemm_mode<GM_F32>(qsteps, count, sm, s, x, go, gt, mmax, nb, segs, nseg);
  else
    launch_gemm_mode<GM_F64>(qsteps, count, sm, s, x, go, gt, mmax, nb, segs, nseg);
}

// tpw = tiles per warp of the stage's largest output tile
template <int S>
static void launch_gemm_tc(int tpw, int count, size_t sm, cudaStream_t s, const ExecCtx* x, const GemmOut* go,
                           const GemmTerm* gt, int mmax, int nb, const BatchSeg* segs, int nseg) {
  if (tpw <= 1)
    k_gemm_tc<S, 1><<<count, 256, sm, s>>>(x, go, gt, mmax, nb, segs, nseg);
  else if (tpw <= 2)
    k_gemm_tc<S, 2><<<count, 256, sm, s>>>(x, go, gt, mmax, nb, segs, nseg);
  else
    k_gemm_tc<S, 4><<<count, 256, sm, s>>>(x, go, gt, mmax, nb, segs, nseg);
}

int stage_launches(const Stage& st) {
  return (st.kind == ST_SVD && st.smem > 8 * SVD_SMALL_DOUBLES) ? 2 : 1;
}

GemmShape gemm_shape(int aux) {
  GemmShape g;
  const int shape = aux & ~GEMM_AUX_FLAGS;
  g.mmax = shape ? ((shape >> 16) & 0xff) : GT;
  g.nb = shape ? (shape & 0xffff) : GT;
  g.slices = (aux & GEMM_AUX_TC7) ? 7 : (aux & GEMM_AUX_TC5) ? 5 : 0;
  g.mode = (aux & GEMM_AUX_DF) ? GM_DF : (aux & GEMM_AUX_FP32) ? GM_F32 : GM_F64;
  if (g.slices) {
    const int tiles = ((g.mmax + 15) / 16) * ((g.nb + 7) / 8);
    g.variant = (tiles + 7) / 8;                 // tiles per warp
    g.variant = g.variant <= 1 ? 1 : g.variant <= 2 ? 2 : 4;
    g.smem = gemm_tc_smem_bytes(g.slices, g.mmax, g.nb);
  } else {
    const int rstep = 256 / g.nb;
    const int qsteps = (g.mmax + rstep - 1) / rstep;  // outputs per thread
    g.variant = qsteps <= 1 ? 1 : qsteps <= 4 ? 4 : GQ;
    g.smem = (int)((g.mode == GM_F32 ? sizeof(float) : sizeof(double)) * gemm_smem_doubles(g.mmax, g.nb));
  }
  return g;
}

// A GEMM stage (x, j: one product; segs: a batched launch of `count` jobs).
static void launch_gemm_stage(const GemmShape& g, int count, const ExecCtx* x, const GemmOut* go,
                              const GemmTerm* gt, const BatchSeg* segs, int nseg, cudaStream_t s) {
  if (g.slices == 7)
    launch_gemm_tc<7>(g.variant, count, g.smem, s, x, go, gt, g.mmax, g.nb, segs, nseg);
  else if (g.slices == 5)
    launch_gemm_tc<5>(g.variant, count, g.smem, s, x, go, gt, g.mmax, g.nb, segs, nseg);
  else
    launch_gemm(g.mode, g.variant, count, g.smem, s, x, go, gt, g.mmax, g.nb, segs, nseg);
}

static void launch_kind(const Stage& st, int count, const ExecCtx* x, const DeviceJobs& j, const BatchSeg* segs,
                        int nseg, cudaStream_t s) {
  switch (st.kind) {
    case ST_GEMM:
      launch_gemm_stage(gemm_shape(st.aux), count, x, segs ? nullptr : j.gemm_out + st.first, j.gemm_term, segs,
                        nseg, s);
      break;
    case ST_COPY:
      k_copy<<<count, 256, 0, s>>>(x, segs ? nullptr : j.copy + st.first, segs, nseg);
      break;
    case ST_QR:
      k_qr<<<count, 256, st.smem, s>>>(x, segs ? nullptr : j.qr + st.first, st.smem / 8, segs, nseg);
      break;
    case ST_QAPPLY:
      k_qapply<<<count, 256, 0, s>>>(x, segs ? nullptr : j.qapply + st.first, segs, nseg);
      break;
    case ST_SVD:
      {
      // st.aux = largest column count of the stage; st.smem covers the
      // per-column arrays of any job and the matrices that fit
      const int cmax = st.aux > 0 ? st.aux : SVD_MAXDIM;
      const size_t sm = st.smem > 0 ? (size_t)st.smem : 8 * (size_t)SVD_SMEM_DOUBLES;
      const SvdJob* jobs = segs ? nullptr : j.svd + st.first;
      if (stage_launches(st) == 2) {
        // jobs that fit SVD_SMALL_DOUBLES in 128-thread CTAs (five per SM),
        // the rest in the stage's full-size CTAs
        k_svd<<<count, 128, 8 * (size_t)SVD_SMALL_DOUBLES, s>>>(x, jobs, st.first, SVD_SMALL_DOUBLES, cmax, -1,
                                                                SVD_SMALL_DOUBLES, segs, nseg);
        k_svd<<<count, 256, sm, s>>>(x, jobs, st.first, (int)(sm / 8), cmax, SVD_SMALL_DOUBLES, INT_MAX, segs, nseg);
      } else {
        k_svd<<<count, 256, sm, s>>>(x, jobs, st.first, (int)(sm / 8), cmax, -1, INT_MAX, segs, nseg);
      }
    }
      break;
    case ST_NORM:
    {
      const int nmax = st.aux > 0 ? st.aux : NORM_MAXN;
      k_norm<<<count, 128, norm_smem_bytes(nmax), s>>>(x, segs ? nullptr : j.norm + st.first, nmax, segs, nseg);
    }
      break;
    case ST_SCAN:
      k_scan<<<(count + 127) / 128, 128, 0, s>>>(x, j.scan + st.first, count);
      break;
  }
}

void launch_stage(const Stage& st, const ExecCtx* x, const DeviceJobs& j, cudaStream_t s) {
  if (st.count <= 0) return;
  launch_kind(st, st.count, x, j, nullptr, 0, s);
}

void launch_stage_batched(const Stage& st, const BatchSeg* segs, int nseg, int total, cudaStream_t s) {
  if (total <= 0 || st.kind == ST_SCAN) return;  // scans are launched per product
  DeviceJobs none{};
  launch_kind(st, total, nullptr, none, segs, nseg, s);
}

void launch_gemm_batched(const GemmShape& g, const BatchSeg* segs, int nseg, int total, cudaStream_t s) {
  if (total > 0) launch_gemm_stage(g, total, nullptr, nullptr, nullptr, segs, nseg, s);
}

int gemm_chain_blocks_per_sm(const GemmShape& g) {
  int nb = 0;
  cudaError_t e = cudaSuccess;
  if (g.slices == 7) {
    if (g.variant <= 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gemm_tc_chain<7, 1>, 256, g.smem);
    else if (g.variant <= 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gemm_tc_chain<7, 2>, 256, g.smem);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gemm_tc_chain<7, 4>, 256, g.smem);
  } else if (g.slices == 5) {
    if (g.variant <= 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gemm_tc_chain<5, 1>, 256, g.smem);
    else if (g.variant <= 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gemm_tc_chain<5, 2>, 256, g.smem);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gemm_tc_chain<5, 4>, 256, g.smem);
  } else {
#define H2_OCC(Q, M) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gemm_chain<Q, M>, 256, g.smem)
    if (g.mode == GM_DF) {
      if (g.variant == 1) H2_OCC(1, GM_DF); else if (g.variant == 4) H2_OCC(4, GM_DF); else H2_OCC(GQ, GM_DF);
    } else if (g.mode == GM_F32) {
      if (g.variant == 1) H2_OCC(1, GM_F32); else if (g.variant == 4) H2_OCC(4, GM_F32); else H2_OCC(GQ, GM_F32);
    } else {
      if (g.variant == 1) H2_OCC(1, GM_F64); else if (g.variant == 4) H2_OCC(4, GM_F64); else H2_OCC(GQ, GM_F64);
    }
#undef H2_OCC
  }
  return e == cudaSuccess ? nb : 0;
}

void launch_gemm_chain(const GemmShape& g, int grid, const BatchSeg* segs, int nseg, int total, int* ctr,
                       cudaStream_t s) {
#define H2_CH(Q, M) k_gemm_chain<Q, M><<<grid, 256, g.smem, s>>>(segs, nseg, total, ctr, g.mmax, g.nb)
#define H2_TCH(S_, T) k_gemm_tc_chain<S_, T><<<grid, 256, g.smem, s>>>(segs, nseg, total, ctr, g.mmax, g.nb)
  if (g.slices == 7) {
    if (g.variant <= 1) H2_TCH(7, 1); else if (g.variant <= 2) H2_TCH(7, 2); else H2_TCH(7, 4);
  } else if (g.slices == 5) {
    if (g.variant <= 1) H2_TCH(5, 1); else if (g.variant <= 2) H2_TCH(5, 2); else H2_TCH(5, 4);
  } else if (g.mode == GM_DF) {
    if (g.variant == 1) H2_CH(1, GM_DF); else if (g.variant == 4) H2_CH(4, GM_DF); else H2_CH(GQ, GM_DF);
  } else if (g.mode == GM_F32) {
    if (g.variant == 1) H2_CH(1, GM_F32); else if (g.variant == 4) H2_CH(4, GM_F32); else H2_CH(GQ, GM_F32);
  } else {
    if (g.variant == 1) H2_CH(1, GM_F64); else if (g.variant == 4) H2_CH(4, GM_F64); else H2_CH(GQ, GM_F64);
  }
#undef H2_CH
#undef H2_TCH
}

}  // namespace h2
