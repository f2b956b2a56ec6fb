// C ABI of the library (include/h2.h): handle management, device upload of
// the inputs, and execution of the planned stage lists on the GPU.
//
// A product plan is built once per operand structure and options and kept in
// a small LRU cache shared by all operand pairs of that structure; its stage
// list is captured into a CUDA graph on first use and replayed afterwards.
// The graph reads every pointer from a per-plan device control block
// (ExecCtx), which is rewritten before each replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <thread>
#include <vector>

#include "../../include/h2.h"
#include "h2_assemble.h"
#include "h2_build.h"
#include "h2_internal.h"
#include "h2_kernels.h"
#include "h2_plan.h"

namespace h2 {

static thread_local std::string g_last_cuda;

static int cuda_fail(cudaError_t e, const char* where) {
  g_last_cuda = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // allocation failures are not sticky: clear and report
    return H2_ENOMEM;
  }
  return H2_ECUDA;
}
#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

static std::mutex g_init_mu;
static bool g_inited = false;
static cudaStream_t g_stream = nullptr;
static uint64_t g_uid = 0;

static int lib_init() {
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (g_inited) return H2_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return H2_ENOTREADY;
  CK(kernels_init());
  CK(cudaStreamCreateWithFlags(&g_stream, cudaStreamNonBlocking));
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  g_inited = true;
  return H2_OK;
}

// --------------------------------------------------- plan device state ----
struct PlanRT {
  std::shared_ptr<Plan> plan;
  std::shared_ptr<PlanRT> blob_owner;  // clones: the instance whose job arrays they use
  void* d_blob = nullptr;      // job arrays + slot init + idx + konst + rank_src (owner only)
  DeviceJobs dj;
  int* d_slot_init = nullptr;
  int* d_idx = nullptr;
  double* d_konst = nullptr;
  int* d_rank_src = nullptr;
  char* d_ctrl = nullptr;      // ExecCtx, scal, nrm, slots, err
  ExecCtx* d_ctx = nullptr;
  double* d_scal = nullptr;
  double* d_nrm = nullptr;
  int* d_slot = nullptr;
  int* d_err = nullptr;
  double* d_ws = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t last = nullptr;  // completion of the last replay (workspace reuse)
  int nrank = 0;
  // pinned ring of control headers (asynchronous upload without a host wait)
  static constexpr int RING = 64;
  static constexpr int HDR = 1024;
  char* h_ring = nullptr;
  cudaEvent_t ring_ev[RING] = {};
  int ring_next = 0;
  ~PlanRT() {
    if (last) cudaEventSynchronize(last);  // the last replay may still use the workspace
    if (graph) cudaGraphExecDestroy(graph);
    if (last) cudaEventDestroy(last);
    for (auto& e : ring_ev)
      if (e) cudaEventDestroy(e);
    if (h_ring) cudaFreeHost(h_ring);
    cudaFree(d_blob);
    cudaFree(d_ctrl);
    cudaFree(d_ws);
  }
};

template <class T>
static size_t put(std::vector<char>& blob, const std::vector<T>& v) {
  size_t off = (blob.size() + 255) & ~size_t(255);
  blob.resize(off + v.size() * sizeof(T));
  if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}

static int upload_plan(PlanRT& rt, const std::vector<int>& rank_src) {
  Plan& P = *rt.plan;
  std::vector<char> blob;
  const size_t o_go = put(blob, P.gout), o_gt = put(blob, P.gterm), o_cp = put(blob, P.copy), o_qr = put(blob, P.qr),
               o_qa = put(blob, P.qap), o_sv = put(blob, P.svd), o_sc = put(blob, P.scan), o_nm = put(blob, P.norm),
               o_si = put(blob, P.slot_init), o_ix = put(blob, P.idx), o_k = put(blob, P.konst),
               o_rs = put(blob, rank_src);
  CK(cudaMalloc(&rt.d_blob, std::max<size_t>(blob.size(), 256)));
  CK(cudaMemcpy(rt.d_blob, blob.data(), blob.size(), cudaMemcpyHostToDevice));
  char* b = (char*)rt.d_blob;
  rt.dj.gemm_out = (const GemmOut*)(b + o_go);
  rt.dj.gemm_term = (const GemmTerm*)(b + o_gt);
  rt.dj.copy = (const CopyJob*)(b + o_cp);
  rt.dj.qr = (const QrJob*)(b + o_qr);
  rt.dj.qapply = (const QApplyJob*)(b + o_qa);
  rt.dj.svd = (const SvdJob*)(b + o_sv);
  rt.dj.scan = (const ScanJob*)(b + o_sc);
  rt.dj.norm = (const NormJob*)(b + o_nm);
  rt.d_slot_init = (int*)(b + o_si);
  rt.d_idx = (int*)(b + o_ix);
  rt.d_konst = (double*)(b + o_k);
  rt.d_rank_src = (int*)(b + o_rs);
  rt.nrank = (int)rank_src.size();
  const size_t nslot = std::max<size_t>(P.slot_init.size(), 1);
  const size_t sz = 512 + 16 * (size_t)P.nscal + 4 * nslot + 64;
  CK(cudaMalloc(&rt.d_ctrl, sz));
  rt.d_ctx = (ExecCtx*)rt.d_ctrl;
  rt.d_scal = (double*)(rt.d_ctrl + 512);
  rt.d_nrm = rt.d_scal + P.nscal;
  rt.d_slot = (int*)(rt.d_nrm + P.nscal);
  rt.d_err = rt.d_slot + nslot;
  CK(cudaMalloc(&rt.d_ws, std::max<int64_t>(P.ws_len + P.fac_len, 1) * sizeof(double)));
  CK(cudaEventCreateWithFlags(&rt.last, cudaEventDisableTiming));
  return H2_OK;
}

// Writes the control block (ExecCtx + parameters) through a pinned ring slot.
static int enqueue_header(PlanRT& rt, const ExecCtx& ctx, const double* params, cudaStream_t s) {
  if (!rt.h_ring) {
    CK(cudaMallocHost(&rt.h_ring, (size_t)PlanRT::RING * PlanRT::HDR));
    for (auto& e : rt.ring_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  const int slot = rt.ring_next;
  rt.ring_next = (rt.ring_next + 1) % PlanRT::RING;
  CK(cudaEventSynchronize(rt.ring_ev[slot]));  // previous use of this slot has been copied
  char* h = rt.h_ring + (size_t)slot * PlanRT::HDR;
  std::memset(h, 0, 512 + sizeof(double) * PARAM_COUNT);
  std::memcpy(h, &ctx, sizeof(ctx));
  for (int i = 0; i < PARAM_COUNT; ++i) std::memcpy(h + 512 + 8 * i, &params[i], 8);
  CK(cudaStreamWaitEvent(s, rt.last, 0));
  CK(cudaMemcpyAsync(rt.d_ctrl, h, 512 + sizeof(double) * PARAM_COUNT, cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(rt.ring_ev[slot], s));
  return H2_OK;
}

// Enqueue one execution of the plan on stream s (graph replay when captured).
static int run_plan(PlanRT& rt, double* bx, double* by, double* bc, int* out_int, const double* params,
                    cudaStream_t s, bool use_graph) {
  Plan& P = *rt.plan;
  ExecCtx ctx{};
  ctx.base[AR_WS] = rt.d_ws;
  ctx.base[AR_X] = bx;
  ctx.base[AR_Y] = by;
  ctx.base[AR_C] = bc;
  ctx.base[AR_K] = rt.d_konst;
  ctx.base[AR_F] = rt.d_ws + P.ws_len;
  ctx.slot = rt.d_slot;
  ctx.scal = rt.d_scal;
  ctx.nrm = rt.d_nrm;
  ctx.err = rt.d_err;
  ctx.idx = rt.d_idx;
  ctx.out_int = out_int;
  ctx.rank_src = rt.d_rank_src;
  ctx.nrank = out_int ? rt.nrank : 0;
  // header: ExecCtx then the parameters at scal[0..PARAM_COUNT)
  {
    int rc = enqueue_header(rt, ctx, params, s);
    if (rc) return rc;
  }
  if (use_graph && !rt.graph) {
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    if (!P.slot_init.empty())
      cudaMemcpyAsync(rt.d_slot, rt.d_slot_init, sizeof(int) * P.slot_init.size(), cudaMemcpyDeviceToDevice, cs);
    cudaMemsetAsync(rt.d_err, 0, sizeof(int), cs);
    for (const Stage& st : P.stages) launch_stage(st, rt.d_ctx, rt.dj, cs);
    launch_finalize(rt.d_ctx, rt.nrank, cs);
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "capture");
    e = cudaGraphInstantiate(&rt.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate");
  }
  if (use_graph) {
    CK(cudaGraphLaunch(rt.graph, s));
  } else {
    if (!P.slot_init.empty())
      CK(cudaMemcpyAsync(rt.d_slot, rt.d_slot_init, sizeof(int) * P.slot_init.size(), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(rt.d_err, 0, sizeof(int), s));
    for (const Stage& st : P.stages) launch_stage(st, rt.d_ctx, rt.dj, s);
    launch_finalize(rt.d_ctx, rt.nrank, s);
  }
  CK(cudaGetLastError());
  CK(cudaEventRecord(rt.last, s));
  return H2_OK;
}

// Stage-by-stage execution with CUDA events; per kernel kind: launches, jobs,
// device time and the algorithmic work with the ranks the device decided.
static int run_plan_profiled(PlanRT& rt, double* bx, double* by, double* bc, int* out_int, const double* params,
                             cudaStream_t s, h2_kernel_prof* prof) {
  Plan& P = *rt.plan;
  int* d_sweeps = nullptr;
  CK(cudaMalloc(&d_sweeps, 2 * sizeof(int) * std::max<size_t>(P.svd.size(), 1)));
  CK(cudaMemset(d_sweeps, 0, 2 * sizeof(int) * std::max<size_t>(P.svd.size(), 1)));
  ExecCtx ctx{};
  ctx.base[AR_WS] = rt.d_ws;
  ctx.base[AR_X] = bx;
  ctx.base[AR_Y] = by;
  ctx.base[AR_C] = bc;
  ctx.base[AR_K] = rt.d_konst;
  ctx.base[AR_F] = rt.d_ws + P.ws_len;
  ctx.slot = rt.d_slot;
  ctx.scal = rt.d_scal;
  ctx.nrm = rt.d_nrm;
  ctx.err = rt.d_err;
  ctx.idx = rt.d_idx;
  ctx.out_int = out_int;
  ctx.rank_src = rt.d_rank_src;
  ctx.nrank = out_int ? rt.nrank : 0;
  ctx.svd_sweeps = d_sweeps;
  {
    int rc = enqueue_header(rt, ctx, params, s);
    if (rc) return rc;
  }
  if (!P.slot_init.empty())
    CK(cudaMemcpyAsync(rt.d_slot, rt.d_slot_init, sizeof(int) * P.slot_init.size(), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(rt.d_err, 0, sizeof(int), s));
  const size_t ns = P.stages.size();
  std::vector<cudaEvent_t> ev(2 * ns + 2);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  for (size_t i = 0; i < ns; ++i) {
    CK(cudaEventRecord(ev[2 * i], s));
    launch_stage(P.stages[i], rt.d_ctx, rt.dj, s);
    CK(cudaEventRecord(ev[2 * i + 1], s));
  }
  CK(cudaEventRecord(ev[2 * ns], s));
  launch_finalize(rt.d_ctx, rt.nrank, s);
  CK(cudaEventRecord(ev[2 * ns + 1], s));
  CK(cudaGetLastError());
  CK(cudaEventRecord(rt.last, s));
  CK(cudaStreamSynchronize(s));
  std::vector<int> slot(P.slot_init.size()), sweeps(2 * P.svd.size());
  if (!slot.empty()) CK(cudaMemcpy(slot.data(), rt.d_slot, slot.size() * 4, cudaMemcpyDeviceToHost));
  if (!sweeps.empty()) CK(cudaMemcpy(sweeps.data(), d_sweeps, sweeps.size() * 4, cudaMemcpyDeviceToHost));
  cudaFree(d_sweeps);
  auto dv = [&](const Dim& d) {
    int v = d.c;
    if (d.s1 >= 0) v += slot[d.s1];
    if (d.s2 >= 0) v += slot[d.s2];
    if (d.mc >= 0) v = std::min(v, d.mc + (d.ms >= 0 ? slot[d.ms] : 0));
    return (double)v;
  };
  for (int k = 0; k < H2_PROFILE_KINDS; ++k) prof[k] = h2_kernel_prof{0, 0, 0.0, 0.0, 0.0};
  // H2_PROFILE_STAGES=1 prints one line per stage to stderr (diagnostics)
  const bool verbose = std::getenv("H2_PROFILE_STAGES") != nullptr;
  for (size_t i = 0; i <= ns; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
    const int kind = i < ns ? (P.stages[i].kind == ST_NORM ? 7 : P.stages[i].kind) : 6;
    h2_kernel_prof& pr = prof[kind];
    pr.launches += i < ns ? stage_launches(P.stages[i]) : 1;
    pr.ms += ms;
    if (i == ns) continue;
    const Stage& st = P.stages[i];
    pr.jobs += st.count;
    double st_fl = 0.0, st_tfl = 0.0, st_by = 0.0;
    // tensor-core GEMM stages: multiply-adds issued to the tensor cores, as
    // mma.sync m16n8k16 slice products (S(S+1)/2 per 16 x 8 tile and k step of
    // 16; k chunks of 32, the last one rounded up to 16)
    const int tc_slices = st.kind == ST_GEMM ? gemm_shape(st.aux).slices : 0;
    auto tc_flops = [&](double mm, double nn, double kk) {
      if (mm <= 0 || nn <= 0 || kk <= 0) return 0.0;
      const double full = std::floor(kk / 32.0), rem = kk - 32.0 * full;
      const double ksteps = 2.0 * full + std::ceil(rem / 16.0);
      return std::ceil(mm / 16.0) * std::ceil(nn / 8.0) * ksteps * (tc_slices * (tc_slices + 1) / 2) * 4096.0;
    };
    double sw_sum = 0.0, sw_max = 0.0, rows_sum = 0.0, cols_sum = 0.0, rows_max = 0.0, cols_max = 0.0;
    double glob_jobs = 0.0, glob_fl = 0.0;  // SVD jobs whose matrix stays in global memory
    for (int j = 0; j < st.count; ++j) {
      double fl = 0, by = 0;
      const int64_t J = st.first + j;
      switch (st.kind) {
        case ST_GEMM: {
          const GemmOut& O = P.gout[J];
          const double m = dv(O.m), n = O.clampn ? std::min(dv(O.n), 64.0) : dv(O.n);
          if (m <= 0 || n <= 0) break;
          by += 8 * m * n * (O.beta ? 2 : 1);
          for (int t = O.t0; t < O.t1; ++t) {
            const GemmTerm& T = P.gterm[t];
            if (T.b.arena < 0) {
              fl += m * n;
              by += 8 * m * n;
            } else if (T.c.arena < 0) {
              const double k1 = dv(T.k1);
              fl += 2 * m * n * k1;
              by += 8 * (m * k1 + k1 * n);
              if (tc_slices) st_tfl += tc_flops(m, n, k1);
            } else {
              const double k1 = dv(T.k1), k2 = dv(T.k2);
              fl += 2 * m * k1 * k2 + 2 * m * k2 * n;
              by += 8 * (m * k1 + k1 * k2 + k2 * n);
              if (tc_slices) st_tfl += tc_flops(m, k2, k1) + tc_flops(m, n, k2);
            }
          }
          break;
        }
        case ST_COPY: {
          const CopyJob& C = P.copy[J];
          const double r = dv(C.rows), c = dv(C.cols);
          by += 8 * (r * c + std::max(r, dv(C.zrows)) * std::max(c, dv(C.zcols)));
          break;
        }
        case ST_QR: {
          const QrJob& Q = P.qr[J];
          const double r = dv(Q.rows), c = dv(Q.cols);
          if (Q.rank_slot >= 0) {
            // j = 0..k-1 Householder steps on (r - j) x (c - j) trailing parts
            const double k = slot[Q.rank_slot];
            fl += 4 * k * r * c - 2 * k * k * (r + c) + 4 * k * k * k / 3;
          } else {
            fl += r >= c ? 2 * r * c * c - 2 * c * c * c / 3 : 2 * c * r * r - 2 * r * r * r / 3;
          }
          by += 16 * r * c;
          break;
        }
        case ST_QAPPLY: {
          const QApplyJob& Q = P.qap[J];
          const double r = dv(Q.rows), q = std::min(dv(Q.q), dv(Q.rows)), nc = dv(Q.ncols);
          fl += std::max(0.0, 4 * r * q * nc - 2 * q * q * nc);
          by += 8 * (r * q + 2 * r * nc);
          break;
        }
        case ST_NORM: {
          // N^T N (symmetric half), tridiagonalisation (4/3 n^3)
          const double n = dv(P.norm[J].n);
          fl += n * n * (n + 1) + 4.0 * n * n * n / 3.0;
          by += 8 * n * n;
          break;
        }
        case ST_SVD: {
          const SvdJob& S = P.svd[J];
          const double r = dv(S.rows), c = dv(S.cols);
          // per sweep: one dot product per pair and the column norms; 6 flops per
          // row for each applied rotation
          fl += (r * c * (c - 1) + 2 * r * c) * sweeps[2 * J] + 6 * r * sweeps[2 * J + 1] + 2 * r * c;
          by += 16 * r * c;
          sw_sum += sweeps[2 * J];
          sw_max = std::max(sw_max, (double)sweeps[2 * J]);
          rows_sum += r;
          cols_sum += c;
          rows_max = std::max(rows_max, r);
          cols_max = std::max(cols_max, c);
          if (svd_colarr_doubles((int)c) + (r + 1) * c > st.smem / 8) {
            glob_jobs += 1;
            glob_fl += fl;
          }
          break;
        }
        default:
          break;
      }
      pr.flops += fl;
      pr.bytes += by;
      st_fl += fl;
      st_by += by;
    }
    if (tc_slices) {
      h2_kernel_prof& tc = prof[8];
      tc.launches += stage_launches(st);
      tc.jobs += st.count;
      tc.ms += ms;
      tc.flops += st_tfl;
      tc.bytes += st_by;
    }
    if (verbose) {
      std::fprintf(stderr, "stage %4zu kind %d tag %2d jobs %7d smem %6d ms %9.4f gflop %9.4f tflops %6.3f", i,
                   st.kind, st.tag, st.count, st.smem, ms, st_fl / 1e9, ms > 0 ? st_fl / ms / 1e9 : 0.0);
      if (st.kind == ST_SVD && st.count > 0)
        std::fprintf(stderr, " rows %.1f cols %.1f sweeps %.2f max %.0f | max rows %.0f cols %.0f | in global %.0f jobs %.3f gflop",
                     rows_sum / st.count, cols_sum / st.count, sw_sum / st.count, sw_max, rows_max, cols_max, glob_jobs,
                     glob_fl / 1e9);
      std::fprintf(stderr, "\n");
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return H2_OK;
}

static int map_err(int dev_err) {
  switch (dev_err) {
    case 0: return H2_OK;
    case -4: return H2_ETIMEOUT;
    case -5: return H2_ENOCONV;
    case -7: return H2_ERANK;
    default: return H2_EINVAL;
  }
}

static MatDesc desc_of(const h2_matrix* A) {
  MatDesc d;
  d.rows = A->rows.get();
  d.cols = A->cols.get();
  d.blocks = A->blocks.get();
  d.k = A->kpad;
  d.off_V = A->off_V;
  d.off_E = A->off_E;
  d.off_W = A->off_W;
  d.off_F = A->off_F;
  d.off_S = A->off_S;
  d.off_N = A->off_N;
  d.off_VF = A->off_VF;
  d.off_WF = A->off_WF;
  return d;
}

// Explicit level bases of a matrix (needed when it is a factor or expanded).
// Structure signature of a matrix: everything a product plan depends on
// (trees, block tree, padded rank, arena layout, admissibility); the numeric
// contents are reached through the arena base pointers at replay time.
static uint64_t matrix_sig(const h2_matrix* M) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  uint64_t eta_bits;
  std::memcpy(&eta_bits, &M->eta, sizeof eta_bits);
  mix(M->rows->hash);
  mix(M->cols->hash);
  mix(M->blocks->sig);
  mix((uint64_t)M->kpad);
  mix((uint64_t)M->dim);
  mix(eta_bits);
  mix((uint64_t)M->same_basis);
  for (int64_t v : {M->off_V, M->off_E, M->off_W, M->off_F, M->off_S, M->off_N, M->off_VF, M->off_WF, M->arena_len})
    mix((uint64_t)v);
  return h;
}

// Product plans, shared by every operand pair of the same structure; least
// recently used first out.  An entry holds the host plan and one or more
// device instances: instance 0 owns the job arrays, further instances (for
// products of the same structure running at once, see h2_server) share them
// and have their own workspace, control block, graph and completion event.
struct PlanKey {
  uint64_t a, b;
  int opt;
  bool operator==(const PlanKey& o) const { return a == o.a && b == o.b && opt == o.opt; }
};
struct PlanEntry {
  std::shared_ptr<Plan> plan;
  std::mutex mu;  // guards inst
  std::vector<std::shared_ptr<PlanRT>> inst;
  std::vector<int> rank_src;
};
constexpr size_t PLAN_CACHE_MAX = 4;
std::mutex g_plans_mu;
std::list<std::pair<PlanKey, std::shared_ptr<PlanEntry>>> g_plans;  // most recent first

static std::shared_ptr<PlanEntry> plan_lookup(const PlanKey& k) {
  std::lock_guard<std::mutex> lk(g_plans_mu);
  for (auto it = g_plans.begin(); it != g_plans.end(); ++it)
    if (it->first == k) {
      g_plans.splice(g_plans.begin(), g_plans, it);
      return g_plans.front().second;
    }
  return nullptr;
}

static void plan_insert(const PlanKey& k, std::shared_ptr<PlanEntry> e) {
  std::shared_ptr<PlanEntry> evicted;
  {
    std::lock_guard<std::mutex> lk(g_plans_mu);
    g_plans.emplace_front(k, std::move(e));
    if (g_plans.size() > PLAN_CACHE_MAX) {
      evicted = std::move(g_plans.back().second);  // released outside the lock
      g_plans.pop_back();
    }
  }
}

static void plan_cache_clear() {
  std::list<std::pair<PlanKey, std::shared_ptr<PlanEntry>>> old;
  {
    std::lock_guard<std::mutex> lk(g_plans_mu);
    old.swap(g_plans);
  }
}

// Device bytes of one instance of a plan beyond the shared job arrays.
static int64_t instance_bytes(const Plan& P) {
  return (P.ws_len + P.fac_len) * 8 + 512 + 16 * (int64_t)P.nscal + 4 * (int64_t)P.slot_init.size() + 64;
}

// A further instance sharing the job arrays of `base`.
static int clone_instance(const std::shared_ptr<PlanRT>& base, std::shared_ptr<PlanRT>& out) {
  auto rt = std::make_shared<PlanRT>();
  rt->plan = base->plan;
  rt->blob_owner = base;
  rt->dj = base->dj;
  rt->d_slot_init = base->d_slot_init;
  rt->d_idx = base->d_idx;
  rt->d_konst = base->d_konst;
  rt->d_rank_src = base->d_rank_src;
  rt->nrank = base->nrank;
  const Plan& P = *rt->plan;
  const size_t nslot = std::max<size_t>(P.slot_init.size(), 1);
  const size_t sz = 512 + 16 * (size_t)P.nscal + 4 * nslot + 64;
  CK(cudaMalloc(&rt->d_ctrl, sz));
  rt->d_ctx = (ExecCtx*)rt->d_ctrl;
  rt->d_scal = (double*)(rt->d_ctrl + 512);
  rt->d_nrm = rt->d_scal + P.nscal;
  rt->d_slot = (int*)(rt->d_nrm + P.nscal);
  rt->d_err = rt->d_slot + nslot;
  CK(cudaMalloc(&rt->d_ws, std::max<int64_t>(P.ws_len + P.fac_len, 1) * sizeof(double)));
  CK(cudaEventCreateWithFlags(&rt->last, cudaEventDisableTiming));
  out = rt;
  return H2_OK;
}

// Batched matrix-vector products: plans per (matrix structure, nrhs), and the
// permutations between the caller's ordering (column-major n x nrhs) and the
// cluster ordering of the plan (row-major n x nrhs).
constexpr int MV_MAXRHS = 4096;
struct MvKey {
  uint64_t sig;
  int nrhs;
  bool operator==(const MvKey& o) const { return sig == o.sig && nrhs == o.nrhs; }
};
constexpr size_t MV_CACHE_MAX = 4;
std::mutex g_mv_mu;
std::list<std::pair<MvKey, std::shared_ptr<PlanRT>>> g_mv;  // most recent first

static std::shared_ptr<PlanRT> mv_lookup(const MvKey& k) {
  std::lock_guard<std::mutex> lk(g_mv_mu);
  for (auto it = g_mv.begin(); it != g_mv.end(); ++it)
    if (it->first == k) {
      g_mv.splice(g_mv.begin(), g_mv, it);
      return g_mv.front().second;
    }
  return nullptr;
}

static void mv_insert(const MvKey& k, std::shared_ptr<PlanRT> rt) {
  std::shared_ptr<PlanRT> evicted;
  std::lock_guard<std::mutex> lk(g_mv_mu);
  g_mv.emplace_front(k, std::move(rt));
  if (g_mv.size() > MV_CACHE_MAX) {
    evicted = std::move(g_mv.back().second);
    g_mv.pop_back();
  }
}

// Xc[r * nrhs + j] = X[j * n + perm[r]]
__global__ void k_perm_gather(const double* __restrict__ X, const int* __restrict__ perm, int64_t n, int nrhs,
                              double* __restrict__ Xc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / nrhs;
    const int j = (int)(e % nrhs);
    Xc[e] = X[(int64_t)j * n + perm[r]];
  }
}

// Y[j * n + perm[r]] = Yc[r * nrhs + j]
__global__ void k_perm_scatter(const double* __restrict__ Yc, const int* __restrict__ perm, int64_t n, int nrhs,
                               double* __restrict__ Y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / nrhs;
    const int j = (int)(e % nrhs);
    Y[(int64_t)j * n + perm[r]] = Yc[e];
  }
}

static int ensure_level_bases(h2_matrix* A, cudaStream_t s) {
  if (A->levels_ready) return H2_OK;
  const double params[PARAM_COUNT] = {0.0, 0.0};
  {
    PlanRT rt;
    rt.plan = make_levelbasis_plan(*A->rows, A->kpad, AR_X, A->off_V, A->off_E, A->off_VF);
    int rc = upload_plan(rt, {});
    if (rc) return rc;
    rc = run_plan(rt, A->d_arena, nullptr, nullptr, nullptr, params, s, false);
    if (rc) return rc;
    if (!A->same_basis) {
      PlanRT rt2;
      rt2.plan = make_levelbasis_plan(*A->cols, A->kpad, AR_X, A->off_W, A->off_F, A->off_WF);
      rc = upload_plan(rt2, {});
      if (rc) return rc;
      rc = run_plan(rt2, A->d_arena, nullptr, nullptr, nullptr, params, s, false);
      if (rc) return rc;
      CK(cudaStreamSynchronize(s));
    }
    CK(cudaStreamSynchronize(s));
  }
  A->levels_ready = true;
  return H2_OK;
}

}  // namespace h2

using namespace h2;

// The opaque H-matrix product handle.
struct h2_hmatrix {
  std::shared_ptr<h2::Tree> rows, cols;
  std::shared_ptr<h2::BlockTree> blocks;
  double* d_arena = nullptr;
  int64_t arena_len = 0, off_N = 0;
  std::vector<int64_t> off_L, off_R;
  std::vector<int> w;
  int* d_int = nullptr;  // [rank of each admissible leaf][err]
  cudaEvent_t done = nullptr;
};

extern "C" {

const char* h2_strerror(int code) {
  switch (code) {
    case H2_OK: return "ok";
    case H2_EINVAL: return "invalid argument";
    case H2_ETREE: return "column cluster tree of A differs from the row cluster tree of B";
    case H2_ENOMEM: return "out of memory";
    case H2_ETIMEOUT: return "device wait timed out";
    case H2_ENOCONV: return "Jacobi SVD did not converge";
    case H2_ECUDA: return "CUDA error";
    case H2_ERANK: return "adaptive rank above max_rank";
    case H2_ENOTREADY: return "no CUDA device";
    default: return "unknown error";
  }
}

const char* h2_last_cuda_error(void) { return g_last_cuda.c_str(); }

int h2_build(const double* points, int64_t n, const h2_build_opts* o, h2_matrix** out) {
  if (!out) return H2_EINVAL;
  *out = nullptr;
  if (!points || !o || n <= 0 || n > (int64_t)1 << 30 || o->dim < 1 || o->dim > 3 || o->leaf_size < 2 ||
      o->order < 1 || o->order > 8 || !(o->eta > 0) || o->kernel < 0 || o->kernel > 3)
    return H2_EINVAL;
  for (int64_t i = 0; i < n * o->dim; ++i)
    if (!std::isfinite(points[i])) return H2_EINVAL;
  int k = 1;
  for (int a = 0; a < o->dim; ++a) k *= o->order;
  if (k > GEMM_MAXTILE || o->leaf_size > SVD_MAXDIM) return H2_EINVAL;
  int rc = lib_init();
  if (rc) return rc;
  auto A = new h2_matrix();
  try {
    A->dim = o->dim;
    A->eta = o->eta;
    A->kpad = k;
    A->rows = std::make_shared<Tree>();
    build_cluster_tree(points, n, o->dim, o->leaf_size, *A->rows);
    A->cols = A->rows;
    A->blocks = std::make_shared<BlockTree>();
    build_block_tree(*A->rows, *A->cols, o->eta, *A->blocks);
    const Tree& T = *A->rows;
    const BlockTree& BT = *A->blocks;
    A->same_basis = true;
    A->off_V = 0;
    A->off_E = A->off_V + (int64_t)T.n * k;
    A->off_S = A->off_E + (int64_t)T.ncl * k * k;
    A->off_N = A->off_S + (int64_t)BT.adm_list.size() * k * k;
    A->off_VF = A->off_N + BT.near_total;
    A->off_W = A->off_V;
    A->off_F = A->off_E;
    A->off_WF = A->off_VF;
    A->arena_len = A->off_VF + (int64_t)(T.depth + 1) * T.n * k;
    if (cudaMalloc(&A->d_arena, A->arena_len * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      delete A;
      return H2_ENOMEM;
    }
    // E_0 (the root has no parent) stays zero
    cudaMemsetAsync(A->d_arena + A->off_E, 0, (size_t)k * k * sizeof(double), g_stream);
    std::string err;
    rc = assemble_device(points, T, BT, o->order, o->kernel, o->kparam, A->d_arena + A->off_V,
                         A->d_arena + A->off_E, A->d_arena + A->off_S, A->d_arena + A->off_N, g_stream, err);
    if (rc) {
      g_last_cuda = err;
      h2_free(A);
      return rc;
    }
    std::vector<int> ints(2 * T.ncl + 1, k);
    ints[2 * T.ncl] = 0;
    cudaMalloc(&A->d_int, ints.size() * sizeof(int));
    cudaMemcpy(A->d_int, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice);
    A->uid = ++g_uid;
    rc = ensure_level_bases(A, g_stream);
    if (rc) {
      h2_free(A);
      return rc;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      h2_free(A);
      return cuda_fail(e, "h2_build");
    }
  } catch (...) {
    delete A;
    return H2_EINVAL;
  }
  *out = A;
  return H2_OK;
}

void h2_free(h2_matrix* A) {
  if (!A) return;
  if (A->done) {
    cudaEventSynchronize(A->done);
    cudaEventDestroy(A->done);
  }
  if (A->d_arena) cudaFree(A->d_arena);
  if (A->d_int) cudaFree(A->d_int);
  if (A->d_perm) cudaFree(A->d_perm);
  delete A;
}

static int hmul_impl(const h2_matrix* Ac, const h2_matrix* Bc, double eps, const h2_mul_opts* opts,
                     h2_hmatrix** Cout);

// Squared relative noise floor of the Jacobi SVDs of a product (PARAM_SVD_FLOOR).
// Columns below floor * ||M||_F are rounding noise of the contractions that
// formed M; resolving them to relative precision costs sweeps and changes no
// kept singular value.  FP64: eps * 2^-20 clamped to [2^-50, 2^-40], i.e. at
// least 2^20 below the tightest relative truncation tolerance of the product
// (eps/3/(2n^2) with n <= 8 in the agglomeration, and the basis tolerances);
// eps = 0 keeps every direction above 2^-50.  Compensated contractions
// (precision 2) and the 7-slice tensor-core form (precision 4), whose
// rounding is about 1e-13 or below: 2^-40.  The 5-slice form (precision 3,
// 40-bit slicing): 2^-30.
static double svd_noise_floor(double eps, int precision) {
  double f;
  if (precision == 2 || precision == 4) f = 9.094947017729282e-13;  // 2^-40
  else if (precision == 3) f = 9.313225746154785e-10;                // 2^-30
  else if (eps > 0.0) f = std::min(9.094947017729282e-13, std::max(8.881784197001252e-16, eps * 9.5367431640625e-07));
  else f = 8.881784197001252e-16;  // 2^-50
  return f * f;
}

// Validated arguments of a product.
struct MulArgs {
  h2_matrix* A = nullptr;
  h2_matrix* B = nullptr;
  double eps = 0, theta = 0.25;
  int max_rank = 0, precision = 0, svd_sweeps = 0;
  bool sync = true;
  cudaStream_t stream = nullptr;
  PlanKey key{};
};

static int mul_args(const h2_matrix* Ac, const h2_matrix* Bc, double eps, const h2_mul_opts* opts, MulArgs& m) {
  if (!Ac || !Bc || !(eps >= 0.0) || !std::isfinite(eps)) return H2_EINVAL;
  m.A = const_cast<h2_matrix*>(Ac);
  m.B = const_cast<h2_matrix*>(Bc);
  if (m.A->cols->hash != m.B->rows->hash || m.A->cols->n != m.B->rows->n) return H2_ETREE;
  if (m.A->kpad != m.B->kpad) return H2_EINVAL;
  m.eps = eps;
  m.theta = (opts && opts->theta > 0.0) ? opts->theta : 0.25;
  if (!(m.theta < 0.5)) return H2_EINVAL;
  m.max_rank = opts ? opts->max_rank : 0;
  m.precision = opts ? opts->precision : 0;
  if (m.precision < 0 || m.precision > 4) return H2_EINVAL;
  if (m.max_rank < 0 || m.max_rank > GEMM_MAXTILE) return H2_EINVAL;
  m.sync = opts ? opts->sync != 0 : true;
  m.svd_sweeps = opts ? opts->svd_max_sweeps : 0;
  if (m.svd_sweeps < 0) return H2_EINVAL;
  m.stream = (opts && opts->stream) ? (cudaStream_t)opts->stream : g_stream;
  m.key = PlanKey{matrix_sig(m.A), matrix_sig(m.B),
                  (m.precision * 100 + m.max_rank) * 1000 + (int)std::lround(m.theta * 997.0)};
  return H2_OK;
}

// The cached plan entry of a product (planned and uploaded on a miss).
static int mul_entry(const MulArgs& m, std::shared_ptr<PlanEntry>& e) {
  e = plan_lookup(m.key);
  if (e) return H2_OK;
  MulOptions mo;
  mo.eta = m.A->eta;
  mo.theta = m.theta;
  mo.max_rank = m.max_rank;
  mo.precision = m.precision;
  auto ne = std::make_shared<PlanEntry>();
  try {
    ne->plan = make_product_plan(desc_of(m.A), desc_of(m.B), mo);
  } catch (const std::exception& ex) {
    g_last_cuda = ex.what();
    return H2_EINVAL;
  }
  ne->rank_src = ne->plan->rank_row_slot;
  ne->rank_src.insert(ne->rank_src.end(), ne->plan->rank_col_slot.begin(), ne->plan->rank_col_slot.end());
  auto rt = std::make_shared<PlanRT>();
  rt->plan = ne->plan;
  int rc = upload_plan(*rt, ne->rank_src);
  if (rc == H2_ENOMEM) {
    // the cached plans hold device memory: release them and retry once
    plan_cache_clear();
    rt = std::make_shared<PlanRT>();
    rt->plan = ne->plan;
    rc = upload_plan(*rt, ne->rank_src);
  }
  if (rc) return rc;
  ne->inst.push_back(rt);
  plan_insert(m.key, ne);
  e = ne;
  return H2_OK;
}

// A new product matrix C for plan P (storage allocated on stream s, its
// coefficient area cleared).
static int new_product_matrix(const MulArgs& m, const Plan& P, cudaStream_t s, h2_matrix** Cout) {
  h2_matrix* A = m.A;
  h2_matrix* B = m.B;
  auto C = new h2_matrix();
  C->dim = A->dim;
  C->eta = A->eta;
  C->kpad = P.kpad;
  C->rows = A->rows;
  C->cols = B->cols;
  C->blocks = P.cblocks;
  C->same_basis = false;
  C->off_V = P.c_off_V;
  C->off_E = P.c_off_E;
  C->off_W = P.c_off_W;
  C->off_F = P.c_off_F;
  C->off_S = P.c_off_S;
  C->off_N = P.c_off_N;
  C->off_VF = P.c_len;
  C->off_WF = C->off_VF + (int64_t)(C->rows->depth + 1) * C->rows->n * P.kpad;
  C->arena_len = C->off_WF + (int64_t)(C->cols->depth + 1) * C->cols->n * P.kpad;
  C->nagglomerated = P.nagg;
  C->launches = 1;  // the finalize kernel
  for (const Stage& st : P.stages) C->launches += stage_launches(st);
  C->workspace_bytes = (P.ws_len + P.fac_len) * 8;
  C->uid = ++g_uid;
  C->stream = s;
  if (cudaMallocAsync(&C->d_arena, C->arena_len * sizeof(double), s) != cudaSuccess ||
      cudaMallocAsync(&C->d_int, (2 * C->rows->ncl + 1) * sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    h2_free(C);
    return H2_ENOMEM;
  }
  cudaMemsetAsync(C->d_arena, 0, P.c_len * sizeof(double), s);
  *Cout = C;
  return H2_OK;
}

// Per-product parameters (scal[0..PARAM_COUNT)).
static void product_params(const MulArgs& m, double* params) {
  params[PARAM_TOL_BASIS] = m.eps / 4.0 * std::sqrt(1.0 - 2.0 * m.theta);
  params[PARAM_TOL_AGG] = m.eps / 3.0;
  params[PARAM_SVD_FLOOR] = svd_noise_floor(m.eps, m.precision);
  params[PARAM_SVD_SWEEPS] = (double)m.svd_sweeps;
}

// Enqueues the product on stream s with plan instance rt; *Cout holds C,
// whose `done` event marks its completion.
static int enqueue_product(const MulArgs& m, PlanRT& rt, cudaStream_t s, h2_kernel_prof* prof, h2_matrix** Cout) {
  h2_matrix* A = m.A;
  h2_matrix* B = m.B;
  int rc;
  if ((rc = ensure_level_bases(A, s)) || (rc = ensure_level_bases(B, s))) return rc;
  h2_matrix* C = nullptr;
  if ((rc = new_product_matrix(m, *rt.plan, s, &C))) return rc;
  double params[PARAM_COUNT];
  product_params(m, params);
  rc = prof ? run_plan_profiled(rt, A->d_arena, B->d_arena, C->d_arena, C->d_int, params, s, prof)
            : run_plan(rt, A->d_arena, B->d_arena, C->d_arena, C->d_int, params, s, true);
  if (rc) {
    h2_free(C);
    return rc;
  }
  cudaEventCreateWithFlags(&C->done, cudaEventDisableTiming);
  cudaEventRecord(C->done, s);
  *Cout = C;
  return H2_OK;
}

static int mul_impl(const h2_matrix* Ac, const h2_matrix* Bc, double eps, const h2_mul_opts* opts, h2_kernel_prof* prof,
                    h2_matrix** Cout) {
  if (!Cout) return H2_EINVAL;
  *Cout = nullptr;
  MulArgs m;
  int rc = mul_args(Ac, Bc, eps, opts, m);
  if (rc) return rc;
  if ((rc = lib_init())) return rc;
  std::shared_ptr<PlanEntry> e;
  if ((rc = mul_entry(m, e))) return rc;
  std::shared_ptr<PlanRT> rt;
  {
    std::lock_guard<std::mutex> lk(e->mu);
    rt = e->inst[0];  // replays of one instance are ordered by its event
  }
  if ((rc = enqueue_product(m, *rt, m.stream, prof, Cout))) return rc;
  if (m.sync) {
    rc = h2_check(*Cout);
    if (rc) {
      h2_free(*Cout);
      *Cout = nullptr;
      return rc;
    }
  }
  return H2_OK;
}

static int hmul_impl(const h2_matrix* Ac, const h2_matrix* Bc, double eps, const h2_mul_opts* opts,
                     h2_hmatrix** Cout) {
  if (!Cout) return H2_EINVAL;
  *Cout = nullptr;
  if (!Ac || !Bc || !(eps >= 0.0) || !std::isfinite(eps)) return H2_EINVAL;
  h2_matrix* A = const_cast<h2_matrix*>(Ac);
  h2_matrix* B = const_cast<h2_matrix*>(Bc);
  if (A->cols->hash != B->rows->hash || A->cols->n != B->rows->n) return H2_ETREE;
  if (A->kpad != B->kpad) return H2_EINVAL;
  if (opts && opts->precision != 0) return H2_EINVAL;
  const int max_rank = opts ? opts->max_rank : 0;
  if (max_rank < 0 || max_rank > GEMM_MAXTILE) return H2_EINVAL;
  const bool sync = opts ? opts->sync != 0 : true;
  cudaStream_t s = (opts && opts->stream) ? (cudaStream_t)opts->stream : g_stream;
  int rc = lib_init();
  if (rc) return rc;
  if ((rc = ensure_level_bases(A, s)) || (rc = ensure_level_bases(B, s))) return rc;
  const PlanKey key{matrix_sig(A), matrix_sig(B), -1 - max_rank};  // H-matrix plans: negative option codes
  std::shared_ptr<PlanEntry> ent = plan_lookup(key);
  if (!ent) {
    MulOptions mo;
    mo.eta = A->eta;
    mo.max_rank = max_rank;
    mo.hmatrix = true;
    ent = std::make_shared<PlanEntry>();
    try {
      ent->plan = make_product_plan(desc_of(A), desc_of(B), mo);
    } catch (const std::exception& ex) {
      g_last_cuda = ex.what();
      return H2_EINVAL;
    }
    ent->rank_src = ent->plan->rank_row_slot;
    auto rt0 = std::make_shared<PlanRT>();
    rt0->plan = ent->plan;
    rc = upload_plan(*rt0, ent->rank_src);
    if (rc == H2_ENOMEM) {
      plan_cache_clear();
      rt0 = std::make_shared<PlanRT>();
      rt0->plan = ent->plan;
      rc = upload_plan(*rt0, ent->rank_src);
    }
    if (rc) return rc;
    ent->inst.push_back(rt0);
    plan_insert(key, ent);
  }
  std::shared_ptr<PlanRT> rt;
  {
    std::lock_guard<std::mutex> elk(ent->mu);
    rt = ent->inst[0];
  }
  const Plan& P = *rt->plan;
  auto C = new h2_hmatrix();
  C->rows = A->rows;
  C->cols = B->cols;
  C->blocks = P.cblocks;
  C->arena_len = P.c_len;
  C->off_N = P.c_off_N;
  C->off_L = P.hm_off_L;
  C->off_R = P.hm_off_R;
  C->w = P.hm_w;
  const size_t nint = P.hm_off_L.size() + 1;
  if (cudaMallocAsync(&C->d_arena, std::max<int64_t>(C->arena_len, 1) * sizeof(double), s) != cudaSuccess ||
      cudaMallocAsync(&C->d_int, nint * sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    h2_hmatrix_free(C);
    return H2_ENOMEM;
  }
  cudaMemsetAsync(C->d_arena, 0, C->arena_len * sizeof(double), s);
  cudaMemsetAsync(C->d_int, 0, nint * sizeof(int), s);
  const double params[PARAM_COUNT] = {0.0, eps / 3.0, svd_noise_floor(eps, 0)};
  rc = run_plan(*rt, A->d_arena, B->d_arena, C->d_arena, C->d_int, params, s, true);
  if (rc) {
    h2_hmatrix_free(C);
    return rc;
  }
  cudaEventCreateWithFlags(&C->done, cudaEventDisableTiming);
  cudaEventRecord(C->done, s);
  *Cout = C;
  if (sync) {
    rc = h2_hmatrix_ranks(C, nullptr, nullptr, nullptr, nullptr);
    if (rc) {
      h2_hmatrix_free(C);
      *Cout = nullptr;
      return rc;
    }
  }
  return H2_OK;
}

int h2_mul(const h2_matrix* A, const h2_matrix* B, double eps, const h2_mul_opts* opts, h2_matrix** C) {
  return mul_impl(A, B, eps, opts, nullptr, C);
}

int h2_mul_h(const h2_matrix* A, const h2_matrix* B, double eps, const h2_mul_opts* opts, h2_hmatrix** C) {
  return hmul_impl(A, B, eps, opts, C);
}

void h2_hmatrix_free(h2_hmatrix* C) {
  if (!C) return;
  if (C->done) {
    cudaEventSynchronize(C->done);
    cudaEventDestroy(C->done);
  }
  if (C->d_arena) cudaFree(C->d_arena);
  if (C->d_int) cudaFree(C->d_int);
  delete C;
}

int h2_hmatrix_ranks(const h2_hmatrix* C, int* ranks, int* nadm, int* rank_max, int64_t* device_bytes) {
  if (!C) return H2_EINVAL;
  if (C->done) CK(cudaEventSynchronize(C->done));
  const int na = (int)C->off_L.size();
  std::vector<int> r(na + 1);
  CK(cudaMemcpy(r.data(), C->d_int, (na + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  if (r[na] != 0) return map_err(r[na]);
  if (ranks) std::copy(r.begin(), r.begin() + na, ranks);
  if (nadm) *nadm = na;
  if (rank_max) *rank_max = na ? *std::max_element(r.begin(), r.begin() + na) : 0;
  if (device_bytes) *device_bytes = C->arena_len * 8 + (na + 1) * 4;
  return H2_OK;
}

int h2_hmatrix_to_dense(const h2_hmatrix* C, double* out, int on_device) {
  if (!C || !out) return H2_EINVAL;
  int rc = lib_init();
  if (rc) return rc;
  if (C->done) CK(cudaEventSynchronize(C->done));
  cudaStream_t s = g_stream;
  PlanRT rt;
  rt.plan = make_hmatrix_dense_plan(*C->rows, *C->cols, *C->blocks, C->off_N, C->off_L, C->off_R, C->w);
  rc = upload_plan(rt, {});
  if (rc) return rc;
  const double params[PARAM_COUNT] = {0.0, 0.0};
  rc = run_plan(rt, C->d_arena, nullptr, nullptr, nullptr, params, s, false);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  const int64_t nr = C->rows->n, nc = C->cols->n;
  std::vector<double> d((size_t)nr * nc), o((size_t)nr * nc);
  CK(cudaMemcpy(d.data(), rt.d_ws, d.size() * 8, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < nr; ++i)
    for (int64_t j = 0; j < nc; ++j) o[(size_t)C->cols->perm[j] * nr + C->rows->perm[i]] = d[(size_t)i * nc + j];
  if (on_device) CK(cudaMemcpy(out, o.data(), o.size() * 8, cudaMemcpyHostToDevice));
  else std::memcpy(out, o.data(), o.size() * 8);
  return H2_OK;
}

int h2_mul_profile(const h2_matrix* A, const h2_matrix* B, double eps, const h2_mul_opts* opts,
                   h2_kernel_prof* out, h2_matrix** C) {
  if (!out) return H2_EINVAL;
  return mul_impl(A, B, eps, opts, out, C);
}

int h2_check(const h2_matrix* C) {
  if (!C) return H2_EINVAL;
  if (C->done) {
    cudaError_t e = cudaEventSynchronize(C->done);
    if (e != cudaSuccess) return cuda_fail(e, "h2_check");
  }
  int err = 0;
  const int ncl = C->rows->ncl;
  CK(cudaMemcpy(&err, C->d_int + 2 * ncl, sizeof(int), cudaMemcpyDeviceToHost));
  return map_err(err);
}

int h2_ranks(const h2_matrix* A, int* rr, int* rc) {
  if (!A || !rr || !rc) return H2_EINVAL;
  if (A->done) cudaEventSynchronize(A->done);
  const int ncl = A->rows->ncl;
  CK(cudaMemcpy(rr, A->d_int, ncl * sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(rc, A->d_int + ncl, ncl * sizeof(int), cudaMemcpyDeviceToHost));
  return H2_OK;
}

int h2_permutation(const h2_matrix* A, int64_t* perm) {
  if (!A || !perm) return H2_EINVAL;
  std::memcpy(perm, A->rows->perm.data(), sizeof(int64_t) * A->rows->n);
  return H2_OK;
}

int h2_info(const h2_matrix* A, h2_stats* st) {
  if (!A || !st) return H2_EINVAL;
  std::memset(st, 0, sizeof(*st));
  const int ncl = A->rows->ncl;
  std::vector<int> rr(ncl), rc(ncl);
  int r = h2_ranks(A, rr.data(), rc.data());
  if (r) return r;
  st->n = A->rows->n;
  st->dim = A->dim;
  st->depth = A->rows->depth;
  st->nclusters = ncl;
  st->nadm = (int)A->blocks->adm_list.size();
  st->ninadm = (int)A->blocks->inadm_list.size();
  st->kpad = A->kpad;
  st->row_rank_min = *std::min_element(rr.begin(), rr.end());
  st->row_rank_max = *std::max_element(rr.begin(), rr.end());
  st->col_rank_min = *std::min_element(rc.begin(), rc.end());
  st->col_rank_max = *std::max_element(rc.begin(), rc.end());
  st->nagglomerated = A->nagglomerated;
  st->device_bytes = A->arena_len * 8;
  st->launches = A->launches;
  st->workspace_bytes = A->workspace_bytes;
  return H2_OK;
}

int h2_matvec(const h2_matrix* Ac, const double* x, double* y, int on_device) {
  return h2_matvec_batch(Ac, x, y, 1, on_device, nullptr);
}

int h2_matvec_batch(const h2_matrix* Ac, const double* X, double* Y, int nrhs, int on_device, void* stream) {
  if (!Ac || !X || !Y || nrhs <= 0 || nrhs > MV_MAXRHS) return H2_EINVAL;
  h2_matrix* A = const_cast<h2_matrix*>(Ac);
  int rc = lib_init();
  if (rc) return rc;
  cudaStream_t s = stream ? (cudaStream_t)stream : g_stream;
  if (A->done) CK(cudaStreamWaitEvent(s, A->done, 0));
  const int64_t nr = A->rows->n, nc = A->cols->n;
  if (!A->d_perm) {
    std::vector<int> p(nr + nc);
    for (int64_t i = 0; i < nr; ++i) p[i] = (int)A->rows->perm[i];
    for (int64_t i = 0; i < nc; ++i) p[nr + i] = (int)A->cols->perm[i];
    CK(cudaMalloc(&A->d_perm, p.size() * sizeof(int)));
    CK(cudaMemcpy(A->d_perm, p.data(), p.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  const MvKey key{matrix_sig(A), nrhs};
  std::shared_ptr<PlanRT> rt = mv_lookup(key);
  if (!rt) {
    rt = std::make_shared<PlanRT>();
    rt->plan = make_matvec_plan(desc_of(A), nrhs);
    if ((rc = upload_plan(*rt, {}))) return rc;
    mv_insert(key, rt);
  }
  const Plan& P = *rt->plan;
  // the plan's workspace is shared by its replays: order this call after the last
  CK(cudaStreamWaitEvent(s, rt->last, 0));
  double* Xc = rt->d_ws + P.mv_ox;
  double* Yc = rt->d_ws + P.mv_oy;
  const double* Xd = X;
  double* Yd = Y;
  double* stage = nullptr;
  if (!on_device) {  // caller arrays on the host: stage them on the device
    CK(cudaMallocAsync(&stage, (size_t)(nr + nc) * nrhs * sizeof(double), s));
    CK(cudaMemcpyAsync(stage, X, (size_t)nc * nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
    Xd = stage;
    Yd = stage + (size_t)nc * nrhs;
  }
  const int64_t nx = nc * nrhs, ny = nr * nrhs;
  k_perm_gather<<<(unsigned)std::min<int64_t>((nx + 255) / 256, 65535 * 8), 256, 0, s>>>(Xd, A->d_perm + nr, nc,
                                                                                         nrhs, Xc);
  const double params[PARAM_COUNT] = {0.0, 0.0};
  rc = run_plan(*rt, A->d_arena, nullptr, nullptr, nullptr, params, s, true);
  if (rc) {
    if (stage) cudaFreeAsync(stage, s);
    return rc;
  }
  k_perm_scatter<<<(unsigned)std::min<int64_t>((ny + 255) / 256, 65535 * 8), 256, 0, s>>>(Yc, A->d_perm, nr, nrhs,
                                                                                          Yd);
  CK(cudaEventRecord(rt->last, s));
  if (!on_device) {
    CK(cudaMemcpyAsync(Y, Yd, (size_t)nr * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaFreeAsync(stage, s));
    CK(cudaStreamSynchronize(s));
  } else if (!stream) {
    CK(cudaStreamSynchronize(s));
  }
  CK(cudaGetLastError());
  return H2_OK;
}

int h2_to_dense(const h2_matrix* Ac, double* out, int on_device) {
  if (!Ac || !out) return H2_EINVAL;
  h2_matrix* A = const_cast<h2_matrix*>(Ac);
  int rc = lib_init();
  if (rc) return rc;
  if (A->done) CK(cudaEventSynchronize(A->done));
  cudaStream_t s = g_stream;
  if ((rc = ensure_level_bases(A, s))) return rc;
  PlanRT rt;
  rt.plan = make_dense_plan(desc_of(A));
  rc = upload_plan(rt, {});
  if (rc) return rc;
  const double params[PARAM_COUNT] = {0.0, 0.0};
  rc = run_plan(rt, A->d_arena, nullptr, nullptr, nullptr, params, s, false);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  const int64_t nr = A->rows->n, nc = A->cols->n;
  std::vector<double> d((size_t)nr * nc), o((size_t)nr * nc);
  CK(cudaMemcpy(d.data(), rt.d_ws, d.size() * 8, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < nr; ++i)
    for (int64_t j = 0; j < nc; ++j) o[(size_t)A->cols->perm[j] * nr + A->rows->perm[i]] = d[(size_t)i * nc + j];
  if (on_device) CK(cudaMemcpy(out, o.data(), o.size() * 8, cudaMemcpyHostToDevice));
  else std::memcpy(out, o.data(), o.size() * 8);
  return H2_OK;
}

}  // extern "C"

// ================================================================= server ====
// Continuous batching of products over resident operands.  Requests queue in
// arrival order; a dispatcher thread admits the oldest ones as soon as a
// stream slot is free and the device memory they need (a further instance of
// their plan when all of its instances are busy, plus the output) fits the
// budget.  Admitted products run concurrently on their own streams, so the
// small stages and tails of one overlap the work of the others.  A host
// callback on each stream marks completion and wakes the dispatcher.
namespace h2 {
namespace {

using Clock = std::chrono::steady_clock;

struct SrvReq {
  int64_t ticket = 0;
  MulArgs m;
  Clock::time_point t_submit, t_start, t_done;
  h2_matrix* C = nullptr;
  int rc = H2_OK;
  int slot = -1;
  std::shared_ptr<PlanRT> inst;
  int64_t out_bytes = 0;
  bool finished = false;   // device work done (callback) or failed at launch
};

}  // namespace
}  // namespace h2

struct h2_server {
  int nslots = 0;
  int64_t budget = 0, used = 0;
  std::vector<cudaStream_t> streams;
  std::vector<bool> slot_busy;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<h2::SrvReq>> pending;
  std::map<int64_t, std::shared_ptr<h2::SrvReq>> live;  // submitted and not yet collected
  std::map<h2::PlanRT*, bool> inst_busy;                // instances in use by this server
  std::vector<std::shared_ptr<h2::PlanEntry>> entries;  // entries this server holds instances of
  int64_t next_ticket = 1;
  bool stop = false;
  std::thread dispatcher;
};

namespace h2 {
namespace {

struct DoneArg {
  h2_server* srv;
  std::shared_ptr<SrvReq> req;
};

// Marks a request done and frees its stream slot and plan instance (the
// work before it on the stream has completed).  Bookkeeping only: no CUDA
// calls, as it runs as a stream host function.  Caller holds srv->mu.
void release_locked(h2_server* S, SrvReq& r) {
  r.t_done = Clock::now();
  r.finished = true;
  if (r.slot >= 0) S->slot_busy[r.slot] = false;
  if (r.inst) S->inst_busy[r.inst.get()] = false;
  r.slot = -1;
  r.inst.reset();
}

void CUDART_CB on_done(void* p) {
  auto* d = static_cast<DoneArg*>(p);
  {
    std::lock_guard<std::mutex> lk(d->srv->mu);
    release_locked(d->srv, *d->req);
  }
  d->srv->cv.notify_all();
  delete d;
}

// Output bytes of a product (its arena and integer array).
int64_t output_bytes(const Plan& P, const h2_matrix* A, const h2_matrix* B) {
  return 8 * (P.c_len + (int64_t)(A->rows->depth + 1) * A->rows->n * P.kpad +
              (int64_t)(B->cols->depth + 1) * B->cols->n * P.kpad) +
         4 * (2 * (int64_t)A->rows->ncl + 1);
}

// Tries to start the oldest pending request; false when it has to wait.
bool try_admit(h2_server* S, std::unique_lock<std::mutex>& lk) {
  if (S->pending.empty()) return false;
  int slot = -1;
  for (int i = 0; i < S->nslots; ++i)
    if (!S->slot_busy[i]) {
      slot = i;
      break;
    }
  if (slot < 0) return false;
  auto req = S->pending.front();
  // plan entry (planning runs without the lock)
  lk.unlock();
  std::shared_ptr<PlanEntry> e;
  int rc = mul_entry(req->m, e);
  lk.lock();
  if (S->pending.empty() || S->pending.front() != req) return true;  // dropped meanwhile: look again
  if (rc) {
    S->pending.pop_front();
    req->rc = rc;
    req->finished = true;
    return true;
  }
  std::vector<std::shared_ptr<PlanRT>> insts;
  {
    std::lock_guard<std::mutex> elk(e->mu);
    insts = e->inst;
  }
  if (std::find(S->entries.begin(), S->entries.end(), e) == S->entries.end()) {
    S->entries.push_back(e);
    S->used += instance_bytes(*e->plan) * (int64_t)insts.size();
  }
  const int64_t out_b = output_bytes(*e->plan, req->m.A, req->m.B);
  std::shared_ptr<PlanRT> inst;
  for (auto& i : insts)
    if (!S->inst_busy[i.get()]) {
      inst = i;
      break;
    }
  bool any_running = false;
  for (bool b : S->slot_busy) any_running |= b;
  if (!inst) {
    const int64_t need = instance_bytes(*e->plan);
    if (S->used + need + out_b > S->budget && any_running) return false;  // wait for memory
    lk.unlock();
    rc = clone_instance(insts[0], inst);
    lk.lock();
    if (rc == H2_OK) {
      std::lock_guard<std::mutex> elk(e->mu);
      e->inst.push_back(inst);
      S->used += need;
    }
    if (S->pending.empty() || S->pending.front() != req) return true;  // dropped meanwhile: look again
    if (rc) {
      if (!any_running) {  // nothing in flight to wait for: fail the request
        S->pending.pop_front();
        req->rc = rc;
        req->finished = true;
        return true;
      }
      return false;
    }
  } else if (S->used + out_b > S->budget && any_running) {
    return false;  // wait for memory; alone it runs regardless
  }
  S->pending.pop_front();
  S->slot_busy[slot] = true;
  S->inst_busy[inst.get()] = true;
  req->slot = slot;
  req->inst = inst;
  req->out_bytes = out_b;
  S->used += out_b;
  req->t_start = Clock::now();
  lk.unlock();
  cudaStream_t st = S->streams[slot];
  rc = enqueue_product(req->m, *inst, st, nullptr, &req->C);
  if (rc == H2_OK) {
    auto* d = new DoneArg{S, req};
    if (cudaLaunchHostFunc(st, on_done, d) != cudaSuccess) {
      delete d;
      cudaStreamSynchronize(st);
      lk.lock();
      release_locked(S, *req);
      return true;
    }
    lk.lock();
  } else {
    lk.lock();
    req->rc = rc;
    release_locked(S, *req);
  }
  return true;
}

void dispatch_loop(h2_server* S) {
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    if (S->stop && S->pending.empty()) break;
    bool progressed = false;
    while (try_admit(S, lk)) progressed = true;
    if (progressed) {
      S->cv.notify_all();
      continue;
    }
    S->cv.wait(lk);
  }
}

}  // namespace
}  // namespace h2

extern "C" {

int h2_server_create(int slots, int64_t mem_budget, h2_server** out) {
  if (!out || slots < 1 || slots > 64 || mem_budget < 0) return H2_EINVAL;
  *out = nullptr;
  int rc = lib_init();
  if (rc) return rc;
  auto S = new h2_server();
  S->nslots = slots;
  if (mem_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete S;
      return H2_ECUDA;
    }
    mem_budget = (int64_t)(0.9 * (double)fr);
  }
  S->budget = mem_budget;
  S->slot_busy.assign(slots, false);
  for (int i = 0; i < slots; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : S->streams) cudaStreamDestroy(x);
      delete S;
      return H2_ECUDA;
    }
    S->streams.push_back(st);
  }
  S->dispatcher = std::thread(dispatch_loop, S);
  *out = S;
  return H2_OK;
}

int h2_server_submit(h2_server* S, const h2_matrix* A, const h2_matrix* B, double eps, const h2_mul_opts* opts,
                     int64_t* ticket) {
  if (!S || !ticket) return H2_EINVAL;
  auto req = std::make_shared<SrvReq>();
  int rc = mul_args(A, B, eps, opts, req->m);
  if (rc) return rc;
  req->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return H2_EINVAL;
    req->ticket = S->next_ticket++;
    S->pending.push_back(req);
    S->live[req->ticket] = req;
    *ticket = req->ticket;
  }
  S->cv.notify_all();
  return H2_OK;
}

int h2_server_wait(h2_server* S, int64_t ticket, h2_matrix** C, double* queued_ms, double* total_ms) {
  if (!S || !C) return H2_EINVAL;
  *C = nullptr;
  std::shared_ptr<SrvReq> req;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->live.find(ticket);
    if (it == S->live.end()) return H2_EINVAL;
    req = it->second;
    S->cv.wait(lk, [&] { return req->finished; });
    S->live.erase(it);
    S->used -= req->out_bytes;
  }
  S->cv.notify_all();
  auto ms = [](Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
  };
  if (queued_ms) *queued_ms = req->rc == H2_OK ? ms(req->t_submit, req->t_start) : 0.0;
  if (total_ms) *total_ms = req->rc == H2_OK ? ms(req->t_submit, req->t_done) : 0.0;
  if (req->rc != H2_OK) return req->rc;
  const int rc = h2_check(req->C);
  if (rc) {
    h2_free(req->C);
    return rc;
  }
  *C = req->C;
  return H2_OK;
}

void h2_server_destroy(h2_server* S) {
  if (!S) return;
  {
    // requests not yet admitted are dropped; running ones finish
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (auto& r : S->pending) {
      r->rc = H2_EINVAL;
      r->finished = true;
    }
    S->pending.clear();
  }
  S->cv.notify_all();
  if (S->dispatcher.joinable()) S->dispatcher.join();
  for (auto st : S->streams) cudaStreamSynchronize(st);
  for (auto& kv : S->live)
    if (kv.second->C) h2_free(kv.second->C);
  for (auto st : S->streams) cudaStreamDestroy(st);
  delete S;
}

}  // extern "C"

// ------------------------------------------------------------ batching ----
// A batch runs many products in merged launches: the stage lists of all its
// products are interleaved so that one launch serves the matching stage of
// every product whose next stage it is (one segment per product), runs of
// consecutive GEMM stages become one persistent launch fed by a device work
// queue, where a job waits (bounded) for its product's previous stage, and
// the whole schedule is captured once in a CUDA graph.  Every product keeps
// its own plan instance (workspace, control block), so the arithmetic of
// every job is the one of the product run alone: results are bitwise equal.
namespace h2 {
namespace {

// Pinned launch choices of the autotuner per GEMM shape class: kernel
// variant (outputs per thread or tiles per warp) and, for persistent chains,
// CTAs per SM.  Neither changes the arithmetic of a job.
struct TuneKey {
  int mode, slices, mmax, nb, chain;
  bool operator<(const TuneKey& o) const {
    return std::tie(mode, slices, mmax, nb, chain) < std::tie(o.mode, o.slices, o.mmax, o.nb, o.chain);
  }
};
struct TuneVal {
  int variant, ctas_per_sm;
  float ms;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

struct BatchLaunch {
  int kind = 0;
  Stage st{};          // representative stage (GEMM: combined shape in aux)
  int seg0 = 0, nseg = 0, total = 0;
  bool chain = false;
  GemmShape g{};
  int grid = 0;        // chains: persistent grid
  int ctr0 = 0, nctr = 0;
  std::vector<std::pair<int, Stage>> scans;  // per-product scan stages
};

// Kernel variants a GEMM shape may use: the smallest that fits its largest
// tile, and the larger ones.
std::vector<int> gemm_variants(const GemmShape& g) {
  std::vector<int> v;
  if (g.slices) {
    for (int t : {1, 2, 4})
      if (t >= g.variant) v.push_back(t);
  } else {
    for (int q : {1, 4, 16})
      if (q >= g.variant) v.push_back(q);
  }
  return v;
}

}  // namespace
}  // namespace h2

struct h2_batch {
  int n = 0;
  std::vector<MulArgs> args;
  std::vector<std::shared_ptr<h2::PlanEntry>> entries;
  std::vector<std::shared_ptr<h2::PlanRT>> inst;
  std::vector<h2_matrix*> C;
  std::vector<h2::BatchLaunch> launches;
  std::vector<h2::BatchSeg> segs;
  h2::BatchSeg* d_segs = nullptr;
  int* d_ctr = nullptr;
  int nctr = 0;
  int nsm = 0;
  int test_wait = 0;
  int kernel_launches = 0;
  cudaStream_t cs = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t done = nullptr;
  ~h2_batch() {
    if (done) cudaEventSynchronize(done);
    if (graph) cudaGraphExecDestroy(graph);
    if (done) cudaEventDestroy(done);
    if (cs) cudaStreamDestroy(cs);
    cudaFree(d_segs);
    cudaFree(d_ctr);
    for (h2_matrix* c : C) h2_free(c);
  }
};

using namespace h2;

// Merged launch sequence of the batch: at every step the stage kind (GEMM:
// with its arithmetic mode; others: with identical launch parameters) that is
// next for the most products runs for all of them; then consecutive GEMM
// launches of one mode are fused into persistent chains.
static int batch_schedule(h2_batch* b) {
  const int P = b->n;
  std::vector<size_t> cur(P, 0);
  b->launches.clear();
  b->segs.clear();
  b->nctr = 0;
  auto key_of = [](const Stage& st) {
    if (st.kind == ST_GEMM) {
      const GemmShape g = gemm_shape(st.aux);
      return std::make_tuple((int)ST_GEMM, g.mode * 16 + g.slices, 0);
    }
    return std::make_tuple(st.kind, st.smem, st.aux);
  };
  for (;;) {
    std::map<std::tuple<int, int, int>, std::pair<int, size_t>> cand;
    for (int p = 0; p < P; ++p) {
      const auto& stages = b->inst[p]->plan->stages;
      if (cur[p] >= stages.size()) continue;
      auto& c = cand[key_of(stages[cur[p]])];
      c.first += 1;
      c.second = std::max(c.second, stages.size() - cur[p]);
    }
    if (cand.empty()) break;
    auto best = cand.begin();
    for (auto it = cand.begin(); it != cand.end(); ++it)
      if (it->second > best->second) best = it;
    const auto key = best->first;
    BatchLaunch L;
    L.kind = std::get<0>(key);
    L.seg0 = (int)b->segs.size();
    int mmax = 1, nb = 1, flags = 0;
    for (int p = 0; p < P; ++p) {
      const auto& stages = b->inst[p]->plan->stages;
      if (cur[p] >= stages.size() || key_of(stages[cur[p]]) != key) continue;
      const Stage& st = stages[cur[p]++];
      if (st.count <= 0) continue;
      if (L.nseg == 0) L.st = st;
      const PlanRT& rt = *b->inst[p];
      if (L.kind == ST_SCAN) {
        L.scans.emplace_back(p, st);
        continue;
      }
      BatchSeg sg{};
      sg.ctx = rt.d_ctx;
      switch (st.kind) {
        case ST_GEMM: sg.jobs = rt.dj.gemm_out + st.first; break;
        case ST_COPY: sg.jobs = rt.dj.copy + st.first; break;
        case ST_QR: sg.jobs = rt.dj.qr + st.first; break;
        case ST_QAPPLY: sg.jobs = rt.dj.qapply + st.first; break;
        case ST_SVD: sg.jobs = rt.dj.svd + st.first; break;
        case ST_NORM: sg.jobs = rt.dj.norm + st.first; break;
        default: break;
      }
      sg.terms = rt.dj.gemm_term;
      sg.start = L.total;
      sg.count = st.count;
      sg.wait_idx = sg.wait_target = sg.done_idx = -1;
      sg.first = (int)st.first;
      sg.done_idx = p;  // product index, replaced by a counter in chains
      L.total += st.count;
      b->segs.push_back(sg);
      ++L.nseg;
      if (st.kind == ST_GEMM) {
        const GemmShape g = gemm_shape(st.aux);
        mmax = std::max(mmax, g.mmax);
        nb = std::max(nb, g.nb);
        flags = st.aux & GEMM_AUX_FLAGS;
      }
    }
    if (L.kind == ST_SCAN) {
      if (!L.scans.empty()) b->launches.push_back(L);
      continue;
    }
    if (L.nseg == 0) continue;
    if (L.kind == ST_GEMM) {
      L.st.aux = (mmax << 16) | nb | flags;
      L.g = gemm_shape(L.st.aux);
    }
    b->launches.push_back(L);
  }
  // fuse runs of GEMM launches of one mode into chains
  std::vector<BatchLaunch> out;
  std::vector<BatchSeg> segs;
  for (size_t i = 0; i < b->launches.size();) {
    BatchLaunch& L = b->launches[i];
    size_t j = i + 1;
    if (L.kind == ST_GEMM)
      while (j < b->launches.size() && b->launches[j].kind == ST_GEMM &&
             (b->launches[j].st.aux & GEMM_AUX_FLAGS) == (L.st.aux & GEMM_AUX_FLAGS))
        ++j;
    if (L.kind != ST_GEMM || j - i < 2) {
      BatchLaunch M = L;
      M.seg0 = (int)segs.size();
      for (int k = 0; k < L.nseg; ++k) segs.push_back(b->segs[L.seg0 + k]);
      out.push_back(M);
      i = j;
      continue;
    }
    BatchLaunch Ch;
    Ch.kind = ST_GEMM;
    Ch.chain = true;
    Ch.seg0 = (int)segs.size();
    Ch.ctr0 = b->nctr;
    int mmax = 1, nb = 1;
    // counters of a chain, relative to its base ctr0: 0 the work queue, then
    // one done counter per segment
    std::map<int, std::pair<int, int>> last;  // product -> (done counter, count) of its latest chain stage
    int nextc = 1;
    for (size_t l = i; l < j; ++l) {
      const BatchLaunch& G = b->launches[l];
      mmax = std::max(mmax, G.g.mmax);
      nb = std::max(nb, G.g.nb);
      for (int k = 0; k < G.nseg; ++k) {
        BatchSeg sg = b->segs[G.seg0 + k];
        const int p = sg.done_idx;
        sg.start = Ch.total;
        auto it = last.find(p);
        if (it != last.end()) {
          sg.wait_idx = it->second.first;
          sg.wait_target = it->second.second;
        } else {
          sg.wait_idx = sg.wait_target = -1;
        }
        sg.done_idx = nextc;
        last[p] = {nextc, sg.count};
        ++nextc;
        Ch.total += sg.count;
        segs.push_back(sg);
        ++Ch.nseg;
      }
    }
    Ch.nctr = nextc;
    b->nctr = Ch.ctr0 + nextc;
    Ch.st = b->launches[i].st;
    Ch.st.aux = (mmax << 16) | nb | (Ch.st.aux & GEMM_AUX_FLAGS);
    Ch.g = gemm_shape(Ch.st.aux);
    out.push_back(Ch);
    i = j;
  }
  for (auto& M : out)
    if (!M.chain)
      for (int k = 0; k < M.nseg; ++k) segs[M.seg0 + k].done_idx = -1;
  // test hook: the first chain's first job waits on a counter nothing sets
  // (one past every chain's counters; zeroed once at upload, never written)
  if (b->test_wait) {
    for (auto& M : out)
      if (M.chain) {
        segs[M.seg0].wait_idx = b->nctr - M.ctr0;
        segs[M.seg0].wait_target = 1;
        ++b->nctr;
        break;
      }
  }
  b->launches.swap(out);
  b->segs.swap(segs);
  // pinned launch choices, persistent grids
  for (auto& M : b->launches) {
    if (M.kind != ST_GEMM) continue;
    int cps = 0;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(TuneKey{M.g.mode, M.g.slices, M.g.mmax, M.g.nb, M.chain ? 1 : 0});
      if (it != g_tune.end()) {
        M.g.variant = it->second.variant;
        cps = it->second.ctas_per_sm;
      }
    }
    if (M.chain) {
      const int occ = gemm_chain_blocks_per_sm(M.g);
      if (occ <= 0) return H2_ECUDA;
      const int c = cps > 0 ? std::min(cps, occ) : occ;
      M.grid = std::min(M.total, c * b->nsm);
    }
  }
  return H2_OK;
}

// Enqueues the batch's launches (graph capture or direct).  tgt: per launch
// the (variant, ctas per SM) to use instead of the scheduled ones (tuning),
// ev: events around every GEMM launch (tuning).
static void batch_enqueue(h2_batch* b, cudaStream_t s, const std::vector<std::pair<int, int>>* tgt,
                          std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev) {
  b->kernel_launches = 0;
  for (int p = 0; p < b->n; ++p) {
    const PlanRT& rt = *b->inst[p];
    const Plan& P = *rt.plan;
    cudaMemsetAsync(b->C[p]->d_arena, 0, P.c_len * sizeof(double), s);
    if (!P.slot_init.empty())
      cudaMemcpyAsync(rt.d_slot, rt.d_slot_init, sizeof(int) * P.slot_init.size(), cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(rt.d_err, 0, sizeof(int), s);
  }
  for (size_t l = 0; l < b->launches.size(); ++l) {
    const BatchLaunch& L = b->launches[l];
    if (L.kind == ST_SCAN) {
      for (const auto& ps : L.scans) {
        launch_stage(ps.second, b->inst[ps.first]->d_ctx, b->inst[ps.first]->dj, s);
        ++b->kernel_launches;
      }
      continue;
    }
    GemmShape g = L.g;
    int grid = L.grid;
    if (L.kind == ST_GEMM && tgt) {
      g.variant = (*tgt)[l].first;
      if (L.chain) {
        const int occ = gemm_chain_blocks_per_sm(g);
        grid = std::min(L.total, std::max(1, std::min((*tgt)[l].second, occ)) * b->nsm);
      }
    }
    if (ev && L.kind == ST_GEMM) cudaEventRecord((*ev)[l].first, s);
    if (L.chain) {
      cudaMemsetAsync(b->d_ctr + L.ctr0, 0, sizeof(int) * L.nctr, s);
      launch_gemm_chain(g, grid, b->d_segs + L.seg0, L.nseg, L.total, b->d_ctr + L.ctr0, s);
      ++b->kernel_launches;
    } else if (L.kind == ST_GEMM) {
      launch_gemm_batched(g, b->d_segs + L.seg0, L.nseg, L.total, s);
      ++b->kernel_launches;
    } else {
      launch_stage_batched(L.st, b->d_segs + L.seg0, L.nseg, L.total, s);
      b->kernel_launches += stage_launches(L.st);
    }
    if (ev && L.kind == ST_GEMM) cudaEventRecord((*ev)[l].second, s);
  }
  for (int p = 0; p < b->n; ++p) {
    launch_finalize(b->inst[p]->d_ctx, b->inst[p]->nrank, s);
    ++b->kernel_launches;
  }
}

static int batch_capture(h2_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
  batch_enqueue(b, b->cs, nullptr, nullptr);
  cudaError_t e = cudaStreamEndCapture(b->cs, &g);
  if (e != cudaSuccess) return cuda_fail(e, "batch capture");
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "batch instantiate");
  return H2_OK;
}

static int batch_upload(h2_batch* b) {
  cudaFree(b->d_segs);
  cudaFree(b->d_ctr);
  b->d_segs = nullptr;
  b->d_ctr = nullptr;
  CK(cudaMalloc(&b->d_segs, std::max<size_t>(b->segs.size(), 1) * sizeof(BatchSeg)));
  if (!b->segs.empty())
    CK(cudaMemcpy(b->d_segs, b->segs.data(), b->segs.size() * sizeof(BatchSeg), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&b->d_ctr, std::max(b->nctr, 1) * sizeof(int)));
  CK(cudaMemset(b->d_ctr, 0, std::max(b->nctr, 1) * sizeof(int)));
  return H2_OK;
}

int h2_batch_create(int nprod, const h2_matrix* const* A, const h2_matrix* const* B, const double* eps,
                    const h2_mul_opts* opts, const h2_batch_opts* bopts, h2_batch** out) {
  if (!out) return H2_EINVAL;
  *out = nullptr;
  if (nprod < 1 || nprod > 4096 || !A || !B || !eps) return H2_EINVAL;
  int rc = lib_init();
  if (rc) return rc;
  auto b = std::make_unique<h2_batch>();
  b->n = nprod;
  b->test_wait = bopts ? bopts->test_unreachable_wait : 0;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
  for (int p = 0; p < nprod; ++p) {
    MulArgs m;
    if ((rc = mul_args(A[p], B[p], eps[p], opts, m))) return rc;
    std::shared_ptr<PlanEntry> e;
    if ((rc = mul_entry(m, e))) return rc;
    std::shared_ptr<PlanRT> base;
    {
      std::lock_guard<std::mutex> lk(e->mu);
      base = e->inst[0];
    }
    std::shared_ptr<PlanRT> rt;  // a workspace of its own for every product of the batch
    if ((rc = clone_instance(base, rt))) return rc;
    if ((rc = ensure_level_bases(m.A, g_stream)) || (rc = ensure_level_bases(m.B, g_stream))) return rc;
    h2_matrix* C = nullptr;
    if ((rc = new_product_matrix(m, *rt->plan, g_stream, &C))) return rc;
    b->C.push_back(C);
    CK(cudaEventCreateWithFlags(&C->done, cudaEventDisableTiming));
    // control block: fixed for the batch's lifetime
    ExecCtx ctx{};
    const Plan& P = *rt->plan;
    ctx.base[AR_WS] = rt->d_ws;
    ctx.base[AR_X] = m.A->d_arena;
    ctx.base[AR_Y] = m.B->d_arena;
    ctx.base[AR_C] = C->d_arena;
    ctx.base[AR_K] = rt->d_konst;
    ctx.base[AR_F] = rt->d_ws + P.ws_len;
    ctx.slot = rt->d_slot;
    ctx.scal = rt->d_scal;
    ctx.nrm = rt->d_nrm;
    ctx.err = rt->d_err;
    ctx.idx = rt->d_idx;
    ctx.out_int = C->d_int;
    ctx.rank_src = rt->d_rank_src;
    ctx.nrank = rt->nrank;
    double params[PARAM_COUNT];
    product_params(m, params);
    std::vector<char> h(512 + sizeof(double) * PARAM_COUNT, 0);
    std::memcpy(h.data(), &ctx, sizeof(ctx));
    std::memcpy(h.data() + 512, params, sizeof(params));
    CK(cudaStreamSynchronize(g_stream));
    CK(cudaMemcpy(rt->d_ctrl, h.data(), h.size(), cudaMemcpyHostToDevice));
    b->args.push_back(m);
    b->entries.push_back(e);
    b->inst.push_back(rt);
  }
  if ((rc = batch_schedule(b.get())) || (rc = batch_upload(b.get())) || (rc = batch_capture(b.get()))) return rc;
  *out = b.release();
  return H2_OK;
}

int h2_batch_run(h2_batch* b, void* stream, int sync) {
  if (!b) return H2_EINVAL;
  cudaStream_t s = stream ? (cudaStream_t)stream : g_stream;
  for (int p = 0; p < b->n; ++p) {
    if (b->args[p].A->done) CK(cudaStreamWaitEvent(s, b->args[p].A->done, 0));
    if (b->args[p].B->done) CK(cudaStreamWaitEvent(s, b->args[p].B->done, 0));
    std::lock_guard<std::mutex> lk(b->C[p]->mu);
    b->C[p]->levels_ready = false;  // the level bases of a result are rebuilt if it is used as an operand
  }
  CK(cudaGraphLaunch(b->graph, s));
  for (int p = 0; p < b->n; ++p) CK(cudaEventRecord(b->C[p]->done, s));
  CK(cudaEventRecord(b->done, s));
  if (!sync) return H2_OK;
  CK(cudaEventSynchronize(b->done));
  for (int p = 0; p < b->n; ++p) {
    const int rc = h2_check(b->C[p]);
    if (rc) return rc;
  }
  return H2_OK;
}

int h2_batch_result(const h2_batch* b, int i, const h2_matrix** C) {
  if (!b || !C || i < 0 || i >= b->n) return H2_EINVAL;
  *C = b->C[i];
  return H2_OK;
}

int h2_batch_info(const h2_batch* b, int* launches, int* chains, int* kernel_launches) {
  if (!b) return H2_EINVAL;
  int nl = 0, nc = 0;
  for (const auto& L : b->launches) {
    nl += L.kind == ST_SCAN ? (int)L.scans.size() : 1;
    nc += L.chain ? 1 : 0;
  }
  if (launches) *launches = nl;
  if (chains) *chains = nc;
  if (kernel_launches) *kernel_launches = b->kernel_launches;
  return H2_OK;
}

int h2_batch_autotune(h2_batch* b, int* ntuned) {
  if (!b) return H2_EINVAL;
  CK(cudaEventSynchronize(b->done));
  const size_t nl = b->launches.size();
  // candidates per GEMM launch: variants x (chains) CTAs per SM
  std::vector<std::vector<std::pair<int, int>>> cand(nl);
  size_t ncand = 1;
  for (size_t l = 0; l < nl; ++l) {
    const BatchLaunch& L = b->launches[l];
    if (L.kind != ST_GEMM) continue;
    GemmShape g0 = gemm_shape(L.st.aux);
    for (int v : gemm_variants(g0)) {
      if (!L.chain) {
        cand[l].push_back({v, 0});
        continue;
      }
      GemmShape g = g0;
      g.variant = v;
      const int occ = gemm_chain_blocks_per_sm(g);
      for (int c = 1; c <= occ; c = (c < occ && 2 * c > occ) ? occ : 2 * c) cand[l].push_back({v, c});
    }
    ncand = std::max(ncand, cand[l].size());
  }
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev(nl);
  for (auto& e : ev) {
    CK(cudaEventCreate(&e.first));
    CK(cudaEventCreate(&e.second));
  }
  std::vector<std::vector<float>> ms(nl, std::vector<float>(ncand, 1e30f));
  std::vector<std::pair<int, int>> tgt(nl, {1, 1});
  for (size_t c = 0; c < ncand; ++c) {
    for (size_t l = 0; l < nl; ++l)
      if (!cand[l].empty()) tgt[l] = cand[l][std::min(c, cand[l].size() - 1)];
    batch_enqueue(b, b->cs, &tgt, &ev);
    CK(cudaStreamSynchronize(b->cs));
    for (size_t l = 0; l < nl; ++l)
      if (!cand[l].empty() && c < cand[l].size()) CK(cudaEventElapsedTime(&ms[l][c], ev[l].first, ev[l].second));
  }
  for (auto& e : ev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  int nt = 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (size_t l = 0; l < nl; ++l) {
      if (cand[l].empty()) continue;
      size_t best = 0;
      for (size_t c = 1; c < cand[l].size(); ++c)
        if (ms[l][c] < ms[l][best]) best = c;
      const BatchLaunch& L = b->launches[l];
      const GemmShape g0 = gemm_shape(L.st.aux);
      const TuneKey k{g0.mode, g0.slices, g0.mmax, g0.nb, L.chain ? 1 : 0};
      auto it = g_tune.find(k);
      if (it == g_tune.end() || ms[l][best] < it->second.ms) {  // a class keeps its fastest choice seen
        g_tune[k] = TuneVal{cand[l][best].first, cand[l][best].second, ms[l][best]};
        ++nt;
      }
    }
  }
  if (ntuned) *ntuned = nt;
  int rc;
  if ((rc = batch_schedule(b)) || (rc = batch_upload(b)) || (rc = batch_capture(b))) return rc;
  return H2_OK;
}

int h2_tuning_table(char* buf, int len) {
  std::string s;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& kv : g_tune) {
      char line[160];
      std::snprintf(line, sizeof line, "mode %d slices %d tile %dx%d %s: variant %d ctas/SM %d (%.3f ms)\n",
                    kv.first.mode, kv.first.slices, kv.first.mmax, kv.first.nb, kv.first.chain ? "chain" : "stage",
                    kv.second.variant, kv.second.ctas_per_sm, kv.second.ms);
      s += line;
    }
  }
  if (buf && len > 0) {
    std::snprintf(buf, (size_t)len, "%s", s.c_str());
  }
  return (int)s.size();
}

void h2_batch_free(h2_batch* b) { delete b; }
