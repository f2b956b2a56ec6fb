// Host planner of the H^2 x H^2 product (Sections 3-5 of Boerm, arXiv
// 2403.01566), GB300 formulation.
//
// The paper's recursion (accumulators with basis trees, Sections 3-4) is
// flattened into level-synchronous batches:
//
//  1. Basis products P_s = W_{X,s}^* V_{Y,s}, leaves then upwards (Section 4.1).
//  2. The product tree (Def. 6) is enumerated symbolically.  Every admissible
//     product leaf contributes "records": case 1 (eq. (6a), addproduct of
//     Fig. 1 unrolled over the block subtree of X below (t,s)) gives
//     V_{X,u} (S_{X,us'} P_{s'} E..E S_{Y,sr}) W_{Y,r}^* at node u, or the
//     nearfield form X|_{u x s'} V_{Y,s'} E..E S_{Y,sr} for inadmissible X
//     leaves; case 2 is the mirror on the adjoint (eq. (6b)); case 3 adds
//     dense leaf products.  Records are keyed by (node, column cluster of the
//     accumulator that received them).
//  3. The accumulator splits of Sections 3.3/4.3 (restriction by E_{X,t'}, right
//     transform by F_{Y,r'}^*) become two pushes: Omega(u,r) = rec(u,r) +
//     Omega(u,parent r) F_{Y,r}^* down the column tree, and the root
//     coefficients ahat_{t'r'} = E_{X,t'} ahat_{tr} F_{Y,r'}^* + Omega(t',r')
//     down the tree of visited accumulators; a final push over desc(t) gives the
//     explicit semi-uniform factors A_tr (|t| x k) and B_tr (|r| x k).
//  4. Admissible target leaves whose induced structure is finer are
//     agglomerated (Section 5.1): the sub-blocks refined to the deepest level
//     form an n x n grid, merged row by row, then the rows, with relative
//     tolerance eps_c/(2 n^2).
//  5. Condensation (QR of the right factor), exact block norms, weighted
//     adaptive row and column bases with the projection climb, and coupling
//     matrices (Sections 5.2-5.3).
#include "h2_plan.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <functional>
#include <stdexcept>
#include <unordered_map>
#include <unordered_set>
#include <set>
#include <array>
#include <tuple>

#include "h2_kernels.h"

namespace h2 {

Plan::~Plan() {}

namespace {

inline Dim DC(int c) { return Dim{c, -1, -1}; }
inline Dim DS(int s, int c = 0) { return Dim{c, s, -1}; }
inline Dim DSS(int s1, int s2) { return Dim{0, s1, s2}; }
inline Ptr PT(int ar, int64_t off) { return Ptr{off, ar, -1, 0, -1, 0}; }
inline Ptr NONE() { return Ptr{0, AR_NONE, -1, 0, -1, 0}; }
inline Ptr padd(Ptr p, int64_t d) {
  p.off += d;
  return p;
}
inline Ptr pdyn(Ptr p, int s, int mult) {
  if (s < 0) return p;
  if (p.ds < 0) {
    p.ds = s;
    p.dm = mult;
  } else {
    p.ds2 = s;
    p.dm2 = mult;
  }
  return p;
}
inline int64_t key2(int a, int b) { return ((int64_t)a << 32) | (uint32_t)b; }

// A matrix reference: pointer, leading dimension, transpose flag.
struct MRef {
  Ptr p;
  int ld;
  int t;
};
inline MRef mref(Ptr p, int ld, int t = 0) { return MRef{p, ld, t}; }
inline MRef rows_of(MRef m, int64_t r0) {  // row offset of a non-transposed ref
  m.p = padd(m.p, r0 * m.ld);
  return m;
}

// Dims that may be static or read from a slot.
struct DimV {
  int c;
  int s;  // slot or -1
  int max;
  Dim d() const { return s >= 0 ? DS(s, c) : DC(c); }
};
inline DimV dv(int c) { return DimV{c, -1, c}; }
inline DimV dvs(int s, int max) { return DimV{0, s, max}; }
// width a + b of two (static or slot) dims
inline Dim merged_width(const DimV& a, const DimV& b) {
  if (a.s >= 0 && b.s >= 0) return Dim{a.c + b.c, a.s, b.s};
  if (a.s >= 0) return Dim{a.c + b.c, a.s, -1};
  if (b.s >= 0) return Dim{a.c + b.c, b.s, -1};
  return Dim{a.c + b.c, -1, -1};
}

// Bits of a planning-time workspace offset that address the inside of a
// buffer (up to 2^36 doubles); the bits above hold the buffer index.
constexpr int WS_LOCAL_BITS = 36;
constexpr int64_t WS_LOCAL_MASK = (int64_t(1) << WS_LOCAL_BITS) - 1;

// Places the tagged workspace buffers of a finished product plan by lifetime
// and rewrites every workspace pointer of its jobs; returns the workspace
// length (doubles).  A buffer lives from the first to the last stage whose
// jobs address it; buffers of the same lifetime are laid out as one group.
// Groups are placed largest first, each at the lowest address that no
// already placed group of overlapping lifetime occupies (offline placement
// with known lifetimes; on the k = 64 sphere at n = 65536 it needs 1.04 times
// the largest live total, against 1.36 for first-fit in order of first use).
// Stages of one product run in order (a chained GEMM stage waits for its
// product's previous one), so two buffers share memory only when no stage can
// see both.  The arithmetic of every job is unchanged: only addresses move.
static int64_t pack_workspace(Plan& P, const std::vector<int64_t>& bufs) {
  const size_t nb = bufs.size();
  std::vector<int> first(nb, INT_MAX), last(nb, -1);
  auto touch = [&](const Ptr& p, int s) {
    if (p.arena != AR_WS) return;
    const size_t id = (size_t)(p.off >> WS_LOCAL_BITS);
    if (id >= nb) throw std::runtime_error("workspace pointer outside every buffer");
    first[id] = std::min(first[id], s);
    last[id] = std::max(last[id], s);
  };
  auto each_ptr = [&](auto&& f) {
    for (size_t si = 0; si < P.stages.size(); ++si) {
      const Stage& st = P.stages[si];
      const int s = (int)si;
      for (int j = 0; j < st.count; ++j) {
        const int64_t J = st.first + j;
        switch (st.kind) {
          case ST_GEMM: {
            GemmOut& O = P.gout[J];
            f(O.o, s);
            for (int t = O.t0; t < O.t1; ++t) {
              GemmTerm& T = P.gterm[t];
              f(T.a, s);
              f(T.b, s);
              f(T.c, s);
            }
            break;
          }
          case ST_COPY: f(P.copy[J].src, s); f(P.copy[J].dst, s); break;
          case ST_QR: f(P.qr[J].a, s); f(P.qr[J].tau, s); f(P.qr[J].r, s); f(P.qr[J].piv, s); break;
          case ST_QAPPLY: f(P.qap[J].a, s); f(P.qap[J].tau, s); f(P.qap[J].y, s); f(P.qap[J].out, s); break;
          case ST_SVD: f(P.svd[J].src, s); f(P.svd[J].u, s); f(P.svd[J].sig, s); f(P.svd[J].piv, s); break;
          case ST_NORM: f(P.norm[J].src, s); break;
          default: break;
        }
      }
    }
  };
  each_ptr([&](Ptr& p, int s) { touch(p, s); });
  // groups of equal lifetime
  std::map<std::pair<int, int>, int64_t> gsize;
  for (size_t i = 0; i < nb; ++i)
    if (last[i] >= 0) gsize[{first[i], last[i]}] += bufs[i];
  struct Grp {
    int first, last;
    int64_t len, base;
  };
  std::vector<Grp> gs;
  gs.reserve(gsize.size());
  for (const auto& [g, len] : gsize) gs.push_back(Grp{g.first, g.second, len, 0});
  std::stable_sort(gs.begin(), gs.end(), [](const Grp& a, const Grp& b) { return a.len > b.len; });
  std::map<std::pair<int, int>, int64_t> gbase;
  int64_t peak = 0;
  std::vector<std::pair<int64_t, int64_t>> busy;  // address ranges of overlapping placed groups
  for (size_t gi = 0; gi < gs.size(); ++gi) {
    Grp& g = gs[gi];
    busy.clear();
    for (size_t pj = 0; pj < gi; ++pj) {
      const Grp& o = gs[pj];
      if (o.last >= g.first && o.first <= g.last) busy.push_back({o.base, o.base + o.len});
    }
    std::sort(busy.begin(), busy.end());
    int64_t at = 0;
    for (const auto& [b0, b1] : busy) {
      if (b0 - at >= g.len) break;
      at = std::max(at, b1);
    }
    g.base = at;
    gbase[{g.first, g.last}] = at;
    peak = std::max(peak, at + g.len);
  }
  // invariant: groups whose lifetimes overlap occupy disjoint addresses
  for (size_t a = 0; a < gs.size(); ++a)
    for (size_t b = a + 1; b < gs.size(); ++b) {
      const Grp &x = gs[a], &y = gs[b];
      if (x.last >= y.first && y.last >= x.first && x.base < y.base + y.len && y.base < x.base + x.len)
        throw std::runtime_error("workspace placement overlaps two live buffers");
    }
  // buffer bases: consecutive inside their group
  std::vector<int64_t> base(nb, 0);
  std::map<std::pair<int, int>, int64_t> gnext = gbase;
  for (size_t i = 0; i < nb; ++i)
    if (last[i] >= 0) {
      int64_t& nx = gnext[{first[i], last[i]}];
      base[i] = nx;
      nx += bufs[i];
    }
  each_ptr([&](Ptr& p, int) {
    if (p.arena != AR_WS) return;
    p.off = base[(size_t)(p.off >> WS_LOCAL_BITS)] + (p.off & WS_LOCAL_MASK);
  });
  return std::max<int64_t>(peak, 1);
}

struct Builder {
  Plan& P;
  int64_t ws = 0, ws_peak = 0;
  std::vector<GemmOut> go;
  std::vector<GemmTerm> gt;
  std::vector<CopyJob> cp;
  std::vector<QrJob> qj;
  std::vector<double> qj_cost;  // static cost bound of each pending QR job
  std::vector<QApplyJob> qa;
  std::vector<SvdJob> sv;
  int sv_maxr = 1, sv_maxc = 1;  // largest pending SVD job
  int64_t sv_need = 0;           // shared memory (doubles) of the largest pending SVD job
  std::vector<double> sv_cost;   // static cost bound of each pending SVD job (from svd_size)
  std::vector<ScanJob> sc;
  std::vector<NormJob> nj;

  explicit Builder(Plan& p) : P(p) {}
  bool fp32_contractions = false;  // precision form 1
  bool df_contractions = false;    // precision form 2
  bool tc5_contractions = false;   // precision form 3 (tensor cores, 5 slices)
  bool tc7_contractions = false;   // precision form 4 (tensor cores, 7 slices, with compensated FP32)
  // Workspace buffers of a product plan are placed by lifetime once the
  // stage list is complete (pack_workspace): while planning, an offset
  // carries its buffer's index above the low WS_LOCAL_BITS bits, which hold
  // the offset inside the buffer.  ws / ws_peak count the bump-allocated
  // doubles (statistics; the placement of helper plans).
  bool tagged = false;
  std::vector<int64_t> bufs;  // sizes (doubles) of the tagged buffers
  int64_t alloc(int64_t n) {
    const int64_t sz = (std::max<int64_t>(n, 1) + 31) & ~int64_t(31);
    const int64_t o = tagged ? ((int64_t)bufs.size() << WS_LOCAL_BITS) : ws;
    if (tagged) bufs.push_back(sz);
    ws += sz;
    ws_peak = std::max(ws_peak, ws);
    return o;
  }
  int64_t fac = 0;  // bump pointer of the terminal-factor arena
  int64_t falloc(int64_t n) {
    const int64_t o = fac;
    fac += (std::max<int64_t>(n, 1) + 31) & ~int64_t(31);
    return o;
  }
  int slot(int init) {
    P.slot_init.push_back(init);
    return (int)P.slot_init.size() - 1;
  }
  int scal() { return P.nscal++; }

  // ---- GEMM jobs
  // Static upper bound of a dim (slot-valued dims: the 64-wide tile limit).
  static int dim_bound(const Dim& d) {
    if (d.s1 >= 0 || d.s2 >= 0) return d.mc >= 0 && d.ms < 0 ? std::min(d.mc, 64) : 64;
    return std::min(d.mc >= 0 && d.ms < 0 ? std::min(d.c, d.mc) : d.c, 64);
  }
  int g_mmax = 1, g_nb = 1;  // shape bounds of the pending GEMM stage
  void out(Ptr o, int ldo, Dim m, Dim n, int beta, int clampn = 0) {
    go.push_back(GemmOut{o, ldo, m, n, beta, (int)gt.size(), (int)gt.size(), clampn});
    g_mmax = std::max(g_mmax, dim_bound(m));
    g_nb = std::max(g_nb, clampn ? 64 : dim_bound(n));
  }
  void term2(MRef a, MRef b, Dim k1, double alpha = 1.0, int sidx = -1) {
    gt.push_back(GemmTerm{a.p, b.p, NONE(), a.ld, b.ld, 0, k1, DC(0), a.t, b.t, 0, alpha, sidx});
    go.back().t1++;
  }
  void term3(MRef a, MRef b, MRef c, Dim k1, Dim k2, double alpha = 1.0) {
    gt.push_back(GemmTerm{a.p, b.p, c.p, a.ld, b.ld, c.ld, k1, k2, a.t, b.t, c.t, alpha, -1});
    go.back().t1++;
    g_nb = std::max(g_nb, dim_bound(k2));
  }
  void add(MRef a, double alpha = 1.0) {
    gt.push_back(GemmTerm{a.p, NONE(), NONE(), a.ld, 0, 0, DC(0), DC(0), a.t, 0, 0, alpha, -1});
    go.back().t1++;
  }
  void flush_gemm(int tag) {
    if (go.empty()) return;
    const int base = (int)P.gterm.size();
    const int64_t first = (int64_t)P.gout.size();
    for (auto& o : go) {
      o.t0 += base;
      o.t1 += base;
      P.gout.push_back(o);
    }
    P.gterm.insert(P.gterm.end(), gt.begin(), gt.end());
    // FP32 contractions: the accumulation phases (basis products, records,
    // pushes, dense leaf products) and the coupling projection; agglomeration,
    // condensation and the bases stay FP64
    const bool f32 = fp32_contractions && (tag <= 9 || tag == 14);  // TAG_P .. TAG_DENSE, TAG_COUPLE
    // Tensor cores for the stages whose static tile bound is 64 x 64 (the
    // dense leaf products, merges, panels): there the slicing of an operand
    // element is shared by 64 outputs.  On smaller tiles the slicing and the
    // 15-28 slice products per step cost more than the compensated FP32
    // arithmetic they replace (measured), so form 4 keeps those compensated.
    const bool big = g_mmax >= 64 && g_nb >= 64;
    // compensated contractions (~1e-13), the 7-slice tensor-core form (about
    // FP64) and the 5-slice form: every GEMM stage
    const int mode_flag = (tc7_contractions && big)  ? GEMM_AUX_TC7
                          : (tc5_contractions)       ? GEMM_AUX_TC5
                          : (df_contractions || tc7_contractions) ? GEMM_AUX_DF
                          : f32                      ? GEMM_AUX_FP32
                                                     : 0;
    P.stages.push_back(Stage{ST_GEMM, first, (int)go.size(), tag, 0, (g_mmax << 16) | g_nb | mode_flag});
    go.clear();
    gt.clear();
    g_mmax = g_nb = 1;
  }
  // ---- copies
  void copy(Ptr src, int lds, Ptr dst, int ldd, Dim rows, Dim cols, int trans, double alpha = 1.0,
            int sidx = -1, Dim zr = DC(0), Dim zc = DC(0)) {
    cp.push_back(CopyJob{src, dst, lds, ldd, rows, cols, zr, zc, trans, alpha, sidx});
  }
  void flush_copy(int tag) {
    if (cp.empty()) return;
    P.stages.push_back(Stage{ST_COPY, (int64_t)P.copy.size(), (int)cp.size(), tag, 0});
    P.copy.insert(P.copy.end(), cp.begin(), cp.end());
    cp.clear();
  }
  // QR job; maxr/maxc are the largest values rows/cols can take (shared-memory
  // sizing of the stage); keep = 1 when a Q application needs the reflectors.
  int qr_smem = 0;
  void qr(Ptr a, int lda, Dim rows, Dim cols, Ptr tau, Ptr r, int ldr, int keep, int maxr, int maxc,
          Ptr piv = NONE(), int rmode = 0, int trunc_idx = -1, int rank_slot = -1) {
    qj.push_back(QrJob{a, tau, r, lda, ldr, rows, cols, keep, piv, rmode, trunc_idx, rank_slot});
    qj_cost.push_back((double)maxr * maxc * maxc);
    const int64_t cap = 6144;  // doubles (48 KB)
    const int64_t need = (int64_t)maxr * maxc;
    if (need <= cap) {
      qr_smem = (int)std::max<int64_t>(qr_smem, need * 8);
    } else if (!keep && maxc <= 64) {
      // R-only: may stream row chunks under the triangle (64 or 128 rows,
      // chosen per stage in flush_qr)
      qr_tsqr = (int)std::max<int64_t>(qr_tsqr, (int64_t)(maxc + 64) * maxc * 8);
      qr_tsqr_big = (int)std::max<int64_t>(qr_tsqr_big, (int64_t)(maxc + 128) * maxc * 8);
      ++qr_stream_jobs;
      if (maxr > 512) ++qr_stream_tall;
      if (trunc_idx >= 0) ++qr_stream_trunc;
    }
  }
  int qr_tsqr = 0, qr_tsqr_big = 0, qr_stream_jobs = 0, qr_stream_tall = 0, qr_stream_trunc = 0;
  // Jobs of one stage are independent: issue them largest first so that the
  // long ones do not start last and leave the tail of the launch to a few SMs.
  template <class Job>
  static void largest_first(std::vector<Job>& jobs, const std::vector<double>& cost) {
    if (cost.size() != jobs.size()) return;
    std::vector<int> ord(jobs.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<Job> out;
    out.reserve(jobs.size());
    for (int i : ord) out.push_back(jobs[i]);
    jobs.swap(out);
  }
  void flush_qr(int tag) {
    if (qj.empty()) return;
    largest_first(qj, qj_cost);
    qj_cost.clear();
    // Streaming row chunks trades L2 traffic for more, shorter steps.  The
    // 96 KB launch (128-row chunks, and jobs of up to 12288 elements wholly in
    // shared memory) wins for stages of mostly tall panels (over 512 rows) and
    // for QRs that stop at the noise floor (in shared memory they stop early;
    // streamed, every column is reduced before the truncated pivoted QR of the
    // triangle).  64-row chunks (three CTAs per SM) win when many short jobs
    // keep every SM busy; a few latency-bound short ones run faster in global
    // memory.  (grid2d n=16384: the 512 basis panels of ~915 rows 8.4 -> 7.7
    // ms, the condensed merge QRs 5.2 -> 4.4 ms; the 96 KB launch for a stage
    // of mostly short panels 2.5 -> 2.9 ms.)
    int smem = qr_smem;
    if (qr_stream_tall > 0 && 2 * qr_stream_tall >= qr_stream_jobs) smem = std::max(smem, qr_tsqr_big);
    else if (qr_stream_trunc > 0) smem = std::max(smem, qr_tsqr_big);
    else if (qj.size() >= 2048) smem = std::max(smem, qr_tsqr);
    P.stages.push_back(Stage{ST_QR, (int64_t)P.qr.size(), (int)qj.size(), tag, smem});
    P.qr.insert(P.qr.end(), qj.begin(), qj.end());
    qj.clear();
    qr_smem = 0;
    qr_tsqr = qr_tsqr_big = qr_stream_jobs = qr_stream_tall = qr_stream_trunc = 0;
  }
  void qapply(Ptr a, int lda, Ptr tau, Dim rows, Dim q, Ptr y, int ldy, Dim ncols, Ptr outp, int ldo) {
    qa.push_back(QApplyJob{a, tau, y, outp, lda, ldy, ldo, rows, q, ncols});
  }
  void flush_qapply(int tag) {
    if (qa.empty()) return;
    P.stages.push_back(Stage{ST_QAPPLY, (int64_t)P.qap.size(), (int)qa.size(), tag, 0});
    P.qap.insert(P.qap.end(), qa.begin(), qa.end());
    qa.clear();
  }
  void svd_size(int rows, int cols) {
    if (rows > SVD_MAXDIM || cols > SVD_MAXDIM) throw std::runtime_error("svd too large");
    sv_cost.push_back((double)rows * cols * cols);
    sv_need = std::max<int64_t>(sv_need, svd_colarr_doubles(cols) + (int64_t)(rows + 1) * cols);
    sv_maxr = std::max(sv_maxr, rows);
    sv_maxc = std::max(sv_maxc, cols);
    P.svd_maxrows = std::max(P.svd_maxrows, rows);
    P.svd_maxcols = std::max(P.svd_maxcols, cols);
  }
  // One stage: shared memory for its largest job (per-column arrays and
  // matrix), capped at SVD_SMEM_DOUBLES; the matrices of larger jobs run in
  // place in global memory, and the launch code runs the small jobs of a
  // mixed stage in small CTAs of their own.  (A one-CTA-per-SM launch for
  // the large jobs measured no faster: it serialises behind the small ones.)
  void flush_svd(int tag) {
    if (sv.empty()) return;
    const int smem = (int)(sizeof(double) * std::max<int64_t>(svd_colarr_doubles(sv_maxc),
                                                              std::min<int64_t>(sv_need, SVD_SMEM_DOUBLES)));
    largest_first(sv, sv_cost);
    P.stages.push_back(Stage{ST_SVD, (int64_t)P.svd.size(), (int)sv.size(), tag, smem, sv_maxc});
    P.svd.insert(P.svd.end(), sv.begin(), sv.end());
    sv.clear();
    sv_cost.clear();
    sv_maxr = sv_maxc = 1;
    sv_need = 0;
  }
  int nj_nmax = 1;  // largest n of the pending norm jobs
  void norm(Ptr src, int lds, DimV n, int norm_idx) {
    if (n.max > NORM_MAXN) throw std::runtime_error("norm matrix too large");
    nj.push_back(NormJob{src, lds, n.d(), norm_idx});
    nj_nmax = std::max(nj_nmax, n.max);
  }
  void flush_norm(int tag) {
    if (nj.empty()) return;
    P.stages.push_back(Stage{ST_NORM, (int64_t)P.norm.size(), (int)nj.size(), tag, 0, nj_nmax});
    P.norm.insert(P.norm.end(), nj.begin(), nj.end());
    nj.clear();
    nj_nmax = 1;
  }
  void scan(const std::vector<int>& in_slots, int out_first) {
    sc.push_back(ScanJob{(int)P.idx.size(), (int)in_slots.size(), out_first});
    P.idx.insert(P.idx.end(), in_slots.begin(), in_slots.end());
  }
  void flush_scan(int tag) {
    if (sc.empty()) return;
    P.stages.push_back(Stage{ST_SCAN, (int64_t)P.scan.size(), (int)sc.size(), tag, 0});
    P.scan.insert(P.scan.end(), sc.begin(), sc.end());
    sc.clear();
  }
  void flush_all(int tag) {
    flush_copy(tag);
    flush_gemm(tag);
  }

  // GEMM output with `rows` static rows split into tiles of GEMM_MAXTILE rows
  // (and static columns into tiles); emit(r0, c0) adds the terms of one tile.
  template <class F>
  void tiles(Ptr o, int ldo, int rows, DimV cols, int beta, F emit) {
    const int T = GEMM_MAXTILE;
    const bool dyn = cols.s >= 0;
    if (dyn && cols.max > T) throw std::runtime_error("dynamic gemm width above tile");
    for (int r0 = 0; r0 < rows; r0 += T) {
      const int nr = std::min(T, rows - r0);
      if (dyn) {
        out(padd(o, (int64_t)r0 * ldo), ldo, DC(nr), cols.d(), beta);
        emit(r0, nr, 0, cols.d());
      } else {
        for (int c0 = 0; c0 < cols.c; c0 += T) {
          const int nc = std::min(T, cols.c - c0);
          out(padd(o, (int64_t)r0 * ldo + c0), ldo, DC(nr), DC(nc), beta);
          emit(r0, nr, c0, DC(nc));
        }
      }
    }
  }
};

enum Tag : int {
  TAG_P = 1, TAG_PRE, TAG_SHAT, TAG_REC, TAG_OMEGA, TAG_AHAT, TAG_DEEP, TAG_EXPAND, TAG_DENSE,
  TAG_AGG, TAG_COND, TAG_ROWB, TAG_COLB, TAG_COUPLE
};

}  // namespace

// ============================================================== product ====
std::shared_ptr<Plan> make_product_plan(const MatDesc& X, const MatDesc& Y, const MulOptions& opt) {
  auto plan = std::make_shared<Plan>();
  Plan& P = *plan;
  Builder B(P);
  B.tagged = true;  // workspace placed by lifetime at the end (pack_workspace)
  B.fp32_contractions = opt.precision == 1;
  B.df_contractions = opt.precision == 2;
  B.tc5_contractions = opt.precision == 3;
  B.tc7_contractions = opt.precision == 4;
  const Tree& TI = *X.rows;
  const Tree& TJ = *X.cols;
  const Tree& TK = *Y.cols;
  const BlockTree& BX = *X.blocks;
  const BlockTree& BY = *Y.blocks;
  const int k = X.k;
  const int D = TJ.depth;
  if (TI.depth != D || TK.depth != D) throw std::runtime_error("trees of different depth");
  const int KP = opt.max_rank > 0 ? opt.max_rank : std::min(64, std::max(32, 2 * k));
  if (2 * KP > SVD_MAXDIM || KP > GEMM_MAXTILE) throw std::runtime_error("max_rank too large");
  const int AGGM = GEMM_MAXTILE;  // cap of agglomerated ranks
  int maxleaf = 0;
  for (int c = Tree::first(D); c < TI.ncl; ++c) maxleaf = std::max(maxleaf, TI.size[c]);
  for (int c = Tree::first(D); c < TK.ncl; ++c) maxleaf = std::max(maxleaf, TK.size[c]);
  if (maxleaf > SVD_MAXDIM) throw std::runtime_error("leaf too large");
  const int MB = std::max({2 * k, AGGM, maxleaf});  // max columns of a block factor
  const double theta = opt.theta;
  P.kpad = KP;

  auto XV = [&](int row) { return mref(PT(AR_X, X.off_V + (int64_t)row * k), k); };
  auto XW = [&](int row) { return mref(PT(AR_X, X.off_W + (int64_t)row * k), k); };
  auto YV = [&](int row) { return mref(PT(AR_Y, Y.off_V + (int64_t)row * k), k); };
  auto YW = [&](int row) { return mref(PT(AR_Y, Y.off_W + (int64_t)row * k), k); };
  auto XE = [&](int c, int t = 0) { return mref(PT(AR_X, X.off_E + (int64_t)c * k * k), k, t); };
  auto XF = [&](int c, int t = 0) { return mref(PT(AR_X, X.off_F + (int64_t)c * k * k), k, t); };
  auto YE = [&](int c, int t = 0) { return mref(PT(AR_Y, Y.off_E + (int64_t)c * k * k), k, t); };
  auto YF = [&](int c, int t = 0) { return mref(PT(AR_Y, Y.off_F + (int64_t)c * k * k), k, t); };
  auto XS = [&](int b, int t = 0) { return mref(PT(AR_X, X.off_S + (int64_t)BX.leafidx[b] * k * k), k, t); };
  auto YS = [&](int b, int t = 0) { return mref(PT(AR_Y, Y.off_S + (int64_t)BY.leafidx[b] * k * k), k, t); };
  auto XN = [&](int b, int t = 0) {
    return mref(PT(AR_X, X.off_N + BX.near_off[BX.leafidx[b]]), TJ.size[BX.s[b]], t);
  };
  auto YN = [&](int b, int t = 0) {
    return mref(PT(AR_Y, Y.off_N + BY.near_off[BY.leafidx[b]]), TK.size[BY.s[b]], t);
  };
  auto XVF = [&](int lvl, int row) { return mref(PT(AR_X, X.off_VF + ((int64_t)lvl * TI.n + row) * k), k); };
  auto YWF = [&](int lvl, int row) { return mref(PT(AR_Y, Y.off_WF + ((int64_t)lvl * TK.n + row) * k), k); };

    P.stats["ws_before_p1"] = B.ws;
// ------------------------------------------------ 1. basis products ----
  const int64_t offP = B.alloc((int64_t)TJ.ncl * k * k);
  auto Pm = [&](int s, int t = 0) { return mref(PT(AR_WS, offP + (int64_t)s * k * k), k, t); };
  for (int s = Tree::first(D); s < TJ.ncl; ++s) {
    B.out(Pm(s).p, k, DC(k), DC(k), 0);
    B.term2(mref(XW(TJ.off[s]).p, k, 1), YV(TJ.off[s]), DC(TJ.size[s]));
  }
  B.flush_gemm(TAG_P);
  for (int l = D - 1; l >= 0; --l) {
    for (int s = Tree::first(l); s < Tree::first(l + 1); ++s) {
      B.out(Pm(s).p, k, DC(k), DC(k), 0);
      for (int i = 0; i < 2; ++i) {
        const int c = Tree::child(s, i);
        B.term3(XF(c, 1), Pm(c), YE(c), DC(k), DC(k));
      }
    }
    B.flush_gemm(TAG_P);
  }

  P.stats["ws_before_p2"] = B.ws;
  // ------------------------------------- 2. product tree (symbolic) ----
  std::vector<std::pair<int, int>> case1, case2, case3;
  std::unordered_set<int64_t> hasP;
  {
    std::vector<std::pair<int, int>> st{{0, 0}};
    while (!st.empty()) {
      auto [xb, yb] = st.back();
      st.pop_back();
      if (BY.is_leaf(yb) && BY.is_adm(yb)) {
        case1.push_back({xb, yb});
      } else if (BX.is_leaf(xb) && BX.is_adm(xb)) {
        case2.push_back({xb, yb});
      } else if (BX.is_leaf(xb) || BY.is_leaf(yb)) {
        case3.push_back({xb, yb});
      } else {
        hasP.insert(key2(BX.t[xb], BY.s[yb]));
        for (int i = 1; i >= 0; --i)
          for (int j = 1; j >= 0; --j)
            for (int l = 1; l >= 0; --l) st.push_back({BX.child(xb, i, j), BY.child(yb, j, l)});
      }
    }
  }
  P.stats["case1"] = case1.size();
  P.stats["case2"] = case2.size();
  P.stats["case3"] = case3.size();
  P.stats["case4"] = hasP.size();

  // case 1: walk the X subtree below (t,s); contributions keyed by (u, r)
  struct Contrib {
    int leaf;  // X (case 1) or Y (case 2) leaf block
    int root;  // Y (case 1) or X (case 2) admissible leaf providing S
  };
  std::map<int64_t, std::vector<Contrib>> recA, recAn, recB, recBn;
  std::set<std::pair<int, int>> needS1, needS2;  // (root block, middle cluster)
  std::set<int> useQx, useNx, useQy, useNy;
  auto need_path = [&](std::set<std::pair<int, int>>& need, int root, int top, int s1) {
    int c = s1;
    while (true) {
      if (!need.insert({root, c}).second) break;
      if (c == top) break;
      c = Tree::parent(c);
    }
  };
  for (auto [xb, yb] : case1) {
    const int r = BY.s[yb], s = BY.t[yb];
    std::vector<int> st{xb};
    while (!st.empty()) {
      const int x = st.back();
      st.pop_back();
      if (!BX.is_leaf(x)) {
        for (int i = 3; i >= 0; --i) st.push_back(BX.child0[x] + i);
        continue;
      }
      const int u = BX.t[x];
      need_path(needS1, yb, s, BX.s[x]);
      if (BX.is_adm(x)) {
        recA[key2(u, r)].push_back({x, yb});
        useQx.insert(x);
      } else {
        recAn[key2(u, r)].push_back({x, yb});
        useNx.insert(x);
      }
    }
  }
  for (auto [xb, yb] : case2) {
    const int t = BX.t[xb], s = BX.s[xb];
    std::vector<int> st{yb};
    while (!st.empty()) {
      const int y = st.back();
      st.pop_back();
      if (!BY.is_leaf(y)) {
        for (int i = 3; i >= 0; --i) st.push_back(BY.child0[y] + i);
        continue;
      }
      const int v = BY.s[y];
      need_path(needS2, xb, s, BY.t[y]);
      if (BY.is_adm(y)) {
        recB[key2(v, t)].push_back({y, xb});
        useQy.insert(y);
      } else {
        recBn[key2(v, t)].push_back({y, xb});
        useNy.insert(y);
      }
    }
  }

  P.stats["ws_before_p3"] = B.ws;
  // ---------------------------- 3. precomputed leaf products, S-hat ----
  std::unordered_map<int, int64_t> offQx, offNx, offQy, offNy;
  for (int x : useQx) {
    offQx[x] = B.alloc((int64_t)k * k);
    B.out(PT(AR_WS, offQx[x]), k, DC(k), DC(k), 0);
    B.term2(XS(x), Pm(BX.s[x]), DC(k));
  }
  for (int y : useQy) {
    offQy[y] = B.alloc((int64_t)k * k);
    B.out(PT(AR_WS, offQy[y]), k, DC(k), DC(k), 0);
    B.term2(YS(y, 1), Pm(BY.t[y], 1), DC(k));
  }
  for (int x : useNx) {
    const int t1 = BX.t[x], s1 = BX.s[x];
    offNx[x] = B.alloc((int64_t)TI.size[t1] * k);
    B.tiles(PT(AR_WS, offNx[x]), k, TI.size[t1], dv(k), 0, [&](int r0, int, int c0, Dim) {
      B.term2(rows_of(XN(x), r0), mref(padd(YV(TJ.off[s1]).p, c0), k), DC(TJ.size[s1]));
    });
  }
  for (int y : useNy) {
    const int s1 = BY.t[y], r1 = BY.s[y];
    offNy[y] = B.alloc((int64_t)TK.size[r1] * k);
    B.tiles(PT(AR_WS, offNy[y]), k, TK.size[r1], dv(k), 0, [&](int r0, int, int c0, Dim) {
      MRef a = YN(y, 1);
      a.p = padd(a.p, r0);  // transposed: row offset r0 of N^T = column offset r0 of N
      B.term2(a, mref(padd(XW(TJ.off[s1]).p, c0), k), DC(TJ.size[s1]));
    });
  }
  B.flush_gemm(TAG_PRE);
  // S-hat(yb, s1) = E_{Y,s1} S-hat(yb, parent s1), root S_{Y,yb};
  // S-hat'(xb, s1) = F_{X,s1} S-hat'(xb, parent s1), root S_{X,xb}^*.
  std::map<std::pair<int, int>, MRef> S1, S2;
  for (auto& pr : needS1)
    if (pr.second == BY.t[pr.first]) S1[pr] = YS(pr.first);
  for (auto& pr : needS2)
    if (pr.second == BX.s[pr.first]) S2[pr] = XS(pr.first, 1);
  for (int l = 1; l <= D; ++l) {
    for (auto& pr : needS1) {
      if (TJ.level[pr.second] != l || S1.count(pr)) continue;
      const int64_t o = B.alloc((int64_t)k * k);
      B.out(PT(AR_WS, o), k, DC(k), DC(k), 0);
      B.term2(YE(pr.second), S1.at({pr.first, Tree::parent(pr.second)}), DC(k));
      S1[pr] = mref(PT(AR_WS, o), k);
    }
    for (auto& pr : needS2) {
      if (TJ.level[pr.second] != l || S2.count(pr)) continue;
      const int64_t o = B.alloc((int64_t)k * k);
      B.out(PT(AR_WS, o), k, DC(k), DC(k), 0);
      B.term2(XF(pr.second), S2.at({pr.first, Tree::parent(pr.second)}), DC(k));
      S2[pr] = mref(PT(AR_WS, o), k);
    }
    B.flush_gemm(TAG_SHAT);
  }

  P.stats["ws_before_p4"] = B.ws;
  // ------------------------------------------------------- 4. records ----
  std::unordered_map<int64_t, MRef> RA, RAn, RB, RBn;
  for (auto& [key, list] : recA) {
    const int64_t o = B.alloc((int64_t)k * k);
    B.out(PT(AR_WS, o), k, DC(k), DC(k), 0);
    for (auto& c : list) B.term2(mref(PT(AR_WS, offQx[c.leaf]), k), S1.at({c.root, BX.s[c.leaf]}), DC(k));
    RA[key] = mref(PT(AR_WS, o), k);
  }
  for (auto& [key, list] : recB) {
    const int64_t o = B.alloc((int64_t)k * k);
    B.out(PT(AR_WS, o), k, DC(k), DC(k), 0);
    for (auto& c : list) B.term2(mref(PT(AR_WS, offQy[c.leaf]), k), S2.at({c.root, BY.t[c.leaf]}), DC(k));
    RB[key] = mref(PT(AR_WS, o), k);
  }
  for (auto& [key, list] : recAn) {
    const int u = (int)(key >> 32);
    const int64_t o = B.alloc((int64_t)TI.size[u] * k);
    B.tiles(PT(AR_WS, o), k, TI.size[u], dv(k), 0, [&](int r0, int, int, Dim) {
      for (auto& c : list)
        B.term2(rows_of(mref(PT(AR_WS, offNx[c.leaf]), k), r0), S1.at({c.root, BX.s[c.leaf]}), DC(k));
    });
    RAn[key] = mref(PT(AR_WS, o), k);
  }
  for (auto& [key, list] : recBn) {
    const int v = (int)(key >> 32);
    const int64_t o = B.alloc((int64_t)TK.size[v] * k);
    B.tiles(PT(AR_WS, o), k, TK.size[v], dv(k), 0, [&](int r0, int, int, Dim) {
      for (auto& c : list)
        B.term2(rows_of(mref(PT(AR_WS, offNy[c.leaf]), k), r0), S2.at({c.root, BY.t[c.leaf]}), DC(k));
    });
    RBn[key] = mref(PT(AR_WS, o), k);
  }
  B.flush_gemm(TAG_REC);
  P.stats["recA"] = RA.size() + RAn.size();
  P.stats["recB"] = RB.size() + RBn.size();

  P.stats["ws_before_p5"] = B.ws;
  // ------------------------------------------- 5. target / visited tree ----
  P.cblocks = std::make_shared<BlockTree>();
  BlockTree& BC = *P.cblocks;
  build_block_tree(TI, TK, opt.eta, BC);
  enum Kind { VK_INNER, VK_SU, VK_AGGROOT, VK_AGGINNER, VK_CELL, VK_OUT };
  struct VNode {
    int t, r, parent, level, kind, cb;  // cb: target block (or -1 inside an agglomeration)
    int agg = -1;                       // agglomeration index for AGGROOT/CELL
    bool dense = false;                 // leaf-level node with dense part (case 3)
    MRef ahat{NONE(), 0, 0}, bhat{NONE(), 0, 0};
    bool has_a = false, has_b = false;
    int64_t dense_off = -1;             // G buffer
    int dense_ar = AR_WS;
    int dense_ld = 0;
    MRef L{NONE(), 0, 0}, R{NONE(), 0, 0};  // explicit factors
    MRef A{NONE(), 0, 0}, Bm{NONE(), 0, 0};  // explicit A_tr, B_tr
  };
  std::vector<VNode> V;
  std::unordered_map<int64_t, int> vindex;
  struct Agg {
    int root;
    int d;
    std::vector<int> cells;  // row-major grid n x n
  };
  std::vector<Agg> aggs;
  std::function<int(int, int)> induced_depth = [&](int t, int r) -> int {
    if (!hasP.count(key2(t, r))) return 0;
    int m = 0;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) m = std::max(m, induced_depth(Tree::child(t, i), Tree::child(r, j)));
    return 1 + m;
  };
  auto addv = [&](int t, int r, int parent, int kind, int cb) {
    VNode n{};
    n.t = t;
    n.r = r;
    n.parent = parent;
    n.level = TI.level[t];
    n.kind = kind;
    n.cb = cb;
    V.push_back(n);
    vindex[key2(t, r)] = (int)V.size() - 1;
    return (int)V.size() - 1;
  };
  {
    std::vector<std::pair<int, int>> st{{0, -1}};  // (target block, parent vnode)
    while (!st.empty()) {
      auto [cb, par] = st.back();
      st.pop_back();
      const int t = BC.t[cb], r = BC.s[cb];
      if (!BC.is_leaf(cb)) {
        const int id = addv(t, r, par, VK_INNER, cb);
        for (int i = 3; i >= 0; --i) st.push_back({BC.child0[cb] + i, id});
      } else if (BC.is_adm(cb)) {
        if (hasP.count(key2(t, r))) {
          const int d = induced_depth(t, r);
          const int id = addv(t, r, par, VK_AGGROOT, cb);
          Agg ag{id, d, {}};
          const int n = 1 << d;
          ag.cells.assign((size_t)n * n, -1);
          // complete quad tree of depth d below (t,r)
          std::vector<std::tuple<int, int, int, int, int, int>> q{{t, r, id, 0, 0, 0}};
          while (!q.empty()) {
            auto [tt, rr, pid, dep, ci, cj] = q.back();
            q.pop_back();
            for (int i = 0; i < 2; ++i)
              for (int j = 0; j < 2; ++j) {
                const int tc = Tree::child(tt, i), rc = Tree::child(rr, j);
                const bool cell = dep + 1 == d;
                const int cid = addv(tc, rc, pid, cell ? VK_CELL : VK_AGGINNER, -1);
                const int ni = ci * 2 + i, nj = cj * 2 + j;
                if (cell) {
                  ag.cells[(size_t)ni * n + nj] = cid;
                  V[cid].agg = (int)aggs.size();
                } else {
                  q.push_back({tc, rc, cid, dep + 1, ni, nj});
                }
              }
          }
          V[id].agg = (int)aggs.size();
          aggs.push_back(ag);
        } else {
          addv(t, r, par, VK_SU, cb);
        }
      } else {
        addv(t, r, par, VK_OUT, cb);
      }
    }
  }
  P.nagg = (int)aggs.size();
  P.stats["visited"] = V.size();
  P.stats["agglomerated"] = aggs.size();

  // dense leaf-level nodes (case 3 products)
  std::map<int, std::vector<std::pair<int, int>>> dense_terms;  // vnode -> (xb, yb)
  for (auto [xb, yb] : case3) {
    const int t = BX.t[xb], r = BY.s[yb];
    auto it = vindex.find(key2(t, r));
    if (it == vindex.end()) throw std::runtime_error("case-3 product outside the visited tree");
    dense_terms[it->second].push_back({xb, yb});
    V[it->second].dense = true;
  }

  P.stats["ws_before_p6"] = B.ws;
  // ------------------------------------------------ 6. Omega pushes ----
  // Omega(u, r) = rec(u, r) + Omega(u, parent r) F_{Y,r}^*  (A side, column tree T_K)
  // OmegaB(v, t) = recB(v, t) + OmegaB(v, parent t) E_{X,t}^*  (B side, row tree T_I)
  struct OmegaSide {
    std::unordered_map<int64_t, MRef>* rec;
    std::unordered_map<int64_t, std::pair<bool, MRef>> memo;
    std::vector<std::vector<std::tuple<int64_t, MRef, MRef, int, int>>> jobs;  // per level
    bool tall;        // nearfield form (|u| x k)
    const Tree* node_tree;
    const Tree* col_tree;
    int transfer_ar;  // arena of the column-tree transfers
    int64_t transfer_off;
  };
  auto make_side = [&](std::unordered_map<int64_t, MRef>* rec, bool tall, const Tree* nt, const Tree* ct, int ar,
                       int64_t toff) {
    OmegaSide s;
    s.rec = rec;
    s.tall = tall;
    s.node_tree = nt;
    s.col_tree = ct;
    s.transfer_ar = ar;
    s.transfer_off = toff;
    s.jobs.resize(D + 1);
    return s;
  };
  OmegaSide OA = make_side(&RA, false, &TI, &TK, AR_Y, Y.off_F);
  OmegaSide OAn = make_side(&RAn, true, &TI, &TK, AR_Y, Y.off_F);
  OmegaSide OB = make_side(&RB, false, &TK, &TI, AR_X, X.off_E);
  OmegaSide OBn = make_side(&RBn, true, &TK, &TI, AR_X, X.off_E);
  std::function<std::pair<bool, MRef>(OmegaSide&, int, int)> omega = [&](OmegaSide& S, int u,
                                                                          int r) -> std::pair<bool, MRef> {
    const int64_t kk = key2(u, r);
    auto it = S.memo.find(kk);
    if (it != S.memo.end()) return it->second;
    std::pair<bool, MRef> prev{false, MRef{NONE(), 0, 0}};
    if (r > 0) prev = omega(S, u, Tree::parent(r));
    auto rit = S.rec->find(kk);
    std::pair<bool, MRef> res{false, MRef{NONE(), 0, 0}};
    if (!prev.first && rit != S.rec->end()) {
      res = {true, rit->second};
    } else if (prev.first) {
      const int rows = S.tall ? S.node_tree->size[u] : k;
      const int64_t o = B.alloc((int64_t)rows * k);
      res = {true, mref(PT(AR_WS, o), k)};
      MRef recm = rit != S.rec->end() ? rit->second : MRef{NONE(), 0, 0};
      S.jobs[S.col_tree->level[r]].push_back({o, prev.second, recm, rows, r});
    }
    S.memo[kk] = res;
    return res;
  };
  // demands
  for (size_t q = 0; q < V.size(); ++q) {
    const VNode& n = V[q];
    if (n.parent >= 0) {
      omega(OA, n.t, n.r);
      omega(OB, n.r, n.t);
    }
  }
  auto is_terminal = [&](const VNode& n) {
    return n.kind == VK_SU || n.kind == VK_CELL || n.kind == VK_OUT;
  };
  auto desc_of = [&](const Tree& T, int c, std::vector<int>& out) {
    out.clear();
    std::vector<int> st{c};
    while (!st.empty()) {
      int x = st.back();
      st.pop_back();
      out.push_back(x);
      if (!T.leaf(x)) {
        st.push_back(Tree::child(x, 1));
        st.push_back(Tree::child(x, 0));
      }
    }
  };
  std::vector<int> tmp;
  for (size_t q = 0; q < V.size(); ++q) {
    const VNode& n = V[q];
    if (!is_terminal(n)) continue;
    desc_of(TI, n.t, tmp);
    for (int u : tmp) {
      if (u != n.t) omega(OA, u, n.r);
      if (TI.leaf(u)) omega(OAn, u, n.r);
    }
    desc_of(TK, n.r, tmp);
    for (int v : tmp) {
      if (v != n.r) omega(OB, v, n.t);
      if (TK.leaf(v)) omega(OBn, v, n.t);
    }
  }
  for (int l = 1; l <= D; ++l) {
    for (OmegaSide* S : {&OA, &OAn, &OB, &OBn}) {
      for (auto& [o, prev, recm, rows, r] : S->jobs[l]) {
        B.tiles(PT(AR_WS, o), k, rows, dv(k), 0, [&](int r0, int, int, Dim) {
          B.term2(rows_of(prev, r0), mref(PT(S->transfer_ar, S->transfer_off + (int64_t)r * k * k), k, 1), DC(k));
          if (recm.p.arena != AR_NONE) B.add(rows_of(recm, r0));
        });
      }
    }
    B.flush_gemm(TAG_OMEGA);
  }

  P.stats["ws_before_p7"] = B.ws;
  // ---------------------------------------- 7. root coefficient pushes ----
  // ahat_q = E_{X,t} ahat_parent F_{Y,r}^* + Omega(t, r);  bhat mirror.
  {
    std::vector<std::vector<int>> bylevel(D + 1);
    for (size_t q = 0; q < V.size(); ++q) bylevel[V[q].level].push_back((int)q);
    for (int l = 1; l <= D; ++l) {
      for (int q : bylevel[l]) {
        VNode& n = V[q];
        const VNode& p = V[n.parent];
        auto om = omega(OA, n.t, n.r);
        if (p.has_a || om.first) {
          const int64_t o = B.alloc((int64_t)k * k);
          B.out(PT(AR_WS, o), k, DC(k), DC(k), 0);
          if (p.has_a) B.term3(XE(n.t), p.ahat, YF(n.r, 1), DC(k), DC(k));
          if (om.first) B.add(om.second);
          n.ahat = mref(PT(AR_WS, o), k);
          n.has_a = true;
        }
        auto omb = omega(OB, n.r, n.t);
        if (p.has_b || omb.first) {
          const int64_t o = B.alloc((int64_t)k * k);
          B.out(PT(AR_WS, o), k, DC(k), DC(k), 0);
          if (p.has_b) B.term3(YF(n.r), p.bhat, XE(n.t, 1), DC(k), DC(k));
          if (omb.first) B.add(omb.second);
          n.bhat = mref(PT(AR_WS, o), k);
          n.has_b = true;
        }
      }
      B.flush_gemm(TAG_AHAT);
    }
  }

  P.stats["ws_before_p8"] = B.ws;
  // ------------------------- 8. deep pushes and explicit A_tr, B_tr -----
  // Buffers: semi-uniform terminals get L = [A, V_{X,t}] (|t| x 2k) and
  // R = [W_{Y,r}, B] (|r| x 2k); dense terminals get A (|t| x k), B (|r| x k).
  for (size_t q = 0; q < V.size(); ++q) {
    VNode& n = V[q];
    if (!is_terminal(n)) continue;
    const int nt = TI.size[n.t], nr = TK.size[n.r];
    const bool dense = n.dense || n.kind == VK_OUT;
    if (!dense) {
      const int64_t oL = B.falloc((int64_t)nt * 2 * k), oR = B.falloc((int64_t)nr * 2 * k);
      n.L = mref(PT(AR_F, oL), 2 * k);
      n.R = mref(PT(AR_F, oR), 2 * k);
      n.A = mref(PT(AR_F, oL), 2 * k);
      n.Bm = mref(PT(AR_F, oR + k), 2 * k);
      B.copy(XVF(n.level, TI.off[n.t]).p, k, padd(n.L.p, k), 2 * k, DC(nt), DC(k), 0);
      B.copy(YWF(n.level, TK.off[n.r]).p, k, n.R.p, 2 * k, DC(nr), DC(k), 0);
    } else {
      n.A = mref(PT(AR_F, B.falloc((int64_t)nt * k)), k);
      n.Bm = mref(PT(AR_F, B.falloc((int64_t)nr * k)), k);
    }
  }
  B.flush_copy(TAG_EXPAND);
  {
    // per terminal, coefficient buffers a_q(u) for u in desc(t)
    struct DeepJob {
      int q;
      int u;
      bool side_b;
    };
    std::vector<std::unordered_map<int, std::pair<bool, MRef>>> acoef(V.size()), bcoef(V.size());
    for (size_t q = 0; q < V.size(); ++q) {
      if (!is_terminal(V[q])) continue;
      acoef[q][V[q].t] = {V[q].has_a, V[q].ahat};
      bcoef[q][V[q].r] = {V[q].has_b, V[q].bhat};
    }
    for (int l = 1; l <= D; ++l) {
      for (size_t q = 0; q < V.size(); ++q) {
        VNode& n = V[q];
        if (!is_terminal(n) || n.level >= l) continue;
        for (int u = Tree::first(l); u < Tree::first(l + 1); ++u) {
          // u in desc(t)?
          int a = u;
          while (TI.level[a] > n.level) a = Tree::parent(a);
          if (a != n.t) continue;
          auto pr = acoef[q].at(Tree::parent(u));
          auto om = omega(OA, u, n.r);
          if (pr.first || om.first) {
            const int64_t o = B.alloc((int64_t)k * k);
            B.out(PT(AR_WS, o), k, DC(k), DC(k), 0);
            if (pr.first) B.term2(XE(u), pr.second, DC(k));
            if (om.first) B.add(om.second);
            acoef[q][u] = {true, mref(PT(AR_WS, o), k)};
          } else {
            acoef[q][u] = {false, MRef{NONE(), 0, 0}};
          }
        }
        for (int v = Tree::first(l); v < Tree::first(l + 1); ++v) {
          int a = v;
          while (TK.level[a] > n.level) a = Tree::parent(a);
          if (a != n.r) continue;
          auto pr = bcoef[q].at(Tree::parent(v));
          auto om = omega(OB, v, n.t);
          if (pr.first || om.first) {
            const int64_t o = B.alloc((int64_t)k * k);
            B.out(PT(AR_WS, o), k, DC(k), DC(k), 0);
            if (pr.first) B.term2(YF(v), pr.second, DC(k));
            if (om.first) B.add(om.second);
            bcoef[q][v] = {true, mref(PT(AR_WS, o), k)};
          } else {
            bcoef[q][v] = {false, MRef{NONE(), 0, 0}};
          }
        }
      }
      B.flush_gemm(TAG_DEEP);
    }
    // leaf expansion: A[rows u] = V_{X,u} a_q(u) + OmegaN(u, r)
    for (size_t q = 0; q < V.size(); ++q) {
      VNode& n = V[q];
      if (!is_terminal(n)) continue;
      for (auto& [u, pr] : acoef[q]) {
        if (!TI.leaf(u)) continue;
        auto om = omega(OAn, u, n.r);
        const int64_t r0u = TI.off[u] - TI.off[n.t];
        B.tiles(padd(n.A.p, r0u * n.A.ld), n.A.ld, TI.size[u], dv(k), 0, [&](int r0, int, int, Dim) {
          if (pr.first) B.term2(XV(TI.off[u] + r0), pr.second, DC(k));
          if (om.first) B.add(rows_of(om.second, r0));
        });
      }
      for (auto& [v, pr] : bcoef[q]) {
        if (!TK.leaf(v)) continue;
        auto om = omega(OBn, v, n.t);
        const int64_t r0v = TK.off[v] - TK.off[n.r];
        B.tiles(padd(n.Bm.p, r0v * n.Bm.ld), n.Bm.ld, TK.size[v], dv(k), 0, [&](int r0, int, int, Dim) {
          if (pr.first) B.term2(YW(TK.off[v] + r0), pr.second, DC(k));
          if (om.first) B.add(rows_of(om.second, r0));
        });
      }
    }
    B.flush_gemm(TAG_EXPAND);
  }

  // Everything the accumulation phases left in the workspace (basis products,
  // S-hat descents, records, Omega/root/deep pushes) is dead now: the
  // terminal factors in AR_F carry the result on.  The recompression phases
  // reuse the workspace from its start.
  P.stats["ws_accumulation"] = B.ws_peak;
  B.ws = 0;
  P.stats["ws_before_p9"] = B.ws;
  // --------------------------------------------- 9. dense terminals ----
  // G = sum X|ts Y|sr (case 3) + A W_{Y,r}^* + V_{X,t} B^*
  // (inadmissible target leaves are written straight into C's nearfield).
  P.c_off_V = 0;
  P.c_off_E = P.c_off_V + (int64_t)TI.n * KP;
  P.c_off_W = P.c_off_E + (int64_t)TI.ncl * KP * KP;
  P.c_off_F = P.c_off_W + (int64_t)TK.n * KP;
  P.c_off_S = P.c_off_F + (int64_t)TK.ncl * KP * KP;
  P.c_off_N = P.c_off_S + (int64_t)BC.adm_list.size() * KP * KP;
  P.c_len = P.c_off_N + BC.near_total;
  for (size_t q = 0; q < V.size(); ++q) {
    VNode& n = V[q];
    if (!(n.dense || n.kind == VK_OUT)) continue;
    const int nt = TI.size[n.t], nr = TK.size[n.r];
    if (n.kind == VK_OUT) {
      n.dense_ar = AR_C;
      n.dense_off = P.c_off_N + BC.near_off[BC.leafidx[n.cb]];
    } else {
      n.dense_ar = AR_WS;
      n.dense_off = B.alloc((int64_t)nt * nr);
    }
    n.dense_ld = nr;
    auto it = dense_terms.find((int)q);
    if (it != dense_terms.end()) {
      B.tiles(PT(n.dense_ar, n.dense_off), nr, nt, dv(nr), 0, [&](int r0, int, int c0, Dim) {
        for (auto [xb, yb] : it->second) {
          MRef yn = YN(yb);
          yn.p = padd(yn.p, c0);
          B.term2(rows_of(XN(xb), r0), yn, DC(TJ.size[BX.s[xb]]));
        }
      });
    }
  }
  B.flush_gemm(TAG_DENSE);
  for (size_t q = 0; q < V.size(); ++q) {
    VNode& n = V[q];
    if (!(n.dense || n.kind == VK_OUT)) continue;
    const int nt = TI.size[n.t], nr = TK.size[n.r];
    const int beta = dense_terms.count((int)q) ? 1 : 0;
    B.tiles(PT(n.dense_ar, n.dense_off), nr, nt, dv(nr), beta, [&](int r0, int, int c0, Dim) {
      B.term2(rows_of(n.A, r0), mref(padd(YW(TK.off[n.r]).p, (int64_t)c0 * k), k, 1), DC(k));
      B.term2(XV(TI.off[n.t] + r0), mref(padd(n.Bm.p, (int64_t)c0 * n.Bm.ld), n.Bm.ld, 1), DC(k));
    });
    if (n.kind != VK_OUT) {  // dense factor (G, I)
      n.L = mref(PT(AR_WS, n.dense_off), nr);
    }
  }
  B.flush_gemm(TAG_DENSE);
  // identity matrix constant for dense factors
  const int64_t offI = 0;
  P.konst.assign((size_t)maxleaf * maxleaf, 0.0);
  for (int i = 0; i < maxleaf; ++i) P.konst[(size_t)i * maxleaf + i] = 1.0;
  for (auto& n : V)
    if (n.dense && n.kind != VK_OUT) n.R = mref(PT(AR_K, offI), maxleaf);

  P.stats["ws_before_p10"] = B.ws;
  // ------------------------------------------- 10. agglomeration ----
  struct Factor {
    MRef L, R;
    DimV m;
    int rows_t, rows_r;
  };
  auto cell_factor = [&](const VNode& n) {
    Factor f;
    f.L = n.L;
    f.R = n.R;
    f.rows_t = TI.size[n.t];
    f.rows_r = TK.size[n.r];
    f.m = n.dense ? dv(f.rows_r) : dv(2 * k);
    return f;
  };
  std::vector<Factor> agg_result(aggs.size());
  // Norm slot of each agglomerated block, written by the SVD of its last merge:
  // the merged block is (Q_c Y_k') Sigma_k' (Q U_k')^T with orthonormal outer
  // factors, so ||G_b||_2 is that SVD's largest singular value (-1: no merge,
  // the condensation computes the norm).
  std::vector<int> agg_nidx(aggs.size(), -1);
  if (!aggs.empty()) {
    // state: per agglomeration, per grid row the accumulated factor
    std::vector<std::vector<Factor>> rowf(aggs.size());
    std::vector<Factor> colf(aggs.size());
    int max_steps = 0;
    for (auto& a : aggs) max_steps = std::max(max_steps, 2 * ((1 << a.d) - 1));
    const int AGGC = 2 * std::max(MB, AGGM);  // widest merged factor pair
    for (size_t a = 0; a < aggs.size(); ++a) {
      const int n = 1 << aggs[a].d;
      for (int i = 0; i < n; ++i) rowf[a].push_back(cell_factor(V[aggs[a].cells[(size_t)i * n]]));
    }
    for (int step = 0; step < max_steps; ++step) {
      struct MergeJob {
        Factor f1, f2;
        bool vertical;
        int agg, row;
        double rel;  // relative tolerance multiplier of eps_c
      };
      std::vector<MergeJob> jobs;
      for (size_t a = 0; a < aggs.size(); ++a) {
        const int n = 1 << aggs[a].d;
        const double rel = 1.0 / (2.0 * n * n);
        if (step < n - 1) {  // column merge j = step+1 in every row
          for (int i = 0; i < n; ++i)
            jobs.push_back({rowf[a][i], cell_factor(V[aggs[a].cells[(size_t)i * n + step + 1]]), false, (int)a, i,
                            rel});
        } else if (step < 2 * (n - 1)) {  // row merge i = step-(n-1)+1
          const int i = step - (n - 1) + 1;
          const Factor f1 = (i == 1) ? rowf[a][0] : colf[a];
          jobs.push_back({f1, rowf[a][i], true, (int)a, i, rel});
        }
      }
      if (jobs.empty()) continue;
      // outputs first (persistent), then scratch (reused by the next step)
      std::vector<Factor> outs(jobs.size());
      for (size_t j = 0; j < jobs.size(); ++j) {
        const MergeJob& J = jobs[j];
        Factor o;
        o.rows_t = J.vertical ? J.f1.rows_t + J.f2.rows_t : J.f1.rows_t;
        o.rows_r = J.vertical ? J.f1.rows_r : J.f1.rows_r + J.f2.rows_r;
        o.L = mref(PT(AR_WS, B.alloc((int64_t)o.rows_t * AGGM)), AGGM);
        o.R = mref(PT(AR_WS, B.alloc((int64_t)o.rows_r * AGGM)), AGGM);
        o.m = dvs(B.slot(0), AGGM);
        outs[j] = o;
      }
      const int64_t mark = B.ws;
      struct Scr {
        int64_t W1, W2, tau1, tau2, rho1, rho2, Gc, Wc, tauc, rhoc, U, sig, piv;
        bool two_step;            // SVD through a second QR (M may not fit the SVD's shared memory)
        int64_t tau2c, R2, Y;     // its reflector scalars, triangle and small singular vectors
        int rslot;                // rows of rho_c kept above the noise floor (slot)
        int qc_max;
      };
      std::vector<Scr> scr(jobs.size());
      for (size_t j = 0; j < jobs.size(); ++j) {
        const MergeJob& J = jobs[j];
        Scr& s = scr[j];
        const int m1 = J.f1.m.max, m2 = J.f2.m.max;
        if (!J.vertical) {
          s.W1 = B.alloc((int64_t)J.f1.rows_r * m1);
          s.W2 = B.alloc((int64_t)J.f2.rows_r * m2);
          s.tau1 = B.alloc(m1);
          s.tau2 = B.alloc(m2);
          s.rho1 = B.alloc((int64_t)m1 * m1);
          s.rho2 = B.alloc((int64_t)m2 * m2);
          // W = R^T (column-major R)
          B.copy(J.f1.R.p, J.f1.R.ld, PT(AR_WS, s.W1), J.f1.rows_r, J.f1.m.d(), DC(J.f1.rows_r), 1);
          B.copy(J.f2.R.p, J.f2.R.ld, PT(AR_WS, s.W2), J.f2.rows_r, J.f2.m.d(), DC(J.f2.rows_r), 1);
          B.qr(PT(AR_WS, s.W1), J.f1.rows_r, DC(J.f1.rows_r), J.f1.m.d(), PT(AR_WS, s.tau1), PT(AR_WS, s.rho1), m1, 1,
               J.f1.rows_r, m1);
          B.qr(PT(AR_WS, s.W2), J.f2.rows_r, DC(J.f2.rows_r), J.f2.m.d(), PT(AR_WS, s.tau2), PT(AR_WS, s.rho2), m2, 1,
               J.f2.rows_r, m2);
        } else {
          s.W1 = B.alloc((int64_t)J.f1.rows_r * (m1 + m2));
          s.tau1 = B.alloc(m1 + m2);
          s.rho1 = B.alloc((int64_t)(m1 + m2) * (m1 + m2));
          B.copy(J.f1.R.p, J.f1.R.ld, PT(AR_WS, s.W1), J.f1.rows_r, J.f1.m.d(), DC(J.f1.rows_r), 1);
          B.copy(J.f2.R.p, J.f2.R.ld, pdyn(PT(AR_WS, s.W1 + (int64_t)J.f1.m.c * J.f1.rows_r), J.f1.m.s, J.f1.rows_r),
                 J.f1.rows_r, J.f2.m.d(), DC(J.f1.rows_r), 1);
          const Dim mm = merged_width(J.f1.m, J.f2.m);
          B.qr(PT(AR_WS, s.W1), J.f1.rows_r, DC(J.f1.rows_r), mm, PT(AR_WS, s.tau1), PT(AR_WS, s.rho1), m1 + m2, 1,
               J.f1.rows_r, m1 + m2);
        }
        s.Gc = B.alloc((int64_t)(J.vertical ? J.f1.rows_t + J.f2.rows_t : J.f1.rows_t) * AGGC);
        s.Wc = B.alloc((int64_t)(J.vertical ? J.f1.rows_t + J.f2.rows_t : J.f1.rows_t) * (m1 + m2));
        s.tauc = B.alloc(m1 + m2);
        s.rhoc = B.alloc((int64_t)(m1 + m2) * AGGC);
        s.U = B.alloc((int64_t)(m1 + m2) * AGGC);
        s.sig = B.alloc(m1 + m2);
        s.piv = B.alloc((m1 + m2 + 1) / 2);  // int32 pivot order of the condensed QR
        {
          // The pivoted QR of Gc stops at the SVD's noise floor: rho_c keeps
          // its first r rows, r at run time.  M = rho_c^T is (m1+m2) x r; when
          // it may not fit the SVD's shared memory, the SVD runs on the
          // triangle R2 of M = Q2 R2 instead: same Gram matrix, hence the same
          // rotations and singular values, with r-long columns; U = Q2 Y
          // afterwards
          const int gr = J.vertical ? J.f1.rows_t + J.f2.rows_t : J.f1.rows_t;
          const int qmax = std::min(m1 + m2, gr);
          s.rslot = B.slot(0);
          s.two_step = svd_colarr_doubles(qmax) + (int64_t)(m1 + m2 + 1) * qmax > SVD_SMEM_DOUBLES;
          if (s.two_step) {
            ++P.stats["agg_two_step"];
            s.tau2c = B.alloc(qmax);
            s.R2 = B.alloc((int64_t)qmax * qmax);
            s.Y = B.alloc((int64_t)qmax * AGGC);
          }
        }
        if (m1 + m2 > AGGC) throw std::runtime_error("agglomeration width");
      }
      B.flush_copy(TAG_AGG);
      B.flush_qr(TAG_AGG);
      // condensed matrix Gc
      for (size_t j = 0; j < jobs.size(); ++j) {
        const MergeJob& J = jobs[j];
        Scr& s = scr[j];
        const int m1 = J.f1.m.max, m2 = J.f2.m.max;
        if (!J.vertical) {
          // Gc = [L1 rho1^T, L2 rho2^T]
          B.tiles(PT(AR_WS, s.Gc), AGGC, J.f1.rows_t, J.f1.m, 0, [&](int r0, int, int c0, Dim) {
            B.term2(rows_of(J.f1.L, r0), mref(PT(AR_WS, s.rho1 + (int64_t)c0 * m1), m1, 1), J.f1.m.d());
          });
          Ptr o2 = pdyn(PT(AR_WS, s.Gc + J.f1.m.c), J.f1.m.s, 1);
          B.tiles(o2, AGGC, J.f1.rows_t, J.f2.m, 0, [&](int r0, int, int c0, Dim) {
            B.term2(rows_of(J.f2.L, r0), mref(PT(AR_WS, s.rho2 + (int64_t)c0 * m2), m2, 1), J.f2.m.d());
          });
        } else {
          // Gc = [L1 rho[:, :m1]^T; L2 rho[:, m1:]^T], rho is (m1+m2) x (m1+m2)
          const int ldr = m1 + m2;
          const Dim qd = merged_width(J.f1.m, J.f2.m);
          for (int c0 = 0; c0 < m1 + m2; c0 += GEMM_MAXTILE) {
            Dim w = qd;
            w.c -= c0;  // columns c0 .. c0+63 of the merged width (clamped)
            for (int part = 0; part < 2; ++part) {
              const Factor& F = part == 0 ? J.f1 : J.f2;
              const int rowoff = part == 0 ? 0 : J.f1.rows_t;
              for (int r0 = 0; r0 < F.rows_t; r0 += GEMM_MAXTILE) {
                const int nr = std::min(GEMM_MAXTILE, F.rows_t - r0);
                B.out(PT(AR_WS, s.Gc + (int64_t)(rowoff + r0) * AGGC + c0), AGGC, DC(nr), w, 0, 1);
                Ptr rb = padd(PT(AR_WS, s.rho1), (int64_t)c0 * ldr);
                if (part == 1) rb = pdyn(padd(rb, J.f1.m.c), J.f1.m.s, 1);
                B.term2(rows_of(F.L, r0), mref(rb, ldr, 1), F.m.d());
              }
            }
          }
        }
      }
      B.flush_gemm(TAG_AGG);
      // QR of Gc, SVD of rho_c^T, new L = Gc V, new R = Q V
      for (size_t j = 0; j < jobs.size(); ++j) {
        const MergeJob& J = jobs[j];
        Scr& s = scr[j];
        const int m1 = J.f1.m.max, m2 = J.f2.m.max;
        const int rows = J.vertical ? J.f1.rows_t + J.f2.rows_t : J.f1.rows_t;
        const Dim wd = merged_width(J.f1.m, J.f2.m);
        B.copy(PT(AR_WS, s.Gc), AGGC, PT(AR_WS, s.Wc), rows, wd, DC(rows), 1);
      }
      B.flush_copy(TAG_AGG);
      for (size_t j = 0; j < jobs.size(); ++j) {
        const MergeJob& J = jobs[j];
        Scr& s = scr[j];
        const int m1 = J.f1.m.max, m2 = J.f2.m.max;
        const int rows = J.vertical ? J.f1.rows_t + J.f2.rows_t : J.f1.rows_t;
        const Dim wd = merged_width(J.f1.m, J.f2.m);
        // two-step jobs take R with its columns back in the original order
        // (R P^T): then M = (R P^T)^T carries the pivot and U needs no permutation
        B.qr(PT(AR_WS, s.Wc), rows, DC(rows), wd, PT(AR_WS, s.tauc), PT(AR_WS, s.rhoc), AGGC, 0, rows,
             J.f1.m.max + J.f2.m.max, PT(AR_WS, s.piv), s.two_step ? 1 : 0, PARAM_SVD_FLOOR, s.rslot);
      }
      B.flush_qr(TAG_AGG);
      // second QR of the two-step jobs: M = rho_c^T = Q2 R2 (in place, the
      // reflectors stay for U = Q2 Y; R2 stored transposed for the SVD)
      for (size_t j = 0; j < jobs.size(); ++j) {
        const MergeJob& J = jobs[j];
        Scr& s = scr[j];
        if (!s.two_step) continue;
        const int m1 = J.f1.m.max, m2 = J.f2.m.max;
        const int gr = J.vertical ? J.f1.rows_t + J.f2.rows_t : J.f1.rows_t;
        const int qmax = std::min(m1 + m2, gr);
        const Dim wd = merged_width(J.f1.m, J.f2.m);
        B.qr(PT(AR_WS, s.rhoc), AGGC, wd, DS(s.rslot, 0), PT(AR_WS, s.tau2c), PT(AR_WS, s.R2), qmax, 1, m1 + m2, qmax,
             NONE(), 2);
      }
      B.flush_qr(TAG_AGG);
      for (size_t j = 0; j < jobs.size(); ++j) {
        const MergeJob& J = jobs[j];
        Scr& s = scr[j];
        const int m1 = J.f1.m.max, m2 = J.f2.m.max;
        // M = rho_c^T ((m1+m2) x (m1+m2)); rows and cols are the merged width
        const Dim wd = merged_width(J.f1.m, J.f2.m);
        if (m1 + m2 > SVD_MAXDIM) throw std::runtime_error("agglomeration svd too large");
        // M = rho_c^T (width x r), r <= min(width, rows of Gc) the rows of
        // rho_c above the noise floor (the rest is zero)
        const int gc_rows = J.vertical ? J.f1.rows_t + J.f2.rows_t : J.f1.rows_t;
        const Dim qcols = DS(s.rslot, 0);
        const bool last = J.vertical && J.row == (1 << aggs[J.agg].d) - 1;
        const int nidx = last ? (agg_nidx[J.agg] = B.scal()) : -1;
        if (s.two_step) {
          const int qmax = std::min(m1 + m2, gc_rows);
          B.svd_size(qmax, qmax);
          B.sv.push_back(SvdJob{PT(AR_WS, s.R2), PT(AR_WS, s.Y), PT(AR_WS, s.sig), qmax, AGGC, qcols, qcols, 1, 2, J.rel,
                                PARAM_TOL_AGG, outs[j].m.s, AGGM, nidx, NONE()});
          continue;
        }
        B.svd_size(m1 + m2, std::min(m1 + m2, gc_rows));
        B.sv.push_back(SvdJob{PT(AR_WS, s.rhoc), PT(AR_WS, s.U), PT(AR_WS, s.sig), AGGC, AGGC, wd, qcols, 1, 2, J.rel,
                              PARAM_TOL_AGG, outs[j].m.s, AGGM, nidx, PT(AR_WS, s.piv)});
      }
      B.flush_svd(TAG_AGG);
      // two-step jobs: U[:, :k'] = Q2 [Y[:, :k']; 0]
      for (size_t j = 0; j < jobs.size(); ++j) {
        const MergeJob& J = jobs[j];
        Scr& s = scr[j];
        if (!s.two_step) continue;
        const Dim wd = merged_width(J.f1.m, J.f2.m);
        B.qapply(PT(AR_WS, s.rhoc), AGGC, PT(AR_WS, s.tau2c), wd, DS(s.rslot, 0), PT(AR_WS, s.Y), AGGC,
                 outs[j].m.d(), PT(AR_WS, s.U), AGGC);
      }
      B.flush_qapply(TAG_AGG);
      for (size_t j = 0; j < jobs.size(); ++j) {
        const MergeJob& J = jobs[j];
        Scr& s = scr[j];
        const Factor& o = outs[j];
        const Dim wd = merged_width(J.f1.m, J.f2.m);
        // L' = Gc U[:, :k']
        B.tiles(o.L.p, o.L.ld, o.rows_t, o.m, 0, [&](int r0, int, int, Dim) {
          B.term2(mref(PT(AR_WS, s.Gc + (int64_t)r0 * AGGC), AGGC), mref(PT(AR_WS, s.U), AGGC), wd);
        });
        // R' = Q U[:, :k']
        if (!J.vertical) {
          B.qapply(PT(AR_WS, s.W1), J.f1.rows_r, PT(AR_WS, s.tau1), DC(J.f1.rows_r), J.f1.m.d(), PT(AR_WS, s.U), AGGC,
                   o.m.d(), o.R.p, o.R.ld);
          B.qapply(PT(AR_WS, s.W2), J.f2.rows_r, PT(AR_WS, s.tau2), DC(J.f2.rows_r), J.f2.m.d(),
                   pdyn(PT(AR_WS, s.U + (int64_t)J.f1.m.c * AGGC), J.f1.m.s, AGGC), AGGC, o.m.d(),
                   padd(o.R.p, (int64_t)J.f1.rows_r * o.R.ld), o.R.ld);
        } else {
          B.qapply(PT(AR_WS, s.W1), J.f1.rows_r, PT(AR_WS, s.tau1), DC(J.f1.rows_r), wd, PT(AR_WS, s.U), AGGC,
                   o.m.d(), o.R.p, o.R.ld);
        }
      }
      B.flush_gemm(TAG_AGG);
      B.flush_qapply(TAG_AGG);
      // advance the state
      for (size_t j = 0; j < jobs.size(); ++j) {
        const MergeJob& J = jobs[j];
        if (!J.vertical) rowf[J.agg][J.row] = outs[j];
        else colf[J.agg] = outs[j];
      }
      B.ws = mark;  // scratch of this step is free again
    }
    for (size_t a = 0; a < aggs.size(); ++a) {
      const int n = 1 << aggs[a].d;
      agg_result[a] = (n == 1) ? rowf[a][0] : colf[a];
    }
  }

  P.stats["ws_before_p11"] = B.ws;
  // ----------------------------------- 11. condensation and norms ----
  struct Final {
    int cb, t, r;
    Factor f;
    int nidx;            // norm / scale index (set already for merged agglomerations)
    int64_t rhoR, rhoL;  // MB x MB row-major
    int64_t Gc, Gcc;     // |t| x MB, |r| x MB
  };
  std::vector<Final> fin;
  for (size_t q = 0; q < V.size(); ++q) {
    const VNode& n = V[q];
    if (n.kind == VK_SU) {
      Final F{n.cb, n.t, n.r, cell_factor(n), -1, 0, 0, 0, 0};
      fin.push_back(F);
    } else if (n.kind == VK_AGGROOT) {
      Final F{n.cb, n.t, n.r, agg_result[n.agg], agg_nidx[n.agg], 0, 0, 0, 0};
      fin.push_back(F);
    }
  }
  std::vector<int> fin_of_cb(BC.t.size(), -1);
  for (size_t i = 0; i < fin.size(); ++i) fin_of_cb[fin[i].cb] = (int)i;
  if (opt.hmatrix) {
    // H-matrix output: every admissible target leaf keeps its accumulated or
    // agglomerated factors (the standard H-matrix approximation the product
    // reaches before the nested-basis recompression); the nearfield is in
    // place already
    P.rank_row_slot.clear();
    P.rank_col_slot.clear();
    for (int cb : BC.adm_list) {
      const int i = fin_of_cb[cb];
      if (i < 0) throw std::runtime_error("admissible leaf without factors");
      const Final& F = fin[i];
      const int w = F.f.m.max;
      const int64_t oL = P.c_len, oR = oL + (int64_t)F.f.rows_t * w;
      P.c_len = oR + (int64_t)F.f.rows_r * w;
      B.copy(F.f.L.p, F.f.L.ld, PT(AR_C, oL), w, DC(F.f.rows_t), F.f.m.d(), 0, 1.0, -1, DC(F.f.rows_t), DC(w));
      B.copy(F.f.R.p, F.f.R.ld, PT(AR_C, oR), w, DC(F.f.rows_r), F.f.m.d(), 0, 1.0, -1, DC(F.f.rows_r), DC(w));
      P.hm_off_L.push_back(oL);
      P.hm_off_R.push_back(oR);
      P.hm_w.push_back(w);
      P.rank_row_slot.push_back(F.f.m.s >= 0 ? F.f.m.s : B.slot(F.f.m.c));
    }
    B.flush_copy(TAG_COUPLE);
    P.stats["ws_bump_bytes"] = B.ws_peak * 8;
    P.ws_len = pack_workspace(P, B.bufs);
    P.fac_len = B.fac;
    P.stats["final_adm"] = fin.size();
    P.stats["stages"] = P.stages.size();
    return plan;
  }
  {
    const int64_t mark = B.ws;
    std::vector<std::array<int64_t, 4>> scr(fin.size());
    std::vector<char> has_norm(fin.size());
    for (size_t i = 0; i < fin.size(); ++i) {
      Final& F = fin[i];
      has_norm[i] = F.nidx >= 0;
      if (!has_norm[i]) F.nidx = B.scal();
      F.rhoR = B.alloc((int64_t)MB * MB);
      F.rhoL = B.alloc((int64_t)MB * MB);
      F.Gc = B.alloc((int64_t)F.f.rows_t * MB);
      F.Gcc = B.alloc((int64_t)F.f.rows_r * MB);
    }
    const int64_t mark2 = B.ws;
    for (size_t i = 0; i < fin.size(); ++i) {
      Final& F = fin[i];
      const int m = F.f.m.max;
      scr[i][0] = B.alloc((int64_t)F.f.rows_r * m);  // WR
      scr[i][1] = B.alloc((int64_t)F.f.rows_t * m);  // WL
      scr[i][2] = B.alloc(m);
      scr[i][3] = B.alloc(m);
      B.copy(F.f.R.p, F.f.R.ld, PT(AR_WS, scr[i][0]), F.f.rows_r, F.f.m.d(), DC(F.f.rows_r), 1);
      B.copy(F.f.L.p, F.f.L.ld, PT(AR_WS, scr[i][1]), F.f.rows_t, F.f.m.d(), DC(F.f.rows_t), 1);
      B.qr(PT(AR_WS, scr[i][0]), F.f.rows_r, DC(F.f.rows_r), F.f.m.d(), PT(AR_WS, scr[i][2]), PT(AR_WS, F.rhoR), MB, 0,
           F.f.rows_r, m);
      B.qr(PT(AR_WS, scr[i][1]), F.f.rows_t, DC(F.f.rows_t), F.f.m.d(), PT(AR_WS, scr[i][3]), PT(AR_WS, F.rhoL), MB, 0,
           F.f.rows_t, m);
    }
    B.flush_copy(TAG_COND);
    B.flush_qr(TAG_COND);
    // G^c = L rhoR^T, G^c' = R rhoL^T, norm matrix rhoL rhoR^T
    std::vector<int64_t> nm(fin.size());
    for (size_t i = 0; i < fin.size(); ++i) {
      Final& F = fin[i];
      B.tiles(PT(AR_WS, F.Gc), MB, F.f.rows_t, F.f.m, 0, [&](int r0, int, int c0, Dim) {
        B.term2(rows_of(F.f.L, r0), mref(PT(AR_WS, F.rhoR + (int64_t)c0 * MB), MB, 1), F.f.m.d());
      });
      B.tiles(PT(AR_WS, F.Gcc), MB, F.f.rows_r, F.f.m, 0, [&](int r0, int, int c0, Dim) {
        B.term2(rows_of(F.f.R, r0), mref(PT(AR_WS, F.rhoL + (int64_t)c0 * MB), MB, 1), F.f.m.d());
      });
      if (has_norm[i]) continue;
      nm[i] = B.alloc((int64_t)MB * MB);
      B.tiles(PT(AR_WS, nm[i]), MB, F.f.m.max, F.f.m, 0, [&](int r0, int nr, int c0, Dim) {
        if (F.f.m.s >= 0) {
          // dynamic width (<= 64): one tile, rows clamped to the rank
          B.go.back().m = F.f.m.d();
        }
        (void)nr;
        B.term2(mref(PT(AR_WS, F.rhoL + (int64_t)r0 * MB), MB),
                mref(PT(AR_WS, F.rhoR + (int64_t)c0 * MB), MB, 1), F.f.m.d());
      });
    }
    B.flush_gemm(TAG_COND);
    for (size_t i = 0; i < fin.size(); ++i) {
      Final& F = fin[i];
      if (has_norm[i]) {
        ++P.stats["norms_from_agglomeration"];
        continue;
      }
      B.norm(PT(AR_WS, nm[i]), MB, F.f.m, F.nidx);
    }
    B.flush_norm(TAG_COND);
    (void)mark;
    (void)mark2;
  }

  P.stats["ws_before_p12"] = B.ws;
  // --------------------------------------- 12. adaptive cluster bases ----
  // row*(t): final admissible blocks whose row cluster is t or an ancestor.
  // The row and the column basis are independent: their levels run in the
  // same launches (twice the jobs per stage).
  struct Side {
    bool rowside;
    const Tree* T;
    int tag;
    int64_t offBasis, offTrans;
    std::vector<std::vector<int>> star;
    std::vector<int> rank;
    std::map<std::pair<int, int>, int64_t> lam;  // Lambda-hat_{c,b} = V_c^* L_b|_c (KP x MB)
    // per level
    std::vector<int> cl, offslot, wmax;
    std::vector<int64_t> panel, rbuf, ubuf, tbuf, pbuf;
    std::vector<int> rq;  // rows of the panel's R kept above the noise floor (slot)
  };
  auto make_basis_side = [&](bool rowside) {
    Side S;
    S.rowside = rowside;
    S.T = rowside ? &TI : &TK;
    S.tag = rowside ? TAG_ROWB : TAG_COLB;
    S.offBasis = rowside ? P.c_off_V : P.c_off_W;
    S.offTrans = rowside ? P.c_off_E : P.c_off_F;
    const Tree& T = *S.T;
    std::vector<std::vector<int>> own(T.ncl);
    S.star.resize(T.ncl);
    for (size_t i = 0; i < fin.size(); ++i) own[rowside ? fin[i].t : fin[i].r].push_back((int)i);
    for (int c = 0; c < T.ncl; ++c) {
      if (c > 0) S.star[c] = S.star[Tree::parent(c)];
      S.star[c].insert(S.star[c].end(), own[c].begin(), own[c].end());
    }
    S.rank.assign(T.ncl, -1);
    for (int c = 0; c < T.ncl; ++c) S.rank[c] = B.slot(0);
    (rowside ? P.rank_row_slot : P.rank_col_slot) = S.rank;
    return S;
  };
  Side SR = make_basis_side(true), SC = make_basis_side(false);
  auto fac_rows = [&](const Side& S, const Final& F) { return S.rowside ? F.f.L : F.f.R; };
  auto blk_cluster = [&](const Side& S, const Final& F) { return S.rowside ? F.t : F.r; };
  auto rho = [&](const Side& S, const Final& F) { return S.rowside ? F.rhoR : F.rhoL; };
  auto Gcond = [&](const Side& S, const Final& F) { return S.rowside ? F.Gc : F.Gcc; };
  const double tol_mult = 1.0;
  // GEMM output columns of a factor width: dynamic widths (<= 64) in one tile,
  // static ones in tiles of GEMM_MAXTILE
  auto col_tiles = [&](const DimV& m, const std::function<void(int, Dim)>& emit) {
    if (m.s >= 0) {
      if (m.max > GEMM_MAXTILE) throw std::runtime_error("dynamic factor width above tile");
      emit(0, m.d());
      return;
    }
    for (int c0 = 0; c0 < m.c; c0 += GEMM_MAXTILE) emit(c0, DC(std::min(GEMM_MAXTILE, m.c - c0)));
  };
  // phase 0: panel widths (prefix sums of the factor widths)
  auto ph_scan = [&](Side& S, int l) {
    const Tree& T = *S.T;
    S.cl.clear();
    for (int c = Tree::first(l); c < Tree::first(l + 1); ++c)
      if (!S.star[c].empty()) S.cl.push_back(c);
    S.offslot.assign(T.ncl, -1);
    S.wmax.assign(T.ncl, 0);
    S.panel.assign(T.ncl, -1);
    S.rbuf.assign(T.ncl, -1);
    S.ubuf.assign(T.ncl, -1);
    S.tbuf.assign(T.ncl, -1);
    S.pbuf.assign(T.ncl, -1);
    S.rq.assign(T.ncl, -1);
    for (int c : S.cl) {
      std::vector<int> in;
      for (int b : S.star[c]) {
        const Final& F = fin[b];
        in.push_back(F.f.m.s >= 0 ? F.f.m.s : B.slot(F.f.m.c));
        S.wmax[c] += F.f.m.max;
      }
      S.offslot[c] = (int)P.slot_init.size();
      for (size_t i = 0; i <= in.size(); ++i) B.slot(0);
      B.scan(in, S.offslot[c]);
    }
  };
  // phase 1: weighted panels
  auto ph_panel = [&](Side& S) {
    const Tree& T = *S.T;
    for (int c : S.cl) {
      const int n = T.leaf(c) ? T.size[c] : 2 * KP;
      S.panel[c] = B.alloc((int64_t)n * S.wmax[c]);
      S.rbuf[c] = B.alloc((int64_t)n * n);
      S.ubuf[c] = B.alloc((int64_t)n * n);
      S.tbuf[c] = B.alloc(n);
      S.pbuf[c] = B.alloc((n + 1) / 2);  // int32 pivot order of the panel QR
      const int lev = T.level[c];
      for (size_t i = 0; i < S.star[c].size(); ++i) {
        const Final& F = fin[S.star[c][i]];
        const int tb = blk_cluster(S, F);
        const double w = std::pow(theta, -0.5 * (lev - T.level[tb]));  // 1/omega up to 1/||G||
        Ptr dst = pdyn(PT(AR_WS, S.panel[c]), S.offslot[c] + (int)i, 1);
        if (T.leaf(c)) {
          // leaf: omega^{-1} G^c_b restricted to the rows of c
          const int64_t r0 = T.off[c] - T.off[tb];
          B.copy(PT(AR_WS, Gcond(S, F) + r0 * MB), MB, dst, S.wmax[c], DC(T.size[c]), F.f.m.d(), 0, w, F.nidx);
        } else {
          // inner: omega^{-1} [Lhat_{c1,b}; Lhat_{c2,b}] rho_b^T
          for (int h = 0; h < 2; ++h) {
            const int ch = Tree::child(c, h);
            Ptr d2 = h == 0 ? dst : pdyn(dst, S.rank[Tree::child(c, 0)], S.wmax[c]);
            col_tiles(F.f.m, [&](int c0, Dim wdim) {
              B.out(padd(d2, c0), S.wmax[c], DS(S.rank[ch]), wdim, 0);
              B.term2(mref(PT(AR_WS, S.lam.at({ch, S.star[c][i]})), MB),
                      mref(PT(AR_WS, rho(S, F) + (int64_t)c0 * MB), MB, 1), F.f.m.d(), w, F.nidx);
            });
          }
        }
      }
    }
  };
  auto rows_dim = [&](const Side& S, int c) {
    const Tree& T = *S.T;
    return T.leaf(c) ? DC(T.size[c]) : DSS(S.rank[Tree::child(c, 0)], S.rank[Tree::child(c, 1)]);
  };
  // phase 2: QR of the panel (column-major view: width x rows)
  auto ph_qr = [&](Side& S) {
    const Tree& T = *S.T;
    for (int c : S.cl) {
      const int n = T.leaf(c) ? T.size[c] : 2 * KP;
      const int nsl = S.offslot[c] + (int)S.star[c].size();  // total width slot
      // the pivoted QR stops at the SVD's noise floor, as in agglomeration:
      // the rows of R it drops are columns of R^T the Jacobi SVD would freeze
      S.rq[c] = B.slot(0);
      B.qr(PT(AR_WS, S.panel[c]), S.wmax[c], DS(nsl), rows_dim(S, c), PT(AR_WS, S.tbuf[c]), PT(AR_WS, S.rbuf[c]), n,
           0, S.wmax[c], n, PT(AR_WS, S.pbuf[c]), 0, PARAM_SVD_FLOOR, S.rq[c]);
    }
  };
  // phase 3: Jacobi SVD of R^T with the truncation rule
  auto ph_svd = [&](Side& S) {
    const Tree& T = *S.T;
    for (int c : S.cl) {
      const int n = T.leaf(c) ? T.size[c] : 2 * KP;
      const Dim rows_d = rows_dim(S, c);
      B.svd_size(n, n);
      // M = R^T (rows x r), r <= min(rows, panel width) the rows of R kept
      const Dim qcols = DS(S.rq[c], 0);
      B.sv.push_back(SvdJob{PT(AR_WS, S.rbuf[c]), PT(AR_WS, S.ubuf[c]), NONE(), n, n, rows_d, qcols, 1, 1, tol_mult,
                            PARAM_TOL_BASIS, S.rank[c], KP, -1, PT(AR_WS, S.pbuf[c])});
    }
  };
  // phase 4: new basis: leaves V_c = U[:, :k_c]; inner E_{c1}, E_{c2} = blocks of U[:, :k_c]
  auto ph_store = [&](Side& S) {
    const Tree& T = *S.T;
    for (int c : S.cl) {
      const int n = T.leaf(c) ? T.size[c] : 2 * KP;
      if (T.leaf(c)) {
        B.copy(PT(AR_WS, S.ubuf[c]), n, PT(AR_C, S.offBasis + (int64_t)T.off[c] * KP), KP, DC(T.size[c]),
               DS(S.rank[c]), 0);
      } else {
        const int c1 = Tree::child(c, 0), c2 = Tree::child(c, 1);
        B.copy(PT(AR_WS, S.ubuf[c]), n, PT(AR_C, S.offTrans + (int64_t)c1 * KP * KP), KP, DS(S.rank[c1]),
               DS(S.rank[c]), 0);
        B.copy(pdyn(PT(AR_WS, S.ubuf[c]), S.rank[c1], n), n, PT(AR_C, S.offTrans + (int64_t)c2 * KP * KP), KP,
               DS(S.rank[c2]), DS(S.rank[c]), 0);
      }
    }
  };
  // phase 5: projection climb: Lhat_{c,b} = V_c^* L_b|_c (leaf) or E_{c1}^* Lhat_{c1,b} + E_{c2}^* Lhat_{c2,b}
  auto ph_climb = [&](Side& S) {
    const Tree& T = *S.T;
    for (int c : S.cl) {
      for (int b : S.star[c]) {
        const Final& F = fin[b];
        const int64_t o = B.alloc((int64_t)KP * MB);
        S.lam[{c, b}] = o;
        col_tiles(F.f.m, [&](int c0, Dim wdim) {
          B.out(PT(AR_WS, o + c0), MB, DS(S.rank[c]), wdim, 0);
          if (T.leaf(c)) {
            const int tb = blk_cluster(S, F);
            MRef Lr = rows_of(fac_rows(S, F), T.off[c] - T.off[tb]);
            Lr.p = padd(Lr.p, c0);
            B.term2(mref(PT(AR_C, S.offBasis + (int64_t)T.off[c] * KP), KP, 1), Lr, DC(T.size[c]));
          } else {
            for (int h = 0; h < 2; ++h) {
              const int ch = Tree::child(c, h);
              B.term2(mref(PT(AR_C, S.offTrans + (int64_t)ch * KP * KP), KP, 1),
                      mref(PT(AR_WS, S.lam.at({ch, b}) + c0), MB), DS(S.rank[ch]));
            }
          }
        });
      }
    }
  };
  for (int l = D; l >= 0; --l) {
    const int64_t mark = B.ws;
    ph_scan(SR, l);
    ph_scan(SC, l);
    B.flush_scan(TAG_ROWB);
    ph_panel(SR);
    ph_panel(SC);
    B.flush_all(TAG_ROWB);
    ph_qr(SR);
    ph_qr(SC);
    B.flush_qr(TAG_ROWB);
    ph_svd(SR);
    ph_svd(SC);
    B.flush_svd(TAG_ROWB);
    ph_store(SR);
    ph_store(SC);
    B.flush_copy(TAG_ROWB);
    B.ws = mark;  // panels and factorizations of this level are free again
    ph_climb(SR);
    ph_climb(SC);
    B.flush_gemm(TAG_ROWB);
  }
  auto& lamR = SR.lam;
  auto& lamC = SC.lam;

  P.stats["ws_before_p13"] = B.ws;
  // --------------------------------------------------- 13. couplings ----
  // S_b = (V_t^* L_b) (W_r^* R_b)^*
  for (size_t i = 0; i < fin.size(); ++i) {
    const Final& F = fin[i];
    const int a = BC.leafidx[F.cb];
    B.out(PT(AR_C, P.c_off_S + (int64_t)a * KP * KP), KP, DS(P.rank_row_slot[F.t]), DS(P.rank_col_slot[F.r]), 0);
    B.term2(mref(PT(AR_WS, lamR.at({F.t, (int)i})), MB), mref(PT(AR_WS, lamC.at({F.r, (int)i})), MB, 1), F.f.m.d());
  }
  B.flush_gemm(TAG_COUPLE);

  P.stats["ws_bump_bytes"] = B.ws_peak * 8;
  P.ws_len = pack_workspace(P, B.bufs);
  P.fac_len = B.fac;
  P.stats["final_adm"] = fin.size();
  P.stats["stages"] = P.stages.size();
  P.stats["gemm_outputs"] = P.gout.size();
  P.stats["gemm_terms"] = P.gterm.size();
  P.stats["svd_jobs"] = P.svd.size();
  P.stats["norm_jobs"] = P.norm.size();
  P.stats["qr_jobs"] = P.qr.size();
  P.stats["ws_bytes"] = P.ws_len * 8;
  return plan;
}

}  // namespace h2

// ======================================================= helper plans ====
namespace h2 {

std::shared_ptr<Plan> make_levelbasis_plan(const Tree& T, int k, int ar, int64_t off_leaf, int64_t off_trans,
                                           int64_t off_out) {
  auto plan = std::make_shared<Plan>();
  Builder B(*plan);
  const int n = T.n, D = T.depth;
  B.copy(PT(ar, off_leaf), k, PT(ar, off_out + (int64_t)D * n * k), k, DC(n), DC(k), 0);
  B.flush_copy(0);
  for (int l = D - 1; l >= 0; --l) {
    for (int c = Tree::first(l + 1); c < Tree::first(l + 2); ++c) {
      const int64_t row = T.off[c];
      B.tiles(PT(ar, off_out + ((int64_t)l * n + row) * k), k, T.size[c], dv(k), 0, [&](int r0, int, int, Dim) {
        B.term2(mref(PT(ar, off_out + ((int64_t)(l + 1) * n + row + r0) * k), k),
                mref(PT(ar, off_trans + (int64_t)c * k * k), k), DC(k));
      });
    }
    B.flush_gemm(0);
  }
  plan->ws_len = B.ws_peak;
  return plan;
}

std::shared_ptr<Plan> make_matvec_plan(const MatDesc& A, int nrhs) {
  auto plan = std::make_shared<Plan>();
  Builder B(*plan);
  const Tree& R = *A.rows;
  const Tree& C = *A.cols;
  const BlockTree& BT = *A.blocks;
  const int k = A.k, D = C.depth;
  const int64_t q = nrhs;  // every vector block is row-major with nrhs columns
  const int64_t ox = B.alloc(C.n * q), oy = B.alloc(R.n * q);
  const int64_t oxh = B.alloc((int64_t)C.ncl * k * q), oyh = B.alloc((int64_t)R.ncl * k * q);
  plan->mv_ox = ox;
  plan->mv_oy = oy;
  // right-hand-side columns in tiles of GEMM_MAXTILE
  auto cols = [&](const std::function<void(int, Dim)>& emit) {
    for (int c0 = 0; c0 < nrhs; c0 += GEMM_MAXTILE) emit(c0, DC(std::min(GEMM_MAXTILE, nrhs - c0)));
  };
  // forward transform x^_s = W_s^* x|_s
  for (int s = Tree::first(D); s < C.ncl; ++s)
    cols([&](int c0, Dim w) {
      B.out(PT(AR_WS, oxh + (int64_t)s * k * q + c0), q, DC(k), w, 0);
      B.term2(mref(PT(AR_X, A.off_W + (int64_t)C.off[s] * k), k, 1), mref(PT(AR_WS, ox + C.off[s] * q + c0), q),
              DC(C.size[s]));
    });
  B.flush_gemm(0);
  for (int l = D - 1; l >= 0; --l) {
    for (int s = Tree::first(l); s < Tree::first(l + 1); ++s)
      cols([&](int c0, Dim w) {
        B.out(PT(AR_WS, oxh + (int64_t)s * k * q + c0), q, DC(k), w, 0);
        for (int i = 0; i < 2; ++i) {
          const int c = Tree::child(s, i);
          B.term2(mref(PT(AR_X, A.off_F + (int64_t)c * k * k), k, 1), mref(PT(AR_WS, oxh + (int64_t)c * k * q + c0), q),
                  DC(k));
        }
      });
    B.flush_gemm(0);
  }
  // coupling y^_t = sum_s S_ts x^_s
  std::vector<std::vector<int>> byrow(R.ncl);
  for (int b : BT.adm_list) byrow[BT.t[b]].push_back(b);
  for (int t = 0; t < R.ncl; ++t)
    cols([&](int c0, Dim w) {
      B.out(PT(AR_WS, oyh + (int64_t)t * k * q + c0), q, DC(k), w, 0);
      for (int b : byrow[t])
        B.term2(mref(PT(AR_X, A.off_S + (int64_t)BT.leafidx[b] * k * k), k),
                mref(PT(AR_WS, oxh + (int64_t)BT.s[b] * k * q + c0), q), DC(k));
    });
  B.flush_gemm(0);
  // backward transform y^_c += E_c y^_parent
  for (int l = 1; l <= D; ++l) {
    for (int c = Tree::first(l); c < Tree::first(l + 1); ++c)
      cols([&](int c0, Dim w) {
        B.out(PT(AR_WS, oyh + (int64_t)c * k * q + c0), q, DC(k), w, 1);
        B.term2(mref(PT(AR_X, A.off_E + (int64_t)c * k * k), k),
                mref(PT(AR_WS, oyh + (int64_t)Tree::parent(c) * k * q + c0), q), DC(k));
      });
    B.flush_gemm(0);
  }
  // leaves: y|_t = V_t y^_t + sum_s N_ts x|_s
  std::vector<std::vector<int>> nrow(R.ncl);
  for (int b : BT.inadm_list) nrow[BT.t[b]].push_back(b);
  for (int t = Tree::first(D); t < R.ncl; ++t) {
    B.tiles(PT(AR_WS, oy + R.off[t] * q), q, R.size[t], dv(nrhs), 0, [&](int r0, int, int c0, Dim) {
      B.term2(mref(PT(AR_X, A.off_V + (int64_t)(R.off[t] + r0) * k), k),
              mref(PT(AR_WS, oyh + (int64_t)t * k * q + c0), q), DC(k));
      for (int b : nrow[t]) {
        const int s = BT.s[b];
        B.term2(mref(PT(AR_X, A.off_N + BT.near_off[BT.leafidx[b]] + (int64_t)r0 * C.size[s]), C.size[s]),
                mref(PT(AR_WS, ox + C.off[s] * q + c0), q), DC(C.size[s]));
      }
    });
  }
  B.flush_gemm(0);
  plan->ws_len = B.ws_peak;
  return plan;
}

std::shared_ptr<Plan> make_hmatrix_dense_plan(const Tree& R, const Tree& C, const BlockTree& BT, int64_t off_N,
                                              const std::vector<int64_t>& off_L, const std::vector<int64_t>& off_R,
                                              const std::vector<int>& w) {
  auto plan = std::make_shared<Plan>();
  Builder B(*plan);
  const int64_t ld = C.n;
  const int64_t od = B.alloc((int64_t)R.n * C.n);
  for (size_t a = 0; a < BT.adm_list.size(); ++a) {
    const int b = BT.adm_list[a], t = BT.t[b], s = BT.s[b];
    B.tiles(PT(AR_WS, od + (int64_t)R.off[t] * ld + C.off[s]), ld, R.size[t], dv(C.size[s]), 0,
            [&](int r0, int, int c0, Dim) {
              B.term2(mref(PT(AR_X, off_L[a] + (int64_t)r0 * w[a]), w[a]),
                      mref(PT(AR_X, off_R[a] + (int64_t)c0 * w[a]), w[a], 1), DC(w[a]));
            });
  }
  B.flush_gemm(0);
  for (size_t a = 0; a < BT.inadm_list.size(); ++a) {
    const int b = BT.inadm_list[a], t = BT.t[b], s = BT.s[b];
    B.copy(PT(AR_X, off_N + BT.near_off[a]), C.size[s], PT(AR_WS, od + (int64_t)R.off[t] * ld + C.off[s]), ld,
           DC(R.size[t]), DC(C.size[s]), 0);
  }
  B.flush_copy(0);
  plan->ws_len = B.ws_peak;
  return plan;
}

std::shared_ptr<Plan> make_dense_plan(const MatDesc& A) {
  auto plan = std::make_shared<Plan>();
  Builder B(*plan);
  const Tree& R = *A.rows;
  const Tree& C = *A.cols;
  const BlockTree& BT = *A.blocks;
  const int k = A.k;
  const int64_t od = B.alloc((int64_t)R.n * C.n);
  const int ld = C.n;
  for (int b : BT.adm_list) {
    const int t = BT.t[b], s = BT.s[b];
    B.tiles(PT(AR_WS, od + (int64_t)R.off[t] * ld + C.off[s]), ld, R.size[t], dv(C.size[s]), 0,
            [&](int r0, int, int c0, Dim) {
              B.term3(mref(PT(AR_X, A.off_VF + ((int64_t)R.level[t] * R.n + R.off[t] + r0) * k), k),
                      mref(PT(AR_X, A.off_S + (int64_t)BT.leafidx[b] * k * k), k),
                      mref(PT(AR_X, A.off_WF + ((int64_t)C.level[s] * C.n + C.off[s] + c0) * k), k, 1), DC(k), DC(k));
            });
  }
  B.flush_gemm(0);
  for (int b : BT.inadm_list) {
    const int t = BT.t[b], s = BT.s[b];
    B.copy(PT(AR_X, A.off_N + BT.near_off[BT.leafidx[b]]), C.size[s], PT(AR_WS, od + (int64_t)R.off[t] * ld + C.off[s]),
           ld, DC(R.size[t]), DC(C.size[s]), 0);
  }
  B.flush_copy(0);
  plan->ws_len = B.ws_peak;
  return plan;
}

}  // namespace h2
