// Host test of the planner: runs a product plan (make_product_plan) with a
// plain CPU interpreter of the stage semantics of h2_ops.h and writes the
// dense product, so that a CPU-only test can compare the planner's job lists
// with the oracle.  Test infrastructure: it links the planner and the host
// tree / Chebyshev construction under test, and states each stage kind in the
// simplest form (no blocking, no precision tricks): GEMM chains, copies,
// Householder QR (with the column pivoting of the kernels), the thin-Q
// application, a cyclic one-sided Jacobi SVD with the truncation modes,
// spectral norms (as the largest singular value) and rank prefix sums.
//
// Usage: stage_interpreter points.bin n dim leaf order eta eps
//            kindA sA dA wA kindB sB dB wB max_rank hmatrix out.bin [svd_sweeps]
// out.bin: dense n x n product (row-major, caller ordering), then the row and
// column ranks per cluster (int32, level order); with hmatrix = 1 the
// H-matrix output variant is expanded instead and no ranks are written.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "host_assembly.h"
#include "../../paper_2403_01566_gb300/csrc/h2_plan.h"

using namespace h2;
using h2host::HostH2;
using h2host::assemble_chebyshev;

namespace {

struct Interp {
  double* base[AR_COUNT] = {};
  std::vector<int> slot;
  std::vector<double> scal, nrm;
  std::vector<int> idx;
  int err = 0;

  int dimv(const Dim& d) const {
    int v = d.c;
    if (d.s1 >= 0) v += slot[d.s1];
    if (d.s2 >= 0) v += slot[d.s2];
    if (d.mc >= 0) v = std::min(v, d.mc + (d.ms >= 0 ? slot[d.ms] : 0));
    return v;
  }
  double* ptr(const Ptr& p) const {
    if (p.arena < 0) return nullptr;
    double* b = base[p.arena] + p.off;
    if (p.ds >= 0) b += (int64_t)slot[p.ds] * p.dm;
    if (p.ds2 >= 0) b += (int64_t)slot[p.ds2] * p.dm2;
    return b;
  }
  static double op(const double* p, int ld, int t, int i, int j) {
    return t ? p[(int64_t)j * ld + i] : p[(int64_t)i * ld + j];
  }

  void gemm(const GemmOut& O, const GemmTerm* terms) {
    const int m = dimv(O.m);
    const int n = O.clampn ? std::min(dimv(O.n), GEMM_MAXTILE) : dimv(O.n);
    if (m <= 0 || n <= 0) return;
    if (m > GEMM_MAXTILE || n > GEMM_MAXTILE) {
      err = -9;
      return;
    }
    std::vector<double> acc((size_t)m * n, 0.0);
    for (int ti = O.t0; ti < O.t1; ++ti) {
      const GemmTerm& T = terms[ti];
      double alpha = T.alpha;
      if (T.scale_idx >= 0) alpha *= scal[T.scale_idx];
      const double* A = ptr(T.a);
      const double* B = ptr(T.b);
      const double* C = ptr(T.c);
      if (!B) {
        for (int i = 0; i < m; ++i)
          for (int j = 0; j < n; ++j) acc[(size_t)i * n + j] += alpha * op(A, T.lda, T.ta, i, j);
        continue;
      }
      const int k1 = dimv(T.k1);
      const int nn = C ? dimv(T.k2) : n;
      std::vector<double> t((size_t)m * nn, 0.0);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < nn; ++j) {
          double s = 0.0;
          for (int l = 0; l < k1; ++l) s += op(A, T.lda, T.ta, i, l) * op(B, T.ldb, T.tb, l, j);
          t[(size_t)i * nn + j] = s;
        }
      if (!C) {
        for (size_t e = 0; e < acc.size(); ++e) acc[e] += alpha * t[e];
        continue;
      }
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
          double s = 0.0;
          for (int l = 0; l < nn; ++l) s += t[(size_t)i * nn + l] * op(C, T.ldc, T.tc, l, j);
          acc[(size_t)i * n + j] += alpha * s;
        }
    }
    double* o = ptr(O.o);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < n; ++j) {
        double& r = o[(int64_t)i * O.ldo + j];
        r = O.beta ? r + acc[(size_t)i * n + j] : acc[(size_t)i * n + j];
      }
  }

  void copy(const CopyJob& J) {
    const int rows = dimv(J.rows), cols = dimv(J.cols);
    const int zr = std::max(rows, dimv(J.zrows)), zc = std::max(cols, dimv(J.zcols));
    const double* S = ptr(J.src);
    double* D = ptr(J.dst);
    double alpha = J.alpha;
    if (J.scale_idx >= 0) alpha *= scal[J.scale_idx];
    for (int i = 0; i < zr; ++i)
      for (int j = 0; j < zc; ++j) {
        double v = 0.0;
        if (S && i < rows && j < cols) v = alpha * (J.trans ? S[(int64_t)j * J.lds + i] : S[(int64_t)i * J.lds + j]);
        D[(int64_t)i * J.ldd + j] = v;
      }
  }

  // Householder QR of the column-major rows x cols matrix, with the column
  // pivoting (largest remaining norm first) when the job asks for it, and the
  // pivoted factorisation stopped once the trailing columns fall below the
  // job's noise floor (squared Frobenius norm <= floor * ||a||_F^2).
  long qr_truncated = 0;  // pivoted QRs stopped at the noise floor
  void qr(const QrJob& J) {
    const int rows = dimv(J.rows), cols = dimv(J.cols);
    double* a = ptr(J.a);
    double* tau = ptr(J.tau);
    const int lda = J.lda;
    int q = std::min(std::max(rows, 0), std::max(cols, 0));
    int* piv = reinterpret_cast<int*>(ptr(J.piv));
    if (piv)
      for (int c = 0; c < cols; ++c) piv[c] = c;
    double thr = -1.0;
    if (piv && J.trunc_idx >= 0) {
      double fro = 0.0;
      for (int c = 0; c < cols; ++c)
        for (int i = 0; i < rows; ++i) fro += a[(int64_t)c * lda + i] * a[(int64_t)c * lda + i];
      thr = scal[J.trunc_idx] * fro;
    }
    for (int j = 0; j < q; ++j) {
      if (piv) {
        int p = j;
        double best = -1.0, rest = 0.0;
        for (int c = j; c < cols; ++c) {
          double s2 = 0.0;
          for (int i = j; i < rows; ++i) s2 += a[(int64_t)c * lda + i] * a[(int64_t)c * lda + i];
          rest += s2;
          if (s2 > best) {
            best = s2;
            p = c;
          }
        }
        if (thr >= 0.0 && rest <= thr) {
          ++qr_truncated;
          for (int c = j; c < q; ++c)
            if (tau) tau[c] = 0.0;
          q = j;
          break;
        }
        if (p != j) {
          for (int i = 0; i < rows; ++i) std::swap(a[(int64_t)j * lda + i], a[(int64_t)p * lda + i]);
          std::swap(piv[j], piv[p]);
        }
      }
      double* col = a + (int64_t)j * lda;
      double s2 = 0.0;
      for (int i = j + 1; i < rows; ++i) s2 += col[i] * col[i];
      double t = 0.0;
      if (s2 > 0.0) {
        const double alpha = col[j];
        const double beta = -std::copysign(std::sqrt(alpha * alpha + s2), alpha);
        t = (beta - alpha) / beta;
        const double sc = 1.0 / (alpha - beta);
        for (int i = j + 1; i < rows; ++i) col[i] *= sc;
        col[j] = beta;
        for (int c = j + 1; c < cols; ++c) {
          double* cc = a + (int64_t)c * lda;
          double p = cc[j];
          for (int i = j + 1; i < rows; ++i) p += col[i] * cc[i];
          const double w = t * p;
          cc[j] -= w;
          for (int i = j + 1; i < rows; ++i) cc[i] -= w * col[i];
        }
      }
      if (tau) tau[j] = t;
    }
    if (J.rank_slot >= 0) slot[J.rank_slot] = q;
    double* r = ptr(J.r);
    if (r)
      for (int i = 0; i < cols; ++i)
        for (int c = 0; c < cols; ++c) {
          const double v = (c >= i && i < q) ? a[(int64_t)c * lda + i] : 0.0;
          const int dc = ((J.rmode & 1) && piv) ? piv[c] : c;  // R P^T: original column order
          if (J.rmode & 2) r[(int64_t)dc * J.ldr + i] = v;      // transposed store
          else r[(int64_t)i * J.ldr + dc] = v;
        }
  }

  void qapply(const QApplyJob& J) {
    const int rows = dimv(J.rows), q = dimv(J.q), nc = dimv(J.ncols);
    const double* a = ptr(J.a);
    const double* tau = ptr(J.tau);
    const double* y = ptr(J.y);
    double* out = ptr(J.out);
    for (int i = 0; i < rows; ++i)
      for (int c = 0; c < nc; ++c) out[(int64_t)i * J.ldo + c] = i < q ? y[(int64_t)i * J.ldy + c] : 0.0;
    for (int j = std::min(q, rows) - 1; j >= 0; --j) {
      const double t = tau[j];
      if (t == 0.0) continue;
      const double* v = a + (int64_t)j * J.lda;
      for (int c = 0; c < nc; ++c) {
        double p = out[(int64_t)j * J.ldo + c];
        for (int i = j + 1; i < rows; ++i) p += v[i] * out[(int64_t)i * J.ldo + c];
        const double w = t * p;
        out[(int64_t)j * J.ldo + c] -= w;
        for (int i = j + 1; i < rows; ++i) out[(int64_t)i * J.ldo + c] -= w * v[i];
      }
    }
  }

  // Cyclic one-sided Jacobi on M (rows x cols); columns below the noise floor
  // (sqrt(scal[PARAM_SVD_FLOOR]) ||M||_F) count as zero.  Writes sigma (sorted), U (rows permuted by the job's
  // pivot order) and the rank of the job's truncation mode.
  void svd(const SvdJob& J) {
    const int rows = dimv(J.rows), cols = dimv(J.cols);
    int* rank_out = J.rank_slot >= 0 ? &slot[J.rank_slot] : nullptr;
    if (rows <= 0 || cols <= 0) {
      if (rank_out) *rank_out = 0;
      if (J.norm_idx >= 0) nrm[J.norm_idx] = scal[J.norm_idx] = 0.0;
      return;
    }
    const double* S = ptr(J.src);
    std::vector<double> M((size_t)rows * cols);
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c)
        M[(size_t)c * rows + r] = J.trans ? S[(int64_t)c * J.lds + r] : S[(int64_t)r * J.lds + c];
    double fro = 0.0;
    for (double v : M) fro += v * v;
    const double tiny2 = fro * scal[PARAM_SVD_FLOOR];
    bool converged = false;
    const int maxsweep = scal[PARAM_SVD_SWEEPS] >= 1.0 ? (int)scal[PARAM_SVD_SWEEPS] : 60;
    for (int sweep = 0; sweep < maxsweep && !converged; ++sweep) {
      converged = true;
      for (int i = 0; i < cols; ++i)
        for (int j = i + 1; j < cols; ++j) {
          double* mi = &M[(size_t)i * rows];
          double* mj = &M[(size_t)j * rows];
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int r = 0; r < rows; ++r) {
            al += mi[r] * mi[r];
            be += mj[r] * mj[r];
            ga += mi[r] * mj[r];
          }
          if (ga == 0.0 || al <= tiny2 || be <= tiny2 || std::fabs(ga) <= 2.5e-15 * std::sqrt(al) * std::sqrt(be))
            continue;
          const double zeta = (be - al) / (2.0 * ga);
          const double t = std::copysign(1.0, zeta) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
          for (int r = 0; r < rows; ++r) {
            const double u = mi[r], v = mj[r];
            mi[r] = c * u - s * v;
            mj[r] = s * u + c * v;
          }
          converged = false;
        }
      if (!converged && sweep == maxsweep - 1) err = -5;
    }
    std::vector<double> sn(cols);
    std::vector<int> pos(cols);
    for (int c = 0; c < cols; ++c) {
      double s = 0.0;
      for (int r = 0; r < rows; ++r) s += M[(size_t)c * rows + r] * M[(size_t)c * rows + r];
      sn[c] = s > tiny2 ? std::sqrt(s) : 0.0;
    }
    for (int c = 0; c < cols; ++c) {
      int p = 0;
      for (int l = 0; l < cols; ++l) p += (sn[l] > sn[c]) || (sn[l] == sn[c] && l < c);
      pos[c] = p;
    }
    double* sig = ptr(J.sig);
    if (sig)
      for (int c = 0; c < cols; ++c) sig[pos[c]] = sn[c];
    const int* upiv = reinterpret_cast<const int*>(ptr(J.piv));
    double* U = ptr(J.u);
    if (U)
      for (int r = 0; r < rows; ++r)
        for (int c = 0; c < cols; ++c)
          U[(int64_t)(upiv ? upiv[r] : r) * J.ldu + pos[c]] = sn[c] > 0.0 ? M[(size_t)c * rows + r] / sn[c] : 0.0;
    const double s0 = *std::max_element(sn.begin(), sn.end());
    const double tol = J.tol_idx >= 0 ? J.tol * scal[J.tol_idx] : J.tol;
    int k = 0;
    if (J.mode == 1)
      for (double v : sn) k += v > tol;
    if (J.mode == 2 && s0 > 0.0)
      for (double v : sn) k += v > tol * s0;
    if (J.norm_idx >= 0) {
      nrm[J.norm_idx] = s0;
      scal[J.norm_idx] = s0 > 0.0 ? 1.0 / s0 : 0.0;
    }
    if (J.mode == 1 || J.mode == 2) {
      if (k > J.cap) {
        err = -7;
        k = J.cap;
      }
      if (rank_out) *rank_out = k;
    }
  }

  void norm(const NormJob& N) {
    SvdJob J{};
    J.src = N.src;
    J.lds = N.lds;
    J.rows = N.n;
    J.cols = N.n;
    J.mode = 4;
    J.norm_idx = N.norm_idx;
    J.rank_slot = -1;
    J.tol_idx = -1;
    J.u = J.sig = J.piv = Ptr{0, AR_NONE, -1, 0, -1, 0};
    svd(J);
  }

  void scan(const ScanJob& J) {
    int s = 0;
    for (int i = 0; i < J.count; ++i) {
      slot[J.out + i] = s;
      s += slot[idx[J.idx_off + i]];
    }
    slot[J.out + J.count] = s;
  }

  void run(const Plan& P) {
    for (const Stage& st : P.stages)
      for (int j = 0; j < st.count; ++j) switch (st.kind) {
          case ST_GEMM: gemm(P.gout[st.first + j], P.gterm.data()); break;
          case ST_COPY: copy(P.copy[st.first + j]); break;
          case ST_QR: qr(P.qr[st.first + j]); break;
          case ST_QAPPLY: qapply(P.qap[st.first + j]); break;
          case ST_SVD: svd(P.svd[st.first + j]); break;
          case ST_SCAN: scan(P.scan[st.first + j]); break;
          case ST_NORM: norm(P.norm[st.first + j]); break;
          default: break;
        }
  }
};

// V_t of every level in cluster order: out[l][row] = (level-l basis row), the
// explicit level bases the planner reads (VF / WF).
std::vector<double> level_bases(const Tree& T, int k, const double* V, const double* E) {
  std::vector<double> out((size_t)(T.depth + 1) * T.n * k);
  std::memcpy(&out[(size_t)T.depth * T.n * k], V, sizeof(double) * T.n * k);
  for (int l = T.depth - 1; l >= 0; --l)
    for (int c = Tree::first(l + 1); c < Tree::first(l + 2); ++c)
      for (int i = 0; i < T.size[c]; ++i) {
        const int row = T.off[c] + i;
        for (int b = 0; b < k; ++b) {
          double s = 0.0;
          for (int a = 0; a < k; ++a)
            s += out[((size_t)(l + 1) * T.n + row) * k + a] * E[((size_t)c * k + a) * k + b];
          out[((size_t)l * T.n + row) * k + b] = s;
        }
      }
  return out;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 19 && argc != 20) {
    std::fprintf(stderr, "usage: see the header of stage_interpreter.cpp\n");
    return 2;
  }
  const int n = std::atoi(argv[2]), dim = std::atoi(argv[3]), leaf = std::atoi(argv[4]), order = std::atoi(argv[5]);
  const double eta = std::atof(argv[6]), eps = std::atof(argv[7]);
  const int kindA = std::atoi(argv[8]);
  const double kpA[4] = {std::atof(argv[9]), std::atof(argv[10]), std::atof(argv[11]), 0.0};
  const int kindB = std::atoi(argv[12]);
  const double kpB[4] = {std::atof(argv[13]), std::atof(argv[14]), std::atof(argv[15]), 0.0};
  const int max_rank = std::atoi(argv[16]);
  const bool hmatrix = std::atoi(argv[17]) != 0;
  std::vector<double> pts((size_t)n * dim);
  FILE* f = std::fopen(argv[1], "rb");
  if (!f || std::fread(pts.data(), 8, pts.size(), f) != pts.size()) return 3;
  std::fclose(f);

  Tree T;
  build_cluster_tree(pts.data(), n, dim, leaf, T);
  BlockTree BT;
  build_block_tree(T, T, eta, BT);
  HostH2 HA, HB;
  assemble_chebyshev(pts.data(), T, BT, order, kindA, kpA, HA);
  assemble_chebyshev(pts.data(), T, BT, order, kindB, kpB, HB);
  const int k = HA.k;
  auto describe = [&](HostH2& H, std::vector<double>& arena, MatDesc& d) {
    d.rows = &T;
    d.cols = &T;
    d.blocks = &BT;
    d.k = k;
    const std::vector<double> VF = level_bases(T, k, H.V.data(), H.E.data());
    d.off_V = 0;
    d.off_E = (int64_t)H.V.size();
    d.off_S = d.off_E + (int64_t)H.E.size();
    d.off_N = d.off_S + (int64_t)H.S.size();
    d.off_VF = d.off_N + (int64_t)H.N.size();
    d.off_W = d.off_V;
    d.off_F = d.off_E;
    d.off_WF = d.off_VF;
    arena.resize(d.off_VF + VF.size());
    std::copy(H.V.begin(), H.V.end(), arena.begin());
    std::copy(H.E.begin(), H.E.end(), arena.begin() + d.off_E);
    std::copy(H.S.begin(), H.S.end(), arena.begin() + d.off_S);
    std::copy(H.N.begin(), H.N.end(), arena.begin() + d.off_N);
    std::copy(VF.begin(), VF.end(), arena.begin() + d.off_VF);
  };
  std::vector<double> arX, arY;
  MatDesc dX, dY;
  describe(HA, arX, dX);
  describe(HB, arY, dY);
  MulOptions mo;
  mo.eta = eta;
  mo.theta = 0.25;
  mo.max_rank = max_rank;
  mo.hmatrix = hmatrix;
  auto P = make_product_plan(dX, dY, mo);

  for (const auto& kv : P->stats) std::printf("stat %s %lld\n", kv.first.c_str(), (long long)kv.second);
  Interp E;
  std::vector<double> ws(std::max<int64_t>(P->ws_len, 1), std::nan("")), fac(std::max<int64_t>(P->fac_len, 1), std::nan(""));
  std::vector<double> arC(std::max<int64_t>(P->c_len, 1), 0.0), kon(P->konst);
  E.base[AR_WS] = ws.data();
  E.base[AR_X] = arX.data();
  E.base[AR_Y] = arY.data();
  E.base[AR_C] = arC.data();
  E.base[AR_K] = kon.data();
  E.base[AR_F] = fac.data();
  E.slot = P->slot_init;
  E.scal.assign(P->nscal, 0.0);
  E.nrm.assign(P->nscal, 0.0);
  E.idx = P->idx;
  E.scal[PARAM_TOL_BASIS] = eps / 4.0 * std::sqrt(1.0 - 2.0 * 0.25);
  E.scal[PARAM_TOL_AGG] = eps / 3.0;
  // noise floor of the FP64 form: eps 2^-20 within [2^-50, 2^-40], squared
  const double fl = eps > 0.0 ? std::min(std::ldexp(1.0, -40), std::max(std::ldexp(1.0, -50), eps * std::ldexp(1.0, -20)))
                              : std::ldexp(1.0, -50);
  E.scal[PARAM_SVD_FLOOR] = fl * fl;
  E.scal[PARAM_SVD_SWEEPS] = argc > 19 ? std::atof(argv[19]) : 0.0;
  E.run(*P);
  if (E.err != 0) {
    std::fprintf(stderr, "interpreter error %d\n", E.err);
    return 4;
  }
  std::printf("stat qr_truncated %ld\n", E.qr_truncated);
  // largest dynamic shared memory a QR / SVD stage asks for, largest norm n
  int smem_qr = 0, smem_svd = 0, norm_n = 0;
  for (const Stage& st : P->stages) {
    if (st.kind == ST_QR) smem_qr = std::max(smem_qr, st.smem);
    if (st.kind == ST_SVD) smem_svd = std::max(smem_svd, st.smem);
    if (st.kind == ST_NORM) norm_n = std::max(norm_n, st.aux);
  }
  std::printf("stat smem_max_qr %d\nstat smem_max_svd %d\nstat norm_max_n %d\n", smem_qr, smem_svd, norm_n);

  // dense expansion in the caller's ordering
  const BlockTree& BC = *P->cblocks;
  std::vector<double> Dn((size_t)n * n, 0.0);
  auto put = [&](int t, int s, int i, int j, double v) {
    Dn[(size_t)T.perm[T.off[t] + i] * n + T.perm[T.off[s] + j]] = v;
  };
  if (hmatrix) {
    for (size_t a = 0; a < BC.adm_list.size(); ++a) {
      const int b = BC.adm_list[a], t = BC.t[b], s = BC.s[b], w = P->hm_w[a];
      const double* L = arC.data() + P->hm_off_L[a];
      const double* R = arC.data() + P->hm_off_R[a];
      for (int i = 0; i < T.size[t]; ++i)
        for (int j = 0; j < T.size[s]; ++j) {
          double v = 0.0;
          for (int q = 0; q < w; ++q) v += L[(size_t)i * w + q] * R[(size_t)j * w + q];
          put(t, s, i, j, v);
        }
    }
  } else {
    const int KP = P->kpad;
    const std::vector<double> VF = level_bases(T, KP, arC.data() + P->c_off_V, arC.data() + P->c_off_E);
    const std::vector<double> WF = level_bases(T, KP, arC.data() + P->c_off_W, arC.data() + P->c_off_F);
    for (size_t a = 0; a < BC.adm_list.size(); ++a) {
      const int b = BC.adm_list[a], t = BC.t[b], s = BC.s[b];
      const double* S = arC.data() + P->c_off_S + (size_t)a * KP * KP;
      for (int i = 0; i < T.size[t]; ++i) {
        const double* v = &VF[((size_t)T.level[t] * n + T.off[t] + i) * KP];
        std::vector<double> vs(KP, 0.0);
        for (int p = 0; p < KP; ++p)
          for (int q = 0; q < KP; ++q) vs[q] += v[p] * S[p * KP + q];
        for (int j = 0; j < T.size[s]; ++j) {
          const double* wr = &WF[((size_t)T.level[s] * n + T.off[s] + j) * KP];
          double sum = 0.0;
          for (int q = 0; q < KP; ++q) sum += vs[q] * wr[q];
          put(t, s, i, j, sum);
        }
      }
    }
  }
  for (size_t a = 0; a < BC.inadm_list.size(); ++a) {
    const int b = BC.inadm_list[a], t = BC.t[b], s = BC.s[b];
    const double* N = arC.data() + P->c_off_N + BC.near_off[a];
    for (int i = 0; i < T.size[t]; ++i)
      for (int j = 0; j < T.size[s]; ++j) put(t, s, i, j, N[(size_t)i * T.size[s] + j]);
  }
  FILE* o = std::fopen(argv[18], "wb");
  if (!o) return 5;
  std::fwrite(Dn.data(), 8, Dn.size(), o);
  if (!hmatrix) {
    std::vector<int> rr(T.ncl), rc(T.ncl);
    for (int c = 0; c < T.ncl; ++c) {
      rr[c] = E.slot[P->rank_row_slot[c]];
      rc[c] = E.slot[P->rank_col_slot[c]];
    }
    std::fwrite(rr.data(), 4, rr.size(), o);
    std::fwrite(rc.data(), 4, rc.size(), o);
  }
  std::fclose(o);
  return 0;
}
