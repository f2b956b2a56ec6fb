// Host FP64 assembly of a Chebyshev H^2-matrix for the CPU stage interpreter
// (test infrastructure; the library assembles on the device).  Leaf bases
// V_t(i, nu) = ell_{t,nu}(x_i), transfer matrices E_{t'}(nu', nu) =
// ell_{t,nu}(xi_{t',nu'}), couplings S_ts = g(xi_t, xi_s) and the dense
// nearfield g(x_i, x_j) with the prescribed diagonal value (eq. (3), Section 2).
#include "host_assembly.h"

#include <cmath>

using h2::BlockTree;
using h2::Tree;

namespace h2host {

namespace {

struct Interp {
  int m, dim, k;
  std::vector<double> nodes;  // ncl x dim x m
  double* nd(int c, int a) { return &nodes[((size_t)c * dim + a) * m]; }
};

void make_interp(const Tree& T, int order, Interp& I) {
  I.m = order;
  I.dim = T.dim;
  I.k = 1;
  for (int a = 0; a < T.dim; ++a) I.k *= order;
  I.nodes = h2::chebyshev_nodes(T, order);
}

// ell_{c,nu}(p) for one point p (dim coordinates) -> out[k]
void lagrange(Interp& I, int c, const double* p, double* out) {
  double l1[3][16];
  for (int a = 0; a < I.dim; ++a) {
    const double* x = I.nd(c, a);
    for (int j = 0; j < I.m; ++j) {
      double v = 1.0;
      for (int i = 0; i < I.m; ++i)
        if (i != j) v *= (p[a] - x[i]) / (x[j] - x[i]);
      l1[a][j] = v;
    }
  }
  for (int nu = 0; nu < I.k; ++nu) {
    int r = nu;
    double v = 1.0;
    for (int a = 0; a < I.dim; ++a) {
      v *= l1[a][r % I.m];
      r /= I.m;
    }
    out[nu] = v;
  }
}

void interp_point(Interp& I, int c, int nu, double* p) {
  int r = nu;
  for (int a = 0; a < I.dim; ++a) {
    p[a] = I.nd(c, a)[r % I.m];
    r /= I.m;
  }
}

}  // namespace

double kernel_value(int kind, const double* kp, const double* x, const double* y, int dim) {
  double r2 = 0.0;
  for (int a = 0; a < dim; ++a) {
    const double d = x[a] - y[a];
    r2 += d * d;
  }
  switch (kind) {
    case 0: return -kp[0] * 0.5 * std::log(r2);
    case 1: return kp[0] / std::sqrt(r2);
    case 2: return kp[0] * std::exp(-r2 / kp[2]);
    default: return kp[0] * std::exp(-std::sqrt(r2) / kp[2]);
  }
}

void assemble_chebyshev(const double* pts, const Tree& T, const BlockTree& B, int order, int kind,
                        const double* kp, HostH2& out) {
  Interp I;
  make_interp(T, order, I);
  const int k = I.k, dim = T.dim;
  out.k = k;
  out.V.assign((size_t)T.n * k, 0.0);
  out.E.assign((size_t)T.ncl * k * k, 0.0);
  for (int l = 0, c = Tree::first(T.depth); l < T.count(T.depth); ++l, ++c)
    for (int i = 0; i < T.size[c]; ++i) {
      const int64_t row = T.off[c] + i;
      lagrange(I, c, pts + T.perm[row] * dim, &out.V[(size_t)row * k]);
    }
  double p[3];
  for (int c = 1; c < T.ncl; ++c) {
    const int par = Tree::parent(c);
    for (int nu2 = 0; nu2 < k; ++nu2) {  // E_c(nu', nu) = ell_{parent,nu}(xi_{c,nu'})
      interp_point(I, c, nu2, p);
      lagrange(I, par, p, &out.E[((size_t)c * k + nu2) * k]);
    }
  }
  out.S.assign((size_t)B.adm_list.size() * k * k, 0.0);
  double q[3];
  for (size_t a = 0; a < B.adm_list.size(); ++a) {
    const int b = B.adm_list[a];
    for (int nu = 0; nu < k; ++nu) {
      interp_point(I, B.t[b], nu, p);
      for (int mu = 0; mu < k; ++mu) {
        interp_point(I, B.s[b], mu, q);
        out.S[(a * k + nu) * k + mu] = kernel_value(kind, kp, p, q, dim);
      }
    }
  }
  out.N.assign((size_t)B.near_total, 0.0);
  for (size_t a = 0; a < B.inadm_list.size(); ++a) {
    const int b = B.inadm_list[a];
    const int t = B.t[b], s = B.s[b];
    double* dst = &out.N[B.near_off[a]];
    for (int i = 0; i < T.size[t]; ++i) {
      const int64_t oi = T.perm[T.off[t] + i];
      for (int j = 0; j < T.size[s]; ++j) {
        const int64_t oj = T.perm[T.off[s] + j];
        dst[(size_t)i * T.size[s] + j] = (oi == oj) ? kp[1] : kernel_value(kind, kp, pts + oi * dim, pts + oj * dim, dim);
      }
    }
  }
}

}  // namespace h2host
