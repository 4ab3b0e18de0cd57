// Host-side 1D tables of the discretisation.  Compiled with -ffp-contract=off: every value
// here is an exact function of the stated operation order, because the device computes the
// graph (face normals, coupling blocks, edge weights) from these tables and the graph must
// be reproducible bit for bit.
#include <cmath>
#include <stdexcept>
#include "common.h"

namespace sn {

static const int NEWTON_STEPS = 100;

// n-point Gauss-Legendre rule on [0,1] (Sec. 2: Gauss-Legendre quadrature of the element
// integrals).  Newton on P_n from x_i = cos(pi (i + 3/4) / (n + 1/2)), a fixed number of
// steps; recurrence P_k = ((2k-1) x P_{k-1} - (k-1) P_{k-2}) / k, P_n' = n (x P_n - P_{n-1})
// / (x^2 - 1).  t = (1 - x)/2 ascending, w = 1 / ((1 - x^2) P_n'^2).
void gauss_legendre(int n, std::vector<double>& t, std::vector<double>& w) {
  t.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int step = 0; step <= NEWTON_STEPS; ++step) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      if (step < NEWTON_STEPS) x = x - p1 / dp;
    }
    t[i] = 0.5 * (1.0 - x);
    w[i] = 1.0 / ((1.0 - x * x) * dp * dp);
  }
}

// Gauss-Lobatto-Legendre nodes of order p on [0,1]: the DG nodal basis.
void gll_nodes(int p, std::vector<double>& x) {
  if (p == 1) {
    x = {0.0, 1.0};
  } else if (p == 2) {
    x = {0.0, 0.5, 1.0};
  } else if (p == 3) {
    double a = 1.0 / std::sqrt(5.0);
    x = {0.0, 0.5 * (1.0 - a), 0.5 * (1.0 + a), 1.0};
  } else {
    throw std::invalid_argument("DG order p must be 1, 2 or 3");
  }
}

// l_j(x) = prod_{k != j} (x - n_k)/(n_j - n_k), left to right from 1.0.
double lagrange(const double* nodes, int n, int j, double x) {
  double v = 1.0;
  for (int k = 0; k < n; ++k)
    if (k != j) v = v * ((x - nodes[k]) / (nodes[j] - nodes[k]));
  return v;
}

// l_j'(x) = sum_{k != j} 1/(n_j - n_k) prod_{l != j,k} (x - n_l)/(n_j - n_l).
double lagrange_deriv(const double* nodes, int n, int j, double x) {
  double d = 0.0;
  for (int k = 0; k < n; ++k) {
    if (k == j) continue;
    double t = 1.0 / (nodes[j] - nodes[k]);
    for (int l = 0; l < n; ++l)
      if (l != j && l != k) t = t * ((x - nodes[l]) / (nodes[j] - nodes[l]));
    d = d + t;
  }
  return d;
}

// product over axes k (left to right from 1.0) of l_{idx_k}(x_k), or l' on deriv_axis.
static double tensor_value(const double* nodes, int n, const int* idx, const double* x, int dim, int deriv_axis) {
  double v = 1.0;
  for (int k = 0; k < dim; ++k)
    v = v * (k == deriv_axis ? lagrange_deriv(nodes, n, idx[k], x[k]) : lagrange(nodes, n, idx[k], x[k]));
  return v;
}

void build_tables(Tables& T, int dim, int p, int r) {
  T.dim = dim;
  T.p = p;
  T.r = r;
  T.nv = p + (dim * r + 1) / 2;
  T.nf = p + r;
  T.N = 1;
  T.Nf = 1;
  T.Nv = 1;
  T.Q = 1;
  for (int k = 0; k < dim; ++k) {
    T.N *= p + 1;
    T.Nv *= r + 1;
    T.Q *= T.nv;
  }
  for (int k = 0; k < dim - 1; ++k) T.Nf *= p + 1;
  gauss_legendre(T.nv, T.glv_t, T.glv_w);
  gauss_legendre(T.nf, T.glf_t, T.glf_w);
  gll_nodes(p, T.gll);
  T.geo.resize(r + 1);
  for (int a = 0; a <= r; ++a) T.geo[a] = (double)a / r;
  T.wq.assign(T.Q, 0.0);
  T.B.assign((size_t)T.Q * T.N, 0.0);
  T.dB.assign((size_t)T.Q * T.N * dim, 0.0);
  T.dV.assign((size_t)T.Q * T.Nv * dim, 0.0);
  T.V.assign((size_t)T.Q * T.Nv, 0.0);
  for (int q = 0; q < T.Q; ++q) {
    int qi[3];
    double x[3];
    double w = 1.0;
    for (int k = 0, rem = q; k < dim; ++k, rem /= T.nv) {
      qi[k] = rem % T.nv;
      x[k] = T.glv_t[qi[k]];
      w = w * T.glv_w[qi[k]];
    }
    T.wq[q] = w;
    for (int m = 0; m < T.N; ++m) {
      int mi[3];
      for (int k = 0, rem = m; k < dim; ++k, rem /= (p + 1)) mi[k] = rem % (p + 1);
      T.B[(size_t)q * T.N + m] = tensor_value(T.gll.data(), p + 1, mi, x, dim, -1);
      for (int j = 0; j < dim; ++j)
        T.dB[((size_t)q * T.N + m) * dim + j] = tensor_value(T.gll.data(), p + 1, mi, x, dim, j);
    }
    for (int m = 0; m < T.Nv; ++m) {
      int mi[3];
      for (int k = 0, rem = m; k < dim; ++k, rem /= (r + 1)) mi[k] = rem % (r + 1);
      for (int j = 0; j < dim; ++j)
        T.dV[((size_t)q * T.Nv + m) * dim + j] = tensor_value(T.geo.data(), r + 1, mi, x, dim, j);
      T.V[(size_t)q * T.Nv + m] = tensor_value(T.geo.data(), r + 1, mi, x, dim, -1);
    }
  }
}

}  // namespace sn
