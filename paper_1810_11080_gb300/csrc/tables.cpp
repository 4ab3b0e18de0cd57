// Host-side 1D tables of the discretisation.  Compiled with -ffp-contract=off: every value
// here is an exact function of the stated operation order, because the device computes the
// graph (face normals, coupling blocks, edge weights) from these tables and the graph must
// be reproducible bit for bit.
#include <algorithm>
#include <cmath>
#include <stdexcept>
#include <utility>
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

// ------------------------------------------------------------------ triangles
// Reference triangle {xi, eta >= 0, xi + eta <= 1}; an order-k node set is v0 = (0,0), v1 = (1,0),
// v2 = (0,1), the k - 1 interior nodes of the faces f0 = v0 v1, f1 = v1 v2, f2 = v2 v0 (at the 1D
// positions pos[1..k-1] along each face), then (k = 3) the centroid.  Its Lagrange basis (total
// degree k) is evaluated through the monomials x^a y^b (a + b <= k) and the inverse Vandermonde
// matrix.  Geometry: P_r on the equispaced positions a/r; DG: P_p on the GLL positions, whose
// restriction to a face is the 1D Lagrange basis of those positions.
namespace {

void tri_nodes(int k, const std::vector<double>& pos, std::vector<double>& xy) {
  const double V[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
  xy.clear();
  for (int i = 0; i < 3; ++i) {
    xy.push_back(V[i][0]);
    xy.push_back(V[i][1]);
  }
  for (int f = 0; f < 3; ++f) {
    const double* A = V[f];
    const double* B = V[(f + 1) % 3];
    for (int j = 1; j < k; ++j) {
      xy.push_back(A[0] + pos[j] * (B[0] - A[0]));
      xy.push_back(A[1] + pos[j] * (B[1] - A[1]));
    }
  }
  if (k == 3) {
    xy.push_back(1.0 / 3.0);
    xy.push_back(1.0 / 3.0);
  }
}

// Monomial exponents (a, b), total degree 0..k, a descending within a degree.
void tri_monomials(int k, std::vector<int>& ea, std::vector<int>& eb) {
  ea.clear();
  eb.clear();
  for (int d = 0; d <= k; ++d)
    for (int a = d; a >= 0; --a) {
      ea.push_back(a);
      eb.push_back(d - a);
    }
}

double ipow_d(double x, int a) {
  double v = 1.0;
  for (int i = 0; i < a; ++i) v *= x;
  return v;
}

// Inverse of the n x n matrix A (row-major) by Gauss-Jordan elimination with partial pivoting.
void invert(int n, std::vector<double> A, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int rr = c + 1; rr < n; ++rr)
      if (std::fabs(A[rr * n + c]) > std::fabs(A[piv * n + c])) piv = rr;
    if (A[piv * n + c] == 0.0) throw std::runtime_error("singular Vandermonde matrix");
    for (int j = 0; j < n; ++j) {
      std::swap(A[c * n + j], A[piv * n + j]);
      std::swap(inv[c * n + j], inv[piv * n + j]);
    }
    const double d = A[c * n + c];
    for (int j = 0; j < n; ++j) {
      A[c * n + j] /= d;
      inv[c * n + j] /= d;
    }
    for (int rr = 0; rr < n; ++rr) {
      if (rr == c) continue;
      const double m = A[rr * n + c];
      if (m == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[rr * n + j] -= m * A[c * n + j];
        inv[rr * n + j] -= m * inv[c * n + j];
      }
    }
  }
}

// Coefficients C [n_mono][n_nodes] (column i = basis function of node i) of the Lagrange basis.
void tri_basis(int k, const std::vector<double>& xy, std::vector<double>& C) {
  std::vector<int> ea, eb;
  tri_monomials(k, ea, eb);
  const int n = (int)ea.size();
  std::vector<double> V((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < n; ++m) V[i * n + m] = ipow_d(xy[2 * i], ea[m]) * ipow_d(xy[2 * i + 1], eb[m]);
  invert(n, V, C);
}

// value and gradient of basis function i at (x, y)
void tri_eval(int k, const std::vector<double>& C, int i, double x, double y, double& v, double& gx, double& gy) {
  std::vector<int> ea, eb;
  tri_monomials(k, ea, eb);
  const int n = (int)ea.size();
  v = gx = gy = 0.0;
  for (int m = 0; m < n; ++m) {
    const double c = C[m * n + i];
    v += c * ipow_d(x, ea[m]) * ipow_d(y, eb[m]);
    if (ea[m] > 0) gx += c * ea[m] * ipow_d(x, ea[m] - 1) * ipow_d(y, eb[m]);
    if (eb[m] > 0) gy += c * eb[m] * ipow_d(x, ea[m]) * ipow_d(y, eb[m] - 1);
  }
}

}  // namespace

// Tables of a triangle problem: collapsed Gauss volume rule (xi = u, eta = v (1 - u), weight
// (w_i w_j) (1 - u_i), n_v = p + r points per direction, point q = i + n_v j); face rule n_f =
// p + r Gauss points per piece as for the tensor elements; DG (P_p) and geometry (P_r) bases at
// the volume points.
void build_tables_tri(Tables& T, int p, int r) {
  if (p < 1 || p > 3 || r < 1 || r > 3) throw std::invalid_argument("triangles: p and r must be 1..3");
  T.dim = 2;
  T.p = p;
  T.r = r;
  T.nv = p + r;
  T.nf = p + r;
  T.N = (p + 1) * (p + 2) / 2;
  T.Nf = p + 1;
  T.Nv = (r + 1) * (r + 2) / 2;
  T.Q = T.nv * T.nv;
  gauss_legendre(T.nv, T.glv_t, T.glv_w);
  gauss_legendre(T.nf, T.glf_t, T.glf_w);
  gll_nodes(p, T.gll);
  T.geo.resize(r + 1);
  for (int a = 0; a <= r; ++a) T.geo[a] = (double)a / r;
  std::vector<double> dgxy, gxy, Cd, Cg;
  tri_nodes(p, T.gll, dgxy);
  tri_nodes(r, T.geo, gxy);
  tri_basis(p, dgxy, Cd);
  tri_basis(r, gxy, Cg);
  T.wq.assign(T.Q, 0.0);
  T.B.assign((size_t)T.Q * T.N, 0.0);
  T.dB.assign((size_t)T.Q * T.N * 2, 0.0);
  T.dV.assign((size_t)T.Q * T.Nv * 2, 0.0);
  T.V.assign((size_t)T.Q * T.Nv, 0.0);
  for (int j = 0; j < T.nv; ++j)
    for (int i = 0; i < T.nv; ++i) {
      const int q = i + T.nv * j;
      const double u = T.glv_t[i], x = u, y = T.glv_t[j] * (1.0 - u);
      T.wq[q] = (T.glv_w[i] * T.glv_w[j]) * (1.0 - u);
      for (int m = 0; m < T.N; ++m) {
        double v, gx, gy;
        tri_eval(p, Cd, m, x, y, v, gx, gy);
        T.B[(size_t)q * T.N + m] = v;
        T.dB[((size_t)q * T.N + m) * 2 + 0] = gx;
        T.dB[((size_t)q * T.N + m) * 2 + 1] = gy;
      }
      for (int m = 0; m < T.Nv; ++m) {
        double v, gx, gy;
        tri_eval(r, Cg, m, x, y, v, gx, gy);
        T.V[(size_t)q * T.Nv + m] = v;
        T.dV[((size_t)q * T.Nv + m) * 2 + 0] = gx;
        T.dV[((size_t)q * T.Nv + m) * 2 + 1] = gy;
      }
    }
}

// ------------------------------------------------------------------ tetrahedra
// Straight-sided tetrahedra (P_1 geometry) with P_1 / P_2 DG bases in closed form (barycentrics
// l0 = ((1 - x) - y) - z, l1 = x, l2 = y, l3 = z; P_2: l ((2 l) - 1) at the vertices, (4 l_a) l_b at
// the edge midpoints (0,1), (1,2), (2,0), (0,3), (1,3), (2,3)), the same operation order as the
// reference formulas so that the mass matrices of the sigma-inverse weights agree bit for bit.
// Volume rule: collapsed Gauss, x = u, y = v (1 - u), z = (w (1 - u)) (1 - v), weight
// ((((w_i w_j) w_k) (1 - u)) (1 - u)) (1 - v), n_v = p + 2 points per direction, q = i + n (j + n k);
// faces: the collapsed triangle rule with n_f = p + 1 points per direction.
namespace {

void tet_eval(int p, double x, double y, double z, double* v, double (*g)[3]) {
  const double l[4] = {((1.0 - x) - y) - z, x, y, z};
  const double gl[4][3] = {{-1.0, -1.0, -1.0}, {1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
  const int E[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};
  if (p == 1) {
    for (int i = 0; i < 4; ++i) {
      v[i] = l[i];
      for (int k = 0; k < 3; ++k) g[i][k] = gl[i][k] * 1.0;
    }
    return;
  }
  for (int i = 0; i < 4; ++i) {
    v[i] = l[i] * ((2.0 * l[i]) - 1.0);
    for (int k = 0; k < 3; ++k) g[i][k] = ((4.0 * l[i]) - 1.0) * gl[i][k];
  }
  for (int m = 0; m < 6; ++m) {
    const int a = E[m][0], b = E[m][1];
    v[4 + m] = (4.0 * l[a]) * l[b];
    for (int k = 0; k < 3; ++k) g[4 + m][k] = 4.0 * (l[b] * gl[a][k] + l[a] * gl[b][k]);
  }
}

}  // namespace

void build_tables_tet(Tables& T, int p) {
  if (p < 1 || p > 2) throw std::invalid_argument("tetrahedra: DG order p must be 1 or 2");
  T.dim = 3;
  T.p = p;
  T.r = 1;
  T.nv = p + 2;
  T.nf = p + 1;
  T.N = p == 1 ? 4 : 10;
  T.Nf = p == 1 ? 3 : 6;
  T.Nv = 4;
  T.Q = T.nv * T.nv * T.nv;
  gauss_legendre(T.nv, T.glv_t, T.glv_w);
  gauss_legendre(T.nf, T.glf_t, T.glf_w);
  gll_nodes(p, T.gll);
  T.geo = {0.0, 1.0};
  T.wq.assign(T.Q, 0.0);
  T.B.assign((size_t)T.Q * T.N, 0.0);
  T.dB.assign((size_t)T.Q * T.N * 3, 0.0);
  T.dV.assign((size_t)T.Q * 4 * 3, 0.0);
  T.V.assign((size_t)T.Q * 4, 0.0);
  const int n = T.nv;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const int q = i + n * (j + n * k);
        const double u = T.glv_t[i], v = T.glv_t[j], w = T.glv_t[k];
        const double x = u, y = v * (1.0 - u), z = (w * (1.0 - u)) * (1.0 - v);
        T.wq[q] = ((((T.glv_w[i] * T.glv_w[j]) * T.glv_w[k]) * (1.0 - u)) * (1.0 - u)) * (1.0 - v);
        double bv[10], bg[10][3];
        tet_eval(p, x, y, z, bv, bg);
        for (int m = 0; m < T.N; ++m) {
          T.B[(size_t)q * T.N + m] = bv[m];
          for (int c = 0; c < 3; ++c) T.dB[((size_t)q * T.N + m) * 3 + c] = bg[m][c];
        }
        tet_eval(1, x, y, z, bv, bg);
        for (int m = 0; m < 4; ++m) {
          T.V[(size_t)q * 4 + m] = bv[m];
          for (int c = 0; c < 3; ++c) T.dV[((size_t)q * 4 + m) * 3 + c] = bg[m][c];
        }
      }
}

}  // namespace sn
