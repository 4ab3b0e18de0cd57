// Device helpers for the one-off geometry and graph kernels: Lagrange bases, face
// coordinates, orientation maps and face normals.  The arithmetic order is the one the
// graph's bit-exact contract fixes (products left to right from 1.0, sums in increasing
// index from 0.0); translation units that need exact reproducibility compile with
// -fmad=false so that no multiply-add is contracted.
#pragma once
#include "common.h"

namespace sn {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

__device__ inline const double* tabp(const DevProblem& P, int off) { return P.tab + off; }

__device__ inline double dlagrange(const double* nodes, int n, int j, double x) {
  double v = 1.0;
  for (int k = 0; k < n; ++k)
    if (k != j) v = v * ((x - nodes[k]) / (nodes[j] - nodes[k]));
  return v;
}

__device__ inline double dlagrange_deriv(const double* nodes, int n, int j, double x) {
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

// Reference coordinates of face f at face coordinates (s0, s1).
__device__ inline void face_ref(int dim, int f, double s0, double s1, double* xi) {
  int axis = f >> 1, side = f & 1;
  int o0 = (axis == 0) ? 1 : 0;
  int o1 = (axis == 2) ? 1 : 2;
  xi[axis] = (double)side;
  xi[o0] = s0;
  if (dim == 3) xi[o1] = s1;
}

// Owner face coordinates -> neighbour face coordinates (orientation code bits: 4 swap,
// 1 flip first, 2 flip second).
__device__ inline void orient_map(int dim, int code, double s0, double s1, double& t0, double& t1) {
  if (dim == 2) {
    t0 = (code & 1) ? 1.0 - s0 : s0;
    t1 = 0.0;
    return;
  }
  double u0 = (code & 4) ? s1 : s0;
  double u1 = (code & 4) ? s0 : s1;
  t0 = (code & 1) ? 1.0 - u0 : u0;
  t1 = (code & 2) ? 1.0 - u1 : u1;
}

// Same map on face-node grid indices (symmetric node sets: 1 - node_i = node_{p-i}).
__host__ __device__ inline void orient_map_idx(int dim, int code, int p, int i, int j, int& t0, int& t1) {
  if (dim == 2) {
    t0 = (code & 1) ? p - i : i;
    t1 = 0;
    return;
  }
  int u0 = (code & 4) ? j : i;
  int u1 = (code & 4) ? i : j;
  t0 = (code & 1) ? p - u0 : u0;
  t1 = (code & 2) ? p - u1 : u1;
}

// Volume node index of face node (i, j) of face f for order p.
__host__ __device__ constexpr int face_vol_index(int dim, int p, int f, int i, int j) {
  const int axis = f >> 1, side = f & 1;
  const int n = p + 1;
  const int t0 = axis == 0 ? side * p : i;
  const int t1 = axis == 1 ? side * p : (axis == 0 ? i : (dim == 3 ? j : 0));
  const int t2 = dim == 3 ? (axis == 2 ? side * p : j) : 0;
  return t0 + n * (t1 + n * t2);
}

// Triangles: local node index of node j (0..k, increasing face coordinate) of face f of an
// order-k node set numbered v0, v1, v2, the k - 1 interior nodes of f0, f1, f2, then the interior
// node; faces f0 = v0 v1, f1 = v1 v2, f2 = v2 v0.
__host__ __device__ constexpr int tri_edge_node(int k, int f, int j) {
  return j == 0 ? f : (j == k ? (f + 1) % 3 : 3 + f * (k - 1) + (j - 1));
}

// Triangle face f: outward scaled normal (T_y, -T_x), T(s) = sum_j x_j l_j'(s) over the face's
// r + 1 control points in increasing j from 0.0 (1D Lagrange on the equispaced nodes geo).
__device__ inline void face_normal_tri(int r, const double* geo, const double* ctrl, int f, double s,
                                       double* nvec) {
  double T0 = 0.0, T1 = 0.0;
  for (int j = 0; j <= r; ++j) {
    const int m = tri_edge_node(r, f, j);
    const double dv = dlagrange_deriv(geo, r + 1, j, s);
    T0 = T0 + ctrl[m * 2 + 0] * dv;
    T1 = T1 + ctrl[m * 2 + 1] * dv;
  }
  nvec[0] = T1;
  nvec[1] = -T0;
}

// Outward face normal scaled by the face Jacobian (cof(J) n_hat) at face coordinates of
// local face f, from the element's control points ctrl [Nv][dim].  Tangents
// T_b = sum over the face's control points (increasing index) of x_m * dv_m/dxi_b, where
// dv is the product over axes (left to right from 1.0) with the face-axis factor 1.
// 2D axis 0: (T1[1], -T1[0]); axis 1: (-T0[1], T0[0]); 3D axis a: T_{a+1} x T_{a+2} (cyclic),
// component i = u_{i+1} v_{i+2} - u_{i+2} v_{i+1}; side 0 negates.
__device__ inline void face_normal(int dim, int r, const double* geo, const double* ctrl, int f, double s0,
                                   double s1, double* nvec) {
  const int axis = f >> 1, side = f & 1;
  double xi[3];
  face_ref(dim, f, s0, s1, xi);
  const int n1 = r + 1;
  const int Nv = (dim == 2) ? n1 * n1 : n1 * n1 * n1;
  int tb[2];
  tb[0] = (axis + 1) % dim;
  tb[1] = (axis + 2) % dim;
  const int ntan = dim - 1;
  // 1D geometry basis values and derivatives on the face's own axes (each factor evaluated once;
  // the products below use the same values as evaluating it per control point)
  double lv[3][MAX_R + 1], ld[3][MAX_R + 1];
  for (int k = 0; k < dim; ++k) {
    if (k == axis) continue;
    for (int a = 0; a < n1; ++a) {
      lv[k][a] = dlagrange(geo, n1, a, xi[k]);
      ld[k][a] = dlagrange_deriv(geo, n1, a, xi[k]);
    }
  }
  double T[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  for (int m = 0; m < Nv; ++m) {
    int mi[3];
    mi[0] = m % n1;
    mi[1] = (m / n1) % n1;
    mi[2] = (dim == 3) ? m / (n1 * n1) : 0;
    if (mi[axis] != side * r) continue;        // other control points contribute exact zeros
    for (int t = 0; t < ntan; ++t) {
      const int b = tb[t];
      double dv = 1.0;
      for (int k = 0; k < dim; ++k) {
        double fac;
        if (k == axis) fac = 1.0;
        else if (k == b) fac = ld[k][mi[k]];
        else fac = lv[k][mi[k]];
        dv = dv * fac;
      }
      for (int c = 0; c < dim; ++c) T[t][c] = T[t][c] + ctrl[m * dim + c] * dv;
    }
  }
  if (dim == 2) {
    const double* t = T[0];
    if (axis == 0) {
      nvec[0] = t[1];
      nvec[1] = -t[0];
    } else {
      nvec[0] = -t[1];
      nvec[1] = t[0];
    }
  } else {
    const double* u = T[0];
    const double* v = T[1];
    for (int c = 0; c < 3; ++c) {
      int a = (c + 1) % 3, b = (c + 2) % 3;
      nvec[c] = u[a] * v[b] - u[b] * v[a];
    }
  }
  if (side == 0)
    for (int c = 0; c < dim; ++c) nvec[c] = -nvec[c];
}

__device__ inline double dot_omega(int dim, const double* om, const double* v) {
  double g = om[0] * v[0];
  for (int k = 1; k < dim; ++k) g = g + om[k] * v[k];
  return g;
}

// Face-node basis values at face coordinates: l_i(t0) (2D), l_i(t0) l_j(t1) (3D).
__device__ inline double face_basis(int dim, const double* gll, int np1, int fn, double t0, double t1) {
  if (dim == 2) return dlagrange(gll, np1, fn, t0);
  return dlagrange(gll, np1, fn % np1, t0) * dlagrange(gll, np1, fn / np1, t1);
}

// All face-node basis values at once (out[fn], fn = i + np1 j): the same products as face_basis,
// each 1D factor evaluated once.
__device__ inline void face_basis_all(int dim, const double* gll, int np1, double t0, double t1, double* out) {
  double l0[MAX_P + 1], l1[MAX_P + 1];
  for (int a = 0; a < np1; ++a) l0[a] = dlagrange(gll, np1, a, t0);
  if (dim == 2) {
    for (int a = 0; a < np1; ++a) out[a] = l0[a];
    return;
  }
  for (int a = 0; a < np1; ++a) l1[a] = dlagrange(gll, np1, a, t1);
  for (int fn = 0; fn < np1 * np1; ++fn) out[fn] = l0[fn % np1] * l1[fn / np1];
}

}  // namespace sn

namespace sn {

// ---- straight-sided tetrahedra (P_1 geometry, P_1 / P_2 DG).  Vertices v0..v3 of the reference
// tetrahedron (0,0,0), (1,0,0), (0,1,0), (0,0,1); face f opposite vertex f with the vertex triple
// tet_face_vert(f, 0..2) ordered so that (B - A) x (C - A) points outwards; face coordinates
// (s, t) = the barycentrics of B and C.  DG nodes: vertices, then (p = 2) the midpoints of the
// edges (0,1), (1,2), (2,0), (0,3), (1,3), (2,3); face nodes: A, B, C, then the AB, BC, CA
// midpoints.  Orientation code k of a shared face: the neighbour's vertex tet_perm(k, j) of its
// triple is our vertex j.
__host__ __device__ constexpr int tet_face_vert(int f, int j) {
  return f == 0 ? (j == 0 ? 1 : (j == 1 ? 2 : 3))
       : f == 1 ? (j == 0 ? 0 : (j == 1 ? 3 : 2))
       : f == 2 ? (j == 0 ? 0 : (j == 1 ? 1 : 3))
                : (j == 0 ? 0 : (j == 1 ? 2 : 1));
}
__host__ __device__ constexpr int tet_perm(int k, int j) {
  return k == 0 ? j : k == 1 ? (j + 1) % 3 : k == 2 ? (j + 2) % 3 : k == 3 ? (j == 0 ? 0 : 3 - j)
       : k == 4 ? 2 - j : (j == 2 ? 2 : 1 - j);
}
__host__ __device__ constexpr int tet_edge_index(int a, int b) {
  return (a + b == 1 && a * b == 0) ? 0 : (a + b == 3 && a * b == 2) ? 1 : (a + b == 2 && a * b == 0) ? 2
       : (a + b == 3 && a * b == 0) ? 3 : (a + b == 4 && a * b == 3) ? 4 : 5;
}
// Volume node of face node j of face f (order p DG).
__host__ __device__ constexpr int tet_face_node(int p, int f, int j) {
  return j < 3 ? tet_face_vert(f, j)
               : 4 + tet_edge_index(tet_face_vert(f, j - 3), tet_face_vert(f, (j - 2) % 3));
}
// Face node of the neighbour that sees our face node j (orientation code k): vertices permuted,
// the midpoint of our face edge (j, j + 1) goes to the neighbour's edge (perm j, perm (j + 1)).
__host__ __device__ constexpr int tet_face_edge(int a, int b) {
  return ((a == 0 && b == 1) || (a == 1 && b == 0)) ? 0 : ((a == 1 && b == 2) || (a == 2 && b == 1)) ? 1 : 2;
}
__host__ __device__ constexpr int tet_nbr_face_node(int k, int j) {
  return j < 3 ? tet_perm(k, j) : 3 + tet_face_edge(tet_perm(k, j - 3), tet_perm(k, (j - 2) % 3));
}

// Outward scaled normal (B - A) x (C - A) of face f: component c = u_a v_b - u_b v_a, a = c + 1,
// b = c + 2 (mod 3); ctrl [4][3].
__device__ inline void face_normal_tet(const double* ctrl, int f, double* nvec) {
  const int A = tet_face_vert(f, 0), B = tet_face_vert(f, 1), C = tet_face_vert(f, 2);
  double u[3], v[3];
  for (int c = 0; c < 3; ++c) {
    u[c] = ctrl[B * 3 + c] - ctrl[A * 3 + c];
    v[c] = ctrl[C * 3 + c] - ctrl[A * 3 + c];
  }
  for (int c = 0; c < 3; ++c) {
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    nvec[c] = u[a] * v[b] - u[b] * v[a];
  }
}

// Face-node basis values at face coordinates (s, t): p = 1, (1 - s) - t, s, t; p = 2, m ((2 m) - 1)
// at the vertices and (4 m_a) m_b at the edge midpoints.
__device__ inline void face_basis_tet(int p, double s, double t, double* out) {
  const double m[3] = {(1.0 - s) - t, s, t};
  if (p == 1) {
    for (int i = 0; i < 3; ++i) out[i] = m[i];
    return;
  }
  for (int i = 0; i < 3; ++i) out[i] = m[i] * ((2.0 * m[i]) - 1.0);
  out[3] = (4.0 * m[0]) * m[1];
  out[4] = (4.0 * m[1]) * m[2];
  out[5] = (4.0 * m[2]) * m[0];
}

// The neighbour's face coordinates of our (s, t): barycentrics permuted by orientation code k.
__device__ inline void orient_tet(int k, double s, double t, double& s2, double& t2) {
  const double m[3] = {(1.0 - s) - t, s, t};
  double mp[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < 3; ++j) mp[tet_perm(k, j)] = m[j];
  s2 = mp[1];
  t2 = mp[2];
}

// Scaled outward normal of face f of any element family at face coordinates (s0, s1).
__device__ inline void face_normal_el(const DevProblem& P, const double* geo, const double* ctrl, int f, double s0,
                                      double s1, double* nvec) {
  if (P.simplex && P.dim == 3) face_normal_tet(ctrl, f, nvec);
  else if (P.simplex) face_normal_tri(P.r, geo, ctrl, f, s0, nvec);
  else face_normal(P.dim, P.r, geo, ctrl, f, s0, s1, nvec);
}

// Volume node index of face node i of face f (face nodes in face-coordinate order).
__device__ inline int face_node_vol(const DevProblem& P, int f, int i) {
  if (P.simplex && P.dim == 3) return tet_face_node(P.p, f, i);
  if (P.simplex) return tri_edge_node(P.p, f, i);
  return face_vol_index(P.dim, P.p, f, i % (P.p + 1), i / (P.p + 1));
}

// All face-node basis values at face coordinates, and one of them (any element family).
__device__ inline void face_basis_el_all(const DevProblem& P, const double* gll, double s0, double s1, double* out) {
  if (P.simplex && P.dim == 3) face_basis_tet(P.p, s0, s1, out);
  else face_basis_all(P.dim, gll, P.p + 1, s0, s1, out);
}
__device__ inline double face_basis_el_one(const DevProblem& P, const double* gll, int i, double s0, double s1) {
  if (P.simplex && P.dim == 3) {
    double v[6];
    face_basis_tet(P.p, s0, s1, v);
    return v[i];
  }
  return face_basis(P.dim, gll, P.p + 1, i, s0, s1);
}

// The neighbour's face coordinates of ours (orientation code).
__device__ inline void orient_map_el(const DevProblem& P, int code, double s0, double s1, double& t0, double& t1) {
  if (P.simplex && P.dim == 3) orient_tet(code, s0, s1, t0, t1);
  else orient_map(P.dim, code, s0, s1, t0, t1);
}

}  // namespace sn
