// Upwind dependency graph on the device (Sec. 3): per (face, direction) the face quadrature
// of this direction, the upwind coupling blocks Fbar of both sides and the edge weights
// (unity / face = max|Fbar| / siginvface = max|M_t^{-1} Fbar|, eq. 22); the inflow mode of every
// (element, face, direction); the inflow blocks of partially-inflow faces for the sweep; and
// the longest-path levels of the kept acyclic graph.
//
// This translation unit is compiled with -fmad=false and follows, operation by operation,
// the order of the CPU oracle's graph stage, so that weights -- and therefore the removed arc
// set and the levels -- are reproduced bit for bit.
#include "devmath.cuh"

namespace sn {

namespace {

struct PointData {
  double s0, s1, w;
};

// 2D: breakpoints of the split at the sign changes of g(s) = Omega . n(s) (degree <= 2).
__device__ void split_2d(const DevProblem& P, const double* ctrl, int f, const double* om, double* brk) {
  const double* geo = tabp(P, P.off_geo);
  double n0[3], nh[3], n1[3];
  face_normal_el(P, geo, ctrl, f, 0.0, 0.0, n0);
  face_normal_el(P, geo, ctrl, f, 0.5, 0.0, nh);
  face_normal_el(P, geo, ctrl, f, 1.0, 0.0, n1);
  const double g0 = dot_omega(2, om, n0), gh = dot_omega(2, om, nh), g1 = dot_omega(2, om, n1);
  const double c0 = g0;
  const double c2 = 2.0 * ((g0 - 2.0 * gh) + g1);
  const double c1 = (g1 - g0) - c2;
  double ra = 2.0, rb = 2.0;     // 2.0 = no root
  if (c2 == 0.0) {
    if (c1 != 0.0) ra = -c0 / c1;
  } else {
    const double disc = c1 * c1 - (4.0 * c2) * c0;
    if (disc >= 0.0) {
      const double sq = sqrt(disc);
      const double qq = -0.5 * (c1 + (c1 >= 0.0 ? sq : -sq));
      ra = qq / c2;
      if (qq != 0.0) rb = c0 / qq;
    }
  }
  ra = (ra > 0.0 && ra < 1.0) ? ra : 1.0;
  rb = (rb > 0.0 && rb < 1.0) ? rb : 1.0;
  brk[0] = 0.0;
  brk[1] = fmin(ra, rb);
  brk[2] = fmax(ra, rb);
  brk[3] = 1.0;
}

// The same breakpoints from the three reference normals n(0), n(1/2), n(1) of the face
// (direction independent, computed once per face).
__device__ void split_2d_cached(const double* nref, const double* om, double* brk) {
  const double g0 = dot_omega(2, om, nref), gh = dot_omega(2, om, nref + 2), g1 = dot_omega(2, om, nref + 4);
  const double c0 = g0;
  const double c2 = 2.0 * ((g0 - 2.0 * gh) + g1);
  const double c1 = (g1 - g0) - c2;
  double ra = 2.0, rb = 2.0;     // 2.0 = no root
  if (c2 == 0.0) {
    if (c1 != 0.0) ra = -c0 / c1;
  } else {
    const double disc = c1 * c1 - (4.0 * c2) * c0;
    if (disc >= 0.0) {
      const double sq = sqrt(disc);
      const double qq = -0.5 * (c1 + (c1 >= 0.0 ? sq : -sq));
      ra = qq / c2;
      if (qq != 0.0) rb = c0 / qq;
    }
  }
  ra = (ra > 0.0 && ra < 1.0) ? ra : 1.0;
  rb = (rb > 0.0 && rb < 1.0) ? rb : 1.0;
  brk[0] = 0.0;
  brk[1] = fmin(ra, rb);
  brk[2] = fmax(ra, rb);
  brk[3] = 1.0;
}

// ---- 3D faces: the kink of max(+-Omega.n, 0) follows the curve g(s0, s1) = Omega . n = 0, and g
// is a polynomial of degree Dg = 2r - 1 in each face coordinate.  Outer coordinate s1: breakpoints
// k/K merged with the roots of the edge polynomials g(0, s1) and g(1, s1) (where the kink curve
// leaves the face); inner coordinate s0, on every outer quadrature line: breakpoints k/K merged
// with the roots of g(., s1).  Every piece carries n_f Gauss-Legendre points.  Point order: outer
// piece, outer point, inner piece, inner point; empty pieces (zero length) carry no points: their
// terms would be +-0 and change no sum.
constexpr int BISECT_STEPS = 60;
constexpr int MAX_DG = 5;            // Q3 geometry: n = T0 x T1 has degree 5 per face coordinate

// Monomial coefficients c[0..D] of the polynomial through (k/D, v_k): divided differences
// (a_k -= a_{k-1}, / (x_k - x_{k-j}), k descending) then nested multiplication (k descending).
__device__ inline void poly_from_samples(int D, const double* v, double* c) {
  double x[MAX_DG + 1], a[MAX_DG + 1];
  for (int k = 0; k <= D; ++k) {
    x[k] = (double)k / (double)D;
    a[k] = v[k];
  }
  for (int j = 1; j <= D; ++j)
    for (int k = D; k >= j; --k) a[k] = (a[k] - a[k - 1]) / (x[k] - x[k - j]);
  double cur[MAX_DG + 1], nxt[MAX_DG + 1];
  cur[0] = a[D];
  int m = 1;
  for (int k = D - 1; k >= 0; --k) {
    nxt[0] = a[k] - x[k] * cur[0];
    for (int i = 1; i < m; ++i) nxt[i] = cur[i - 1] - x[k] * cur[i];
    nxt[m] = cur[m - 1];
    ++m;
    for (int i = 0; i < m; ++i) cur[i] = nxt[i];
  }
  for (int i = 0; i <= D; ++i) c[i] = cur[i];
}

__device__ inline double poly_eval(int D, const double* c, double t) {
  double v = c[D];
  for (int i = D - 1; i >= 0; --i) v = v * t + c[i];
  return v;
}

// Roots in (0, 1) of c0 + c1 t + c2 t^2 (the 2D split's closed form), ascending, 1.0 if absent.
__device__ inline void quad_roots_01(double c0, double c1, double c2, double* out) {
  double ra = 2.0, rb = 2.0;
  if (c2 == 0.0) {
    if (c1 != 0.0) ra = -c0 / c1;
  } else {
    const double disc = c1 * c1 - (4.0 * c2) * c0;
    if (disc >= 0.0) {
      const double sq = sqrt(disc);
      const double qq = -0.5 * (c1 + (c1 >= 0.0 ? sq : -sq));
      ra = qq / c2;
      if (qq != 0.0) rb = c0 / qq;
    }
  }
  ra = (ra > 0.0 && ra < 1.0) ? ra : 1.0;
  rb = (rb > 0.0 && rb < 1.0) ? rb : 1.0;
  out[0] = fmin(ra, rb);
  out[1] = fmax(ra, rb);
}

// Sign-changing roots in (0, 1) of the degree-D polynomial c, ascending, D entries (1.0 where
// unused).  Degree >= 3: the derivative's roots cut [0, 1] into monotone intervals; an interval
// with a strict sign change holds one root, found by BISECT_STEPS bisections from its ends.
__device__ inline void poly_roots_01(int D, const double* c, double* out) {
  if (D == 1) {
    const double r = c[1] != 0.0 ? -c[0] / c[1] : 2.0;
    out[0] = (r > 0.0 && r < 1.0) ? r : 1.0;
    return;
  }
  double d[MAX_DG - 1][MAX_DG + 1];          // derivative chain: d[k] has degree D - k
  for (int i = 0; i <= D; ++i) d[0][i] = c[i];
  for (int k = 1; k <= D - 2; ++k)
    for (int i = 0; i <= D - k; ++i) d[k][i] = (double)(i + 1) * d[k - 1][i + 1];
  double crit[MAX_DG];
  quad_roots_01(d[D - 2][0], d[D - 2][1], d[D - 2][2], crit);
  for (int level = D - 3; level >= 0; --level) {
    const int deg = D - level;
    const double* pc = d[level];
    double brk[MAX_DG + 1];
    brk[0] = 0.0;
    for (int k = 0; k < deg - 1; ++k) brk[k + 1] = crit[k];
    brk[deg] = 1.0;
    double found[MAX_DG];
    for (int k = 0; k < deg; ++k) {
      double lo = brk[k], hi = brk[k + 1];
      const double flo = poly_eval(deg, pc, lo), fhi = poly_eval(deg, pc, hi);
      const bool change = (flo < 0.0 && fhi > 0.0) || (flo > 0.0 && fhi < 0.0);
      found[k] = 1.0;
      if (change) {
        const bool plo = flo > 0.0;
        for (int s = 0; s < BISECT_STEPS; ++s) {
          const double m = 0.5 * (lo + hi);
          if ((poly_eval(deg, pc, m) > 0.0) == plo) lo = m;
          else hi = m;
        }
        found[k] = 0.5 * (lo + hi);
      }
    }
    for (int a = 1; a < deg; ++a)           // ascending (insertion sort)
      for (int b = a; b > 0 && found[b] < found[b - 1]; --b) {
        const double t = found[b];
        found[b] = found[b - 1];
        found[b - 1] = t;
      }
    for (int k = 0; k < deg; ++k) crit[k] = found[k];
  }
  for (int k = 0; k < D; ++k) out[k] = crit[k];
}

// Breakpoints k/K (k = 0..K) merged with nr roots, ascending (insertion sort): K + 1 + nr values.
__device__ inline void merge_breaks(int K, const double* roots, int nr, double* brk) {
  int n = 0;
  for (int k = 0; k <= K; ++k) brk[n++] = (double)k / (double)K;
  for (int k = 0; k < nr; ++k) brk[n++] = roots[k];
  for (int a = 1; a < n; ++a)
    for (int b = a; b > 0 && brk[b] < brk[b - 1]; --b) {
      const double t = brk[b];
      brk[b] = brk[b - 1];
      brk[b - 1] = t;
    }
}

__device__ inline int face_npoints(const DevProblem& P) {
  if (P.dim == 3 && P.simplex) return P.nf * P.nf;          // flat triangle faces: no split
  return (P.dim == 2) ? 3 * P.nf : P.K * P.K * P.nf * P.nf;
}

// Per-warp shared-memory workspace of the 3D rule (doubles).
constexpr int R3_CHUNK = 32;           // points staged per round
struct R3Layout {
  int Dg, nbo, nomax, nip, stride, n;
  int o_roots, o_brk, o_s1, o_w1, o_ilo, o_iln, o_cnt, o_off, o_pts, o_acc;
};
__host__ __device__ inline R3Layout r3_layout(int r, int K, int nf, int Nf) {
  R3Layout L;
  L.Dg = 2 * r - 1;
  L.nbo = K + 1 + 2 * L.Dg;
  L.nomax = (K + 2 * L.Dg) * nf;
  L.nip = K + L.Dg;
  L.stride = 2 + 2 * Nf;
  int o = 0;
  L.o_roots = o; o += 2 * L.Dg;
  L.o_brk = o;   o += L.nbo;
  L.o_s1 = o;    o += L.nomax;
  L.o_w1 = o;    o += L.nomax;
  L.o_ilo = o;   o += L.nomax * L.nip;
  L.o_iln = o;   o += L.nomax * L.nip;
  L.o_cnt = o;   o += L.nomax + 1;         // number of points of outer point o (as a double), then NO
  L.o_off = o;   o += L.nomax + 1;         // first point of outer point o
  L.o_pts = o;   o += R3_CHUNK * L.stride;
  L.o_acc = o;   o += 4 * Nf * Nf;
  L.n = o;
  return L;
}

// Roots of g along the edge s0 = side (as a polynomial in s1) or along the line s1 = const (as a
// polynomial in s0), from the normals at the Dg + 1 equispaced samples.
__device__ inline void line_roots(int Dg, const double* om, const double* nsamp, double* roots) {
  double gv[MAX_DG + 1], c[MAX_DG + 1];
  for (int k = 0; k <= Dg; ++k) gv[k] = dot_omega(3, om, nsamp + 3 * k);
  poly_from_samples(Dg, gv, c);
  poly_roots_01(Dg, c, roots);
}

// Blocks of one (3D face, direction) over the kink-aligned rule: block b = sum over the rule's
// points, in order from 0.0, of (pt[aoff] pt[roff + i]) pt[uoff + j], spec[3 b .. 3 b + 2] =
// (aoff, roff, uoff) on the point rows [a_o, a_n, phi_o[Nf], phi_n[Nf]] (a_o = max(-g, 0) w,
// a_n = max(g, 0) w).  Results in ws[L.o_acc + b Nf^2 + i Nf + j]; nE (optional): the normals at
// the edge samples (s0 = 0 and s0 = 1, s1 = k / Dg), [2][Dg + 1][3].
__device__ void rule3_blocks(const DevProblem& P, const R3Layout& L, const double* ctrl, int f, int code,
                             bool has_nbr, const double* om, const double* nE, double* ws, int lane, int nblk,
                             const int* spec) {
  const int K = P.K, nf = P.nf, Nf = P.Nf, np1 = P.p + 1, Dg = L.Dg, stride = L.stride;
  const double* geo = tabp(P, P.off_geo);
  const double* gll = tabp(P, P.off_gll);
  const double* t = tabp(P, P.off_glf_t);
  const double* wt = tabp(P, P.off_glf_w);
  double* roots = ws + L.o_roots;
  double* s1o = ws + L.o_s1;
  double* w1o = ws + L.o_w1;
  double* ilo = ws + L.o_ilo;
  double* iln = ws + L.o_iln;
  double* cnt = ws + L.o_cnt;
  double* off = ws + L.o_off;
  double* pts = ws + L.o_pts;
  double* acc = ws + L.o_acc;
  // edge roots (lanes 0 and 1), outer breakpoints and outer points (lane 0)
  if (lane < 2) {
    double ns[3 * (MAX_DG + 1)];
    for (int k = 0; k <= Dg; ++k) {
      if (nE) {
        for (int c = 0; c < 3; ++c) ns[3 * k + c] = nE[(lane * (Dg + 1) + k) * 3 + c];
      } else {
        face_normal(3, P.r, geo, ctrl, f, (double)lane, (double)k / (double)Dg, ns + 3 * k);
      }
    }
    line_roots(Dg, om, ns, roots + lane * Dg);
  }
  __syncwarp();
  if (lane == 0) {
    double* brk = ws + L.o_brk;
    merge_breaks(K, roots, 2 * Dg, brk);
    int no = 0;
    for (int v = 0; v + 1 < L.nbo; ++v) {
      const double lo = brk[v], hi = brk[v + 1];
      if (!(hi > lo)) continue;
      const double ln = hi - lo;
      for (int j = 0; j < nf; ++j) {
        s1o[no] = lo + ln * t[j];
        w1o[no] = ln * wt[j];
        ++no;
      }
    }
    cnt[L.nomax] = (double)no;
  }
  __syncwarp();
  const int NO = (int)cnt[L.nomax];
  // inner breakpoints along every outer line
  for (int o = lane; o < NO; o += 32) {
    double ns[3 * (MAX_DG + 1)], rr[MAX_DG], brk[4 + 1 + MAX_DG];
    for (int k = 0; k <= Dg; ++k) face_normal(3, P.r, geo, ctrl, f, (double)k / (double)Dg, s1o[o], ns + 3 * k);
    line_roots(Dg, om, ns, rr);
    merge_breaks(K, rr, Dg, brk);
    int c = 0;
    for (int u = 0; u < K + Dg; ++u) {
      const double lo = brk[u], hi = brk[u + 1];
      if (!(hi > lo)) continue;
      ilo[o * L.nip + c] = lo;
      iln[o * L.nip + c] = hi - lo;
      ++c;
    }
    cnt[o] = (double)(c * nf);
  }
  __syncwarp();
  if (lane == 0) {
    double s = 0.0;
    for (int o = 0; o < NO; ++o) {
      off[o] = s;
      s = s + cnt[o];
    }
    off[NO] = s;
  }
  for (int e = lane; e < nblk * Nf * Nf; e += 32) acc[e] = 0.0;
  __syncwarp();
  const int NP = (int)off[NO];
  for (int c0 = 0; c0 < NP; c0 += R3_CHUNK) {
    const int q = c0 + lane;
    if (lane < R3_CHUNK && q < NP) {
      int o = 0;
      while ((int)off[o + 1] <= q) ++o;
      const int loc = q - (int)off[o], u = loc / nf, i = loc % nf;
      const double lo = ilo[o * L.nip + u], ln = iln[o * L.nip + u];
      const double s0 = lo + ln * t[i], s1 = s1o[o];
      const double w = w1o[o] * (ln * wt[i]);
      double nv[3];
      face_normal(3, P.r, geo, ctrl, f, s0, s1, nv);
      const double g = dot_omega(3, om, nv);
      const double mg = -g;
      double* pt = pts + lane * stride;
      pt[0] = (mg > 0.0 ? mg : 0.0) * w;
      pt[1] = (g > 0.0 ? g : 0.0) * w;
      face_basis_all(3, gll, np1, s0, s1, pt + 2);
      if (has_nbr) {
        double t0, t1;
        orient_map(3, code, s0, s1, t0, t1);
        face_basis_all(3, gll, np1, t0, t1, pt + 2 + Nf);
      }
    }
    __syncwarp();
    const int nq = min(R3_CHUNK, NP - c0);
    for (int e = lane; e < nblk * Nf * Nf; e += 32) {
      const int b = e / (Nf * Nf), ij = e % (Nf * Nf), i = ij / Nf, j = ij % Nf;
      const int aoff = spec[3 * b], roff = spec[3 * b + 1], uoff = spec[3 * b + 2];
      double a = acc[e];
      for (int qq = 0; qq < nq; ++qq) {
        const double* pt = pts + qq * stride;
        a = a + (pt[aoff] * pt[roff + i]) * pt[uoff + j];
      }
      acc[e] = a;
    }
    __syncwarp();
  }
}

__device__ inline PointData face_point(const DevProblem& P, const double* brk, int q) {
  const double* t = tabp(P, P.off_glf_t);
  const double* wt = tabp(P, P.off_glf_w);
  const int nf = P.nf;
  PointData pd;
  if (P.dim == 3 && P.simplex) {
    // tetrahedron face: collapsed triangle rule, point i + nf j at (u_i, v_j (1 - u_i)), weight
    // (w_i w_j) (1 - u_i); Omega . n is constant on the flat face, so there is nothing to split
    const int i = q % nf, j = q / nf;
    pd.s0 = t[i];
    pd.s1 = t[j] * (1.0 - t[i]);
    pd.w = (wt[i] * wt[j]) * (1.0 - t[i]);
  } else if (P.dim == 2) {
    const int piece = q / nf, i = q % nf;
    const double lo = brk[piece], hi = brk[piece + 1];
    const double ln = hi - lo;
    pd.s0 = lo + ln * t[i];
    pd.s1 = 0.0;
    pd.w = ln * wt[i];
  } else {
    // 3D rule without roots (the K x K composite rule) in the rule's point order: point
    // ((v nf + j) K + u) nf + i, outer piece v, outer point j, inner piece u, inner point i
    const int K = P.K;
    const int i = q % nf, u = (q / nf) % K, j = (q / (nf * K)) % nf, v = q / (nf * K * nf);
    const double lo1 = (double)v / (double)K, hi1 = (double)(v + 1) / (double)K, ln1 = hi1 - lo1;
    const double lo0 = (double)u / (double)K, hi0 = (double)(u + 1) / (double)K, ln0 = hi0 - lo0;
    pd.s1 = lo1 + ln1 * t[j];
    pd.s0 = lo0 + ln0 * t[i];
    pd.w = (ln1 * wt[j]) * (ln0 * wt[i]);
  }
  return pd;
}

// Per-point data of one (face, direction) into shared memory; a = max(-g,0) w (owner
// receiving) and max(g,0) w (other side receiving); basis values of both sides' face nodes.
// Layout per point: [a_o, a_n, phi_o[Nf], phi_n[Nf]].
__device__ void fill_points_brk(const DevProblem& P, const double* ctrl, int f, int code, bool has_nbr,
                                const double* om, const double* brk, double* sp, int lane) {
  const int np = face_npoints(P);
  const int Nf = P.Nf, np1 = P.p + 1;
  const int stride = 2 + 2 * Nf;
  const double* geo = tabp(P, P.off_geo);
  const double* gll = tabp(P, P.off_gll);
  for (int q = lane; q < np; q += 32) {
    PointData pd = face_point(P, brk, q);
    double nv[3];
    face_normal_el(P, geo, ctrl, f, pd.s0, pd.s1, nv);
    const double g = dot_omega(P.dim, om, nv);
    const double mg = -g;
    double* o = sp + q * stride;
    o[0] = (mg > 0.0 ? mg : 0.0) * pd.w;
    o[1] = (g > 0.0 ? g : 0.0) * pd.w;
    face_basis_el_all(P, gll, pd.s0, pd.s1, o + 2);
    if (has_nbr) {
      double t0, t1;
      orient_map_el(P, code, pd.s0, pd.s1, t0, t1);
      face_basis_el_all(P, gll, t0, t1, o + 2 + Nf);
    }
  }
  __syncwarp();
}

__device__ void fill_points(const DevProblem& P, const double* ctrl, int f, int code, bool has_nbr,
                            const double* om, double* sp, int lane) {
  double brk[4] = {0.0, 1.0, 1.0, 1.0};
  if (P.dim == 2) split_2d(P, ctrl, f, om, brk);
  fill_points_brk(P, ctrl, f, code, has_nbr, om, brk, sp, lane);
}

// Direction-independent point data of a face for the unsplit rule (breakpoints 0, 1, 1, 1 in
// 2D; the composite rule in 3D): sp rows [-, -, phi_o[Nf], phi_n[Nf]] and wn rows [w, n[dim]].
// The per-direction inflow amounts are then set by cache_amounts with the same operations as
// fill_points_brk.
__device__ void fill_cache(const DevProblem& P, const double* ctrl, int f, int code, double* sp, double* wn,
                           int lane) {
  const double brk[4] = {0.0, 1.0, 1.0, 1.0};
  const int np = face_npoints(P);
  const int Nf = P.Nf, np1 = P.p + 1, dim = P.dim;
  const int stride = 2 + 2 * Nf;
  const double* geo = tabp(P, P.off_geo);
  const double* gll = tabp(P, P.off_gll);
  for (int q = lane; q < np; q += 32) {
    PointData pd = face_point(P, brk, q);
    double nv[3];
    face_normal_el(P, geo, ctrl, f, pd.s0, pd.s1, nv);
    double* w = wn + q * (1 + dim);
    w[0] = pd.w;
    for (int c = 0; c < dim; ++c) w[1 + c] = nv[c];
    double* o = sp + q * stride;
    face_basis_el_all(P, gll, pd.s0, pd.s1, o + 2);
    double t0, t1;
    orient_map_el(P, code, pd.s0, pd.s1, t0, t1);
    face_basis_el_all(P, gll, t0, t1, o + 2 + Nf);
  }
  __syncwarp();
}

__device__ void cache_amounts(const DevProblem& P, const double* wn, const double* om, double* sp, int np, int lane) {
  const int dim = P.dim, stride = 2 + 2 * P.Nf;
  for (int q = lane; q < np; q += 32) {
    const double* w = wn + q * (1 + dim);
    const double g = dot_omega(dim, om, w + 1);
    const double mg = -g;
    double* o = sp + q * stride;
    o[0] = (mg > 0.0 ? mg : 0.0) * w[0];
    o[1] = (g > 0.0 ? g : 0.0) * w[0];
  }
  __syncwarp();
}

// Block entry (i, j): sum_q (a_q phi_r_i(q)) phi_u_j(q), q ascending from 0.0.
__device__ inline double block_entry(const double* sp, int np, int stride, int aoff, int roff, int uoff, int i,
                                     int j) {
  double acc = 0.0;
  for (int q = 0; q < np; ++q) {
    const double* o = sp + q * stride;
    acc = acc + (o[aoff] * o[roff + i]) * o[uoff + j];
  }
  return acc;
}

__device__ inline double warp_max(double v) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

__device__ void copy_ctrl(const DevProblem& P, int64_t e, double* dst, int lane) {
  const int n = P.Nv * P.dim;
  for (int t = lane; t < n; t += 32) dst[t] = P.ctrl[e * n + t];
  __syncwarp();
}

// max |M_t^{-1} Fbar_full| over the Nf nonzero columns; Fbar rows at the receiving element's
// face-node volume indices.  Column c solved by lane c with the plain pivoted LU order.
__device__ double siginv_weight(const DevProblem& P, const double* fbar, int64_t recv, int recv_face,
                                const double* lu, const int32_t* perm, int lane) {
  const int N = P.N, Nf = P.Nf;
  double best = 0.0;
  if (lane < Nf) {
    const double* L = lu + recv * N * N;
    const int32_t* pm = perm + recv * N;
    double y[27];
    double b[27];
    for (int i = 0; i < N; ++i) b[i] = 0.0;
    for (int i = 0; i < Nf; ++i) {
      const int vi = face_node_vol(P, recv_face, i);
      b[vi] = fbar[i * Nf + lane];
    }
    for (int i = 0; i < N; ++i) y[i] = b[pm[i]];
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < i; ++j) y[i] = y[i] - L[i * N + j] * y[j];
    for (int i = N - 1; i >= 0; --i) {
      for (int j = i + 1; j < N; ++j) y[i] = y[i] - L[i * N + j] * y[j];
      y[i] = y[i] / L[i * N + i];
    }
    for (int i = 0; i < N; ++i) best = fmax(best, fabs(y[i]));
  }
  return warp_max(best);
}

}  // namespace

// ------------------------------------------------------------------ sigma_t mass LU
// M_t = sigma_t * M, M_mn = sum_q ((w_q |J_q|) u_m(q)) u_n(q) in increasing q; J from the
// tabulated geometry gradients summed over all control points in increasing index.
__global__ void mass_lu_kernel(DevProblem P, double* __restrict__ lu, int32_t* __restrict__ perm) {
  extern __shared__ double sh[];
  const int64_t e = blockIdx.x;
  const int N = P.N, Q = P.Q, Nv = P.Nv, dim = P.dim;
  double* wdet = sh;          // [Q]
  double* A = sh + Q;         // [N][N]
  __shared__ int32_t pv[32];
  __shared__ int piv_s;
  const double* wq = tabp(P, P.off_wq);
  const double* B = tabp(P, P.off_B);
  const double* dV = tabp(P, P.off_dV);
  const double* ctrl = P.ctrl + e * Nv * dim;
  for (int q = threadIdx.x; q < Q; q += blockDim.x) {
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int m = 0; m < Nv; ++m)
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) J[i][j] = J[i][j] + ctrl[m * dim + i] * dV[((size_t)q * Nv + m) * dim + j];
    double det;
    if (dim == 2) {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    } else {
      const double t0 = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]);
      const double t1 = J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]);
      const double t2 = J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      det = (t0 - t1) + t2;
    }
    wdet[q] = wq[q] * det;
  }
  __syncthreads();
  const double st = P.sig_t[e];
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    const int m = t / N, n = t % N;
    double acc = 0.0;
    for (int q = 0; q < Q; ++q) acc = acc + ((wdet[q] * B[(size_t)q * N + m]) * B[(size_t)q * N + n]);
    A[t] = st * acc;
  }
  if (threadIdx.x < N) pv[threadIdx.x] = threadIdx.x;
  __syncthreads();
  // Doolittle with partial pivoting (first row of largest |A[i][k]|), full row swaps.
  for (int k = 0; k < N; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = fabs(A[k * N + k]);
      for (int i = k + 1; i < N; ++i)
        if (fabs(A[i * N + k]) > best) {
          best = fabs(A[i * N + k]);
          p = i;
        }
      piv_s = p;
    }
    __syncthreads();
    const int p = piv_s;
    if (p != k) {
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double t = A[k * N + j];
        A[k * N + j] = A[p * N + j];
        A[p * N + j] = t;
      }
      if (threadIdx.x == 0) {
        int t = pv[k];
        pv[k] = pv[p];
        pv[p] = t;
      }
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < N; i += blockDim.x) {
      const double l = A[i * N + k] / A[k * N + k];
      A[i * N + k] = l;
      for (int j = k + 1; j < N; ++j) A[i * N + j] = A[i * N + j] - l * A[k * N + j];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) lu[e * N * N + t] = A[t];
  if (threadIdx.x < N) perm[e * N + threadIdx.x] = pv[threadIdx.x];
}

cudaError_t launch_mass_lu(const DevProblem& P, double* lu, int32_t* perm, cudaStream_t s) {
  size_t shmem = sizeof(double) * ((size_t)P.Q + (size_t)P.N * P.N);
  mass_lu_kernel<<<(unsigned)P.E, 64, shmem, s>>>(P, lu, perm);
  return cudaGetLastError();
}

// Edge weights and inflow modes of one (interior face, direction) from its two coupling blocks
// fb = [owner <- neighbour][neighbour <- owner] and their max-entry norms mo, mn; the weight of an
// arc is stored at the receiving element's face: win[d][e][f].
__device__ void emit_weights(const DevProblem& P, int64_t fi, int d, int64_t owner, int64_t nbr, int f, int fn,
                             int weighting, const double* mt_lu, const int32_t* mt_perm, const double* fb,
                             double mo, double mn, double* win, uint32_t* facecode, int lane) {
  const int Nf = P.Nf;
  const bool eo = mo > 0.0, en = mn > 0.0;
  double wo = 0.0, wv = 0.0;
  if (weighting == SN_WEIGHT_UNITY) {
    wo = eo ? 1.0 : 0.0;
    wv = en ? 1.0 : 0.0;
  } else if (weighting == SN_WEIGHT_FACE) {
    wo = mo;
    wv = mn;
  } else {
    wo = eo ? siginv_weight(P, fb, owner, f, mt_lu, mt_perm, lane) : 0.0;
    wv = en ? siginv_weight(P, fb + Nf * Nf, nbr, fn, mt_lu, mt_perm, lane) : 0.0;
  }
  if (lane == 0) {
    const int nfc = P.nfc;
    win[((int64_t)d * P.E + owner) * nfc + f] = wo;         // arc nbr -> owner, owner's face f
    win[((int64_t)d * P.E + nbr) * nfc + fn] = wv;          // arc owner -> nbr, nbr's face fn
    if (eo) atomicOr(&facecode[(int64_t)d * P.E + owner], (en ? MODE_MIXED : MODE_PURE) << (2 * f));
    if (en) atomicOr(&facecode[(int64_t)d * P.E + nbr], (eo ? MODE_MIXED : MODE_PURE) << (2 * fn));
  }
}

// ------------------------------------------------------------------ edge weights
// One warp per interior face, all directions.  The unsplit rule's point data (normals, both
// sides' basis values) are computed once per face; a direction whose 2D split has no root in
// (0, 1) uses them (its breakpoints are exactly 0, 1, 1, 1, so the points, weights and normals
// are the same numbers), and of that rule only the first piece's n_f points have nonzero
// weight: the zero-length pieces add (+0 a) phi phi = +-0 terms, which leave a sum that started
// from +0.0 unchanged, so they are skipped.  Directions whose split has roots recompute their
// points as fill_points does.  iface rows: owner, f, nbr, f_nbr, orient.
__global__ void weights_face_kernel(DevProblem P, const int32_t* __restrict__ iface, int64_t n_iface,
                                    int weighting, const double* __restrict__ mt_lu,
                                    const int32_t* __restrict__ mt_perm, double* __restrict__ win,
                                    uint32_t* facecode, int shm_per_warp) {
  extern __shared__ double sh[];
  const int warp_in_block = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t fi = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_in_block;
  if (fi >= n_iface) return;     // whole warp exits together
  const int32_t* row = iface + fi * 5;
  const int64_t owner = row[0], nbr = row[2];
  const int f = row[1], fn = row[3], code = row[4];
  const int np = face_npoints(P);
  const int Nf = P.Nf, dim = P.dim;
  const int stride = 2 + 2 * Nf;
  double* wsh = sh + (size_t)warp_in_block * shm_per_warp;
  double* ctrl = wsh;                                   // Nv * dim
  double* nref = ctrl + P.Nv * dim;                     // 3 x 2 (2D)
  double* cache = nref + 6;                             // np x stride
  double* wn = cache + np * stride;                     // np x (1 + dim)
  double* scratch = wn + np * (1 + dim);                // np x stride (2D split directions)
  double* fb = scratch + (dim == 2 ? np * stride : 0);  // [2][Nf][Nf]
  // 3D: normals at the edge samples [2][Dg+1][3] and along the composite rule's outer lines
  // [K nf][Dg+1][3] (direction independent), and the rule's workspace
  const R3Layout L = r3_layout(P.r, P.K, P.nf, Nf);
  const int Dg = L.Dg, nlines = P.K * P.nf;
  double* nE = fb + 2 * Nf * Nf;
  const bool r3on = dim == 3 && !P.simplex;
  double* nB = nE + (r3on ? 2 * (Dg + 1) * 3 : 0);
  double* r3 = nB + (r3on ? nlines * (Dg + 1) * 3 : 0);
  copy_ctrl(P, owner, ctrl, lane);
  const double* geo = tabp(P, P.off_geo);
  if (dim == 2 && lane < 3) {
    double nv[3];
    face_normal_el(P, geo, ctrl, f, lane == 0 ? 0.0 : (lane == 1 ? 0.5 : 1.0), 0.0, nv);
    nref[2 * lane] = nv[0];
    nref[2 * lane + 1] = nv[1];
  }
  if (dim == 3 && !P.simplex) {
    const double* t = tabp(P, P.off_glf_t);
    for (int s = lane; s < 2 * (Dg + 1); s += 32)
      face_normal(3, P.r, geo, ctrl, f, (double)(s / (Dg + 1)), (double)(s % (Dg + 1)) / (double)Dg, nE + 3 * s);
    for (int s = lane; s < nlines * (Dg + 1); s += 32) {
      const int ob = s / (Dg + 1), k = s % (Dg + 1), v = ob / P.nf, j = ob % P.nf;
      const double lo = (double)v / (double)P.K, hi = (double)(v + 1) / (double)P.K;
      face_normal(3, P.r, geo, ctrl, f, (double)k / (double)Dg, lo + (hi - lo) * t[j], nB + 3 * s);
    }
  }
  fill_cache(P, ctrl, f, code, cache, wn, lane);
  const int spec3[6] = {0, 2, 2 + Nf, 1, 2 + Nf, 2};   // owner <- neighbour, neighbour <- owner
  for (int d = 0; d < P.M; ++d) {
    const double om[3] = {P.omega[d * 3 + 0], P.omega[d * 3 + 1], P.omega[d * 3 + 2]};
    double brk[4] = {0.0, 1.0, 1.0, 1.0};
    bool unsplit;
    if (dim == 2) {
      split_2d_cached(nref, om, brk);
      unsplit = brk[1] == 1.0 && brk[2] == 1.0;
    } else if (P.simplex) {
      unsplit = true;                    // tetrahedron faces are flat: Omega . n is constant
    } else {
      // no root on either edge and none along the composite rule's outer lines: the rule is the
      // cached composite rule
      bool root = false;
      double rr[MAX_DG];
      if (lane < 2) {
        line_roots(Dg, om, nE + lane * (Dg + 1) * 3, rr);
        for (int k = 0; k < Dg; ++k) root = root || rr[k] < 1.0;
      }
      for (int ob = lane; ob < nlines; ob += 32) {
        line_roots(Dg, om, nB + ob * (Dg + 1) * 3, rr);
        for (int k = 0; k < Dg; ++k) root = root || rr[k] < 1.0;
      }
      unsplit = !__any_sync(0xffffffffu, root);
    }
    if (dim == 3 && !unsplit) {
      rule3_blocks(P, L, ctrl, f, code, true, om, nE, r3, lane, 2, spec3);
      double mo = 0.0, mn = 0.0;
      for (int t2 = lane; t2 < Nf * Nf; t2 += 32) {
        const double bo = r3[L.o_acc + t2], bn = r3[L.o_acc + Nf * Nf + t2];
        fb[t2] = bo;
        fb[Nf * Nf + t2] = bn;
        mo = fmax(mo, fabs(bo));
        mn = fmax(mn, fabs(bn));
      }
      __syncwarp();
      mo = warp_max(mo);
      mn = warp_max(mn);
      emit_weights(P, fi, d, owner, nbr, f, fn, weighting, mt_lu, mt_perm, fb, mo, mn, win, facecode, lane);
      __syncwarp();
      continue;
    }
    const double* sp;
    int npe;
    if (unsplit) {
      npe = dim == 2 ? P.nf : np;
      cache_amounts(P, wn, om, cache, npe, lane);
      sp = cache;
    } else {
      fill_points_brk(P, ctrl, f, code, true, om, brk, scratch, lane);
      sp = scratch;
      npe = np;
    }
    double mo = 0.0, mn = 0.0;
    for (int t = lane; t < Nf * Nf; t += 32) {
      const int i = t / Nf, j = t % Nf;
      const double bo = block_entry(sp, npe, stride, 0, 2, 2 + Nf, i, j);        // owner <- neighbour
      const double bn = block_entry(sp, npe, stride, 1, 2 + Nf, 2, i, j);        // neighbour <- owner
      fb[t] = bo;
      fb[Nf * Nf + t] = bn;
      mo = fmax(mo, fabs(bo));
      mn = fmax(mn, fabs(bn));
    }
    __syncwarp();
    mo = warp_max(mo);
    mn = warp_max(mn);
    emit_weights(P, fi, d, owner, nbr, f, fn, weighting, mt_lu, mt_perm, fb, mo, mn, win, facecode, lane);
    __syncwarp();                        // fb and the point data are rewritten for the next direction
  }
}

static int weights_face_shm_per_warp(const DevProblem& P) {
  const int np = (P.dim == 2) ? 3 * P.nf : (P.simplex ? P.nf * P.nf : P.K * P.K * P.nf * P.nf);
  const int stride = 2 + 2 * P.Nf;
  int n = P.Nv * P.dim + 6 + np * stride + np * (1 + P.dim) + (P.dim == 2 ? np * stride : 0) + 2 * P.Nf * P.Nf;
  if (P.dim == 3 && !P.simplex) {
    const R3Layout L = r3_layout(P.r, P.K, P.nf, P.Nf);
    n += 2 * (L.Dg + 1) * 3 + P.K * P.nf * (L.Dg + 1) * 3 + L.n;
  }
  return n;
}

// Per-warp workspace of the per-(face, direction) kernels: control points, then the 2D rule's
// point rows or the 3D rule's workspace.
static int weights_shm_per_warp(const DevProblem& P) {
  if (P.dim == 3 && !P.simplex) return P.Nv * P.dim + r3_layout(P.r, P.K, P.nf, P.Nf).n;
  const int np = (P.dim == 3) ? P.nf * P.nf : 3 * P.nf;
  return P.Nv * P.dim + np * (2 + 2 * P.Nf) + 2 * P.Nf * P.Nf;
}

cudaError_t launch_weights(const DevProblem& P, const int32_t* iface, int64_t n_iface, int weighting,
                           const double* mt_lu, const int32_t* mt_perm, double* win, uint32_t* facecode,
                           cudaStream_t s) {
  if (n_iface == 0) return cudaSuccess;
  const int spw = weights_face_shm_per_warp(P);
  int warps = 4;
  while (warps > 1 && (size_t)warps * spw * sizeof(double) > 96 * 1024) warps >>= 1;
  const size_t shmem = (size_t)warps * spw * sizeof(double);
  cudaFuncSetAttribute(weights_face_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
  const int64_t blocks = (n_iface + warps - 1) / warps;
  weights_face_kernel<<<(unsigned)blocks, warps * 32, shmem, s>>>(P, iface, n_iface, weighting, mt_lu, mt_perm, win,
                                                                 facecode, spw);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ boundary faces
// Inflow mode of boundary faces: inflow block B_in = sum a_in phi phi, outflow part likewise.
__global__ void bdr_modes_kernel(DevProblem P, const int32_t* __restrict__ bface, int64_t n_bface,
                                 uint32_t* facecode, int shm_per_warp) {
  extern __shared__ double sh[];
  const int warp_in_block = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_in_block;
  if (item >= n_bface * P.M) return;
  const int64_t bi = item / P.M;
  const int d = (int)(item % P.M);
  const int64_t e = bface[bi * 2];
  const int f = bface[bi * 2 + 1];
  double* wsh = sh + (size_t)warp_in_block * shm_per_warp;
  double* ctrl = wsh;
  double* sp = ctrl + P.Nv * P.dim;
  const int np = face_npoints(P);
  const int Nf = P.Nf;
  const int stride = 2 + 2 * Nf;
  copy_ctrl(P, e, ctrl, lane);
  double om[3] = {P.omega[d * 3 + 0], P.omega[d * 3 + 1], P.omega[d * 3 + 2]};
  double mi = 0.0, mo = 0.0;
  if (P.dim == 3 && !P.simplex) {
    const R3Layout L = r3_layout(P.r, P.K, P.nf, Nf);
    const int spec[6] = {0, 2, 2, 1, 2, 2};            // inflow block, outflow block
    rule3_blocks(P, L, ctrl, f, 0, false, om, nullptr, sp, lane, 2, spec);
    for (int t = lane; t < Nf * Nf; t += 32) {
      mi = fmax(mi, fabs(sp[L.o_acc + t]));
      mo = fmax(mo, fabs(sp[L.o_acc + Nf * Nf + t]));
    }
  } else {
    fill_points(P, ctrl, f, 0, false, om, sp, lane);
    for (int t = lane; t < Nf * Nf; t += 32) {
      const int i = t / Nf, j = t % Nf;
      mi = fmax(mi, fabs(block_entry(sp, np, stride, 0, 2, 2, i, j)));
      mo = fmax(mo, fabs(block_entry(sp, np, stride, 1, 2, 2, i, j)));
    }
  }
  mi = warp_max(mi);
  mo = warp_max(mo);
  if (lane == 0 && mi > 0.0) atomicOr(&facecode[(int64_t)d * P.E + e], (mo > 0.0 ? MODE_MIXED : MODE_PURE) << (2 * f));
}

// 3D boundary faces: one warp per face, all directions.  The mode needs only whether the rule has
// points with g < 0 (inflow) and with g > 0 (outflow): the block B = sum max(-/+g, 0) w phi phi has a
// nonzero diagonal entry exactly then (the basis is a partition of unity).  Directions without roots
// on the edges and on the composite rule's outer lines use the cached composite points' normals;
// the others build the split rule's blocks.
__global__ void bdr_modes3_kernel(DevProblem P, const int32_t* __restrict__ bface, int64_t n_bface,
                                  uint32_t* facecode, int shm_per_warp) {
  extern __shared__ double sh[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t bi = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (bi >= n_bface) return;
  const int64_t e = bface[bi * 2];
  const int f = bface[bi * 2 + 1];
  const R3Layout L = r3_layout(P.r, P.K, P.nf, P.Nf);
  const int Dg = L.Dg, nlines = P.K * P.nf, np = P.K * P.K * P.nf * P.nf, Nf = P.Nf;
  double* ctrl = sh + (size_t)wib * shm_per_warp;
  double* nbase = ctrl + P.Nv * 3;               // [np][3]
  double* nE = nbase + np * 3;                   // [2][Dg+1][3]
  double* nB = nE + 2 * (Dg + 1) * 3;            // [nlines][Dg+1][3]
  double* r3 = nB + nlines * (Dg + 1) * 3;
  copy_ctrl(P, e, ctrl, lane);
  const double* geo = tabp(P, P.off_geo);
  const double* t = tabp(P, P.off_glf_t);
  const double brk0[4] = {0.0, 1.0, 1.0, 1.0};
  for (int q = lane; q < np; q += 32) {
    const PointData pd = face_point(P, brk0, q);
    face_normal(3, P.r, geo, ctrl, f, pd.s0, pd.s1, nbase + 3 * q);
  }
  for (int k = lane; k < 2 * (Dg + 1); k += 32)
    face_normal(3, P.r, geo, ctrl, f, (double)(k / (Dg + 1)), (double)(k % (Dg + 1)) / (double)Dg, nE + 3 * k);
  for (int k = lane; k < nlines * (Dg + 1); k += 32) {
    const int ob = k / (Dg + 1), kk = k % (Dg + 1), v = ob / P.nf, j = ob % P.nf;
    const double lo = (double)v / (double)P.K, hi = (double)(v + 1) / (double)P.K;
    face_normal(3, P.r, geo, ctrl, f, (double)kk / (double)Dg, lo + (hi - lo) * t[j], nB + 3 * k);
  }
  __syncwarp();
  const int spec[6] = {0, 2, 2, 1, 2, 2};
  for (int d = 0; d < P.M; ++d) {
    const double om[3] = {P.omega[d * 3 + 0], P.omega[d * 3 + 1], P.omega[d * 3 + 2]};
    bool root = false;
    double rr[MAX_DG];
    if (lane < 2) {
      line_roots(Dg, om, nE + lane * (Dg + 1) * 3, rr);
      for (int k = 0; k < Dg; ++k) root = root || rr[k] < 1.0;
    }
    for (int ob = lane; ob < nlines; ob += 32) {
      line_roots(Dg, om, nB + ob * (Dg + 1) * 3, rr);
      for (int k = 0; k < Dg; ++k) root = root || rr[k] < 1.0;
    }
    bool in = false, out = false;
    if (!__any_sync(0xffffffffu, root)) {
      for (int q = lane; q < np; q += 32) {
        const double g = dot_omega(3, om, nbase + 3 * q);
        in = in || (g < 0.0);
        out = out || (g > 0.0);
      }
      in = __any_sync(0xffffffffu, in);
      out = __any_sync(0xffffffffu, out);
    } else {
      rule3_blocks(P, L, ctrl, f, 0, false, om, nE, r3, lane, 2, spec);
      double mi = 0.0, mo = 0.0;
      for (int t2 = lane; t2 < Nf * Nf; t2 += 32) {
        mi = fmax(mi, fabs(r3[L.o_acc + t2]));
        mo = fmax(mo, fabs(r3[L.o_acc + Nf * Nf + t2]));
      }
      in = warp_max(mi) > 0.0;
      out = warp_max(mo) > 0.0;
      __syncwarp();
    }
    if (lane == 0 && in) atomicOr(&facecode[(int64_t)d * P.E + e], (out ? MODE_MIXED : MODE_PURE) << (2 * f));
  }
}

cudaError_t launch_bdr_modes(const DevProblem& P, const int32_t* bface, int64_t n_bface, uint32_t* facecode,
                             cudaStream_t s) {
  if (n_bface == 0) return cudaSuccess;
  if (P.dim == 3 && !P.simplex) {
    const R3Layout L = r3_layout(P.r, P.K, P.nf, P.Nf);
    const int np = P.K * P.K * P.nf * P.nf;
    const int spw = P.Nv * 3 + np * 3 + 2 * (L.Dg + 1) * 3 + P.K * P.nf * (L.Dg + 1) * 3 + L.n;
    int warps = 4;
    while (warps > 1 && (size_t)warps * spw * sizeof(double) > 96 * 1024) warps >>= 1;
    const size_t shmem = (size_t)warps * spw * sizeof(double);
    cudaFuncSetAttribute(bdr_modes3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
    bdr_modes3_kernel<<<(unsigned)((n_bface + warps - 1) / warps), warps * 32, shmem, s>>>(P, bface, n_bface, facecode,
                                                                                          spw);
    return cudaGetLastError();
  }
  const int spw = weights_shm_per_warp(P);
  int warps = 4;
  while (warps > 1 && (size_t)warps * spw * sizeof(double) > 96 * 1024) warps >>= 1;
  const size_t shmem = (size_t)warps * spw * sizeof(double);
  cudaFuncSetAttribute(bdr_modes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
  const int64_t items = n_bface * P.M;
  bdr_modes_kernel<<<(unsigned)((items + warps - 1) / warps), warps * 32, shmem, s>>>(P, bface, n_bface, facecode,
                                                                                     spw);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ partial-inflow blocks
// For every (face side, direction) with mode MIXED: B = sum_q a phi_i phi_j (receiving side's
// own face-node basis on both indices), stored at slot mixed_off[d][e] + rank of the face
// among e's mixed faces.
__device__ inline int mixed_rank(uint32_t code, int f) {
  int r = 0;
  for (int g = 0; g < f; ++g) r += (face_mode(code, g) == MODE_MIXED);
  return r;
}

__global__ void mixed_blocks_kernel(DevProblem P, const int32_t* __restrict__ iface, int64_t n_iface,
                                    const int32_t* __restrict__ bface, int64_t n_bface,
                                    const uint32_t* __restrict__ facecode, const int32_t* __restrict__ mixed_off,
                                    double* __restrict__ mixedB, float* __restrict__ mixedB32,
                                    float* __restrict__ mixedB32lo, int shm_per_warp) {
  extern __shared__ double sh[];
  const int warp_in_block = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_in_block;
  const int64_t n_faces = n_iface + n_bface;
  if (item >= n_faces * P.M) return;
  const int64_t fi = item / P.M;
  const int d = (int)(item % P.M);
  int64_t e0, e1 = -1;
  int f0, f1 = -1, code = 0;
  if (fi < n_iface) {
    const int32_t* row = iface + fi * 5;
    e0 = row[0];
    f0 = row[1];
    e1 = row[2];
    f1 = row[3];
    code = row[4];
  } else {
    e0 = bface[(fi - n_iface) * 2];
    f0 = bface[(fi - n_iface) * 2 + 1];
  }
  const uint32_t c0 = facecode[(int64_t)d * P.E + e0];
  const uint32_t c1 = (e1 >= 0) ? facecode[(int64_t)d * P.E + e1] : 0u;
  const bool m0 = face_mode(c0, f0) == MODE_MIXED;
  const bool m1 = (e1 >= 0) && face_mode(c1, f1) == MODE_MIXED;
  if (!m0 && !m1) return;
  double* wsh = sh + (size_t)warp_in_block * shm_per_warp;
  double* ctrl = wsh;
  double* sp = ctrl + P.Nv * P.dim;
  const int np = face_npoints(P);
  const int Nf = P.Nf;
  const int stride = 2 + 2 * Nf;
  copy_ctrl(P, e0, ctrl, lane);
  double om[3] = {P.omega[d * 3 + 0], P.omega[d * 3 + 1], P.omega[d * 3 + 2]};
  const double* B0 = nullptr;       // 3D: the two blocks from the rule's workspace
  const double* B1 = nullptr;
  if (P.dim == 3 && !P.simplex) {
    const R3Layout L = r3_layout(P.r, P.K, P.nf, Nf);
    const int spec[6] = {0, 2, 2, 1, 2 + Nf, 2 + Nf};  // owner's inflow block, neighbour's inflow block
    rule3_blocks(P, L, ctrl, f0, code, e1 >= 0, om, nullptr, sp, lane, 2, spec);
    B0 = sp + L.o_acc;
    B1 = sp + L.o_acc + Nf * Nf;
  } else {
    fill_points(P, ctrl, f0, code, e1 >= 0, om, sp, lane);
  }
  if (m0) {
    const int64_t slot = mixed_off[(int64_t)d * P.E + e0] + mixed_rank(c0, f0);
    for (int t = lane; t < Nf * Nf; t += 32) {
      const double v = B0 ? B0[t] : block_entry(sp, np, stride, 0, 2, 2, t / Nf, t % Nf);
      mixedB[slot * Nf * Nf + t] = v;
      mixedB32[slot * Nf * Nf + t] = (float)v;
      mixedB32lo[slot * Nf * Nf + t] = (float)(v - (double)(float)v);
    }
  }
  if (m1) {
    const int64_t slot = mixed_off[(int64_t)d * P.E + e1] + mixed_rank(c1, f1);
    for (int t = lane; t < Nf * Nf; t += 32) {
      const double v = B1 ? B1[t] : block_entry(sp, np, stride, 1, 2 + Nf, 2 + Nf, t / Nf, t % Nf);
      mixedB[slot * Nf * Nf + t] = v;
      mixedB32[slot * Nf * Nf + t] = (float)v;
      mixedB32lo[slot * Nf * Nf + t] = (float)(v - (double)(float)v);
    }
  }
}

cudaError_t launch_mixed_blocks(const DevProblem& P, const int32_t* iface, int64_t n_iface, const int32_t* bface,
                                int64_t n_bface, const uint32_t* facecode, const int32_t* mixed_off,
                                double* mixedB, float* mixedB32, float* mixedB32lo, cudaStream_t s) {
  const int64_t items = (n_iface + n_bface) * P.M;
  if (items == 0) return cudaSuccess;
  const int spw = weights_shm_per_warp(P);
  int warps = 4;
  while (warps > 1 && (size_t)warps * spw * sizeof(double) > 96 * 1024) warps >>= 1;
  const size_t shmem = (size_t)warps * spw * sizeof(double);
  cudaFuncSetAttribute(mixed_blocks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
  mixed_blocks_kernel<<<(unsigned)((items + warps - 1) / warps), warps * 32, shmem, s>>>(
      P, iface, n_iface, bface, n_bface, facecode, mixed_off, mixedB, mixedB32, mixedB32lo, spw);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ levels
__global__ void levels_init_kernel(int32_t* levels, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    levels[i] = 0;
}

cudaError_t launch_levels_init(const DevProblem& P, int32_t* levels, cudaStream_t s) {
  levels_init_kernel<<<1216, 256, 0, s>>>(levels, (int64_t)P.M * P.E);
  return cudaGetLastError();
}

// level(d,e) = max over kept upwind neighbours of level + 1 (0 without kept in-arcs).  Values
// only grow; repeated until nothing changes, this reaches the longest-path layering.
__global__ void levels_relax_kernel(DevProblem P, const uint32_t* __restrict__ facecode, int32_t* levels,
                                    int* changed) {
  const int64_t n = (int64_t)P.M * P.E;
  const int nfc = P.nfc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = i / P.E, e = i % P.E;
    const uint32_t code = facecode[i];
    int best = 0;
    for (int f = 0; f < nfc; ++f) {
      if (face_mode(code, f) == MODE_NONE || face_lagged(code, f)) continue;
      const int64_t nb = P.nbr[e * nfc + f];
      if (nb < 0) continue;
      const int lv = ((volatile int32_t*)levels)[d * P.E + nb] + 1;
      best = lv > best ? lv : best;
    }
    if (best > levels[i]) {
      levels[i] = best;
      *changed = 1;
    }
  }
}

cudaError_t launch_levels_relax(const DevProblem& P, const uint32_t* facecode, int32_t* levels, int* changed,
                                cudaStream_t s) {
  levels_relax_kernel<<<1216, 256, 0, s>>>(P, facecode, levels, changed);
  return cudaGetLastError();
}

}  // namespace sn
