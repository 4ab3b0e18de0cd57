// Stored-inverse forms of the (element, direction) solve.  The matrix A = G + F_e + M_t of a
// pair (the left-hand side of eq. 21: sigma_t, Omega, the element's factors and its inflow
// faces) is the same in every source iteration, so it is inverted once per problem
// (invert_pair) and a sweep only forms the right-hand side and applies the inverse:
//   psi_e = Ainv (src_e + sum_{inflow faces f} B_f trace_f).
// Stored per pair q = d E + e: Ainv column-major at inv + q N^2 (entry (i, j) at j N + i, so the
// lanes of a segment read each column as one contiguous run), and per inflow face (rank r among
// the pair's inflow faces, in face order, slot fidx[q] + r):
//   2D: the folded block C_f = Ainv B_f (N x Nf, column-major, at fblk + slot N Nf), so that
//       psi_e = Ainv src_e + sum_f C_f trace_f: every lane applies the faces with Nf multiply-adds
//       per face and no exchange, and in the dataflow schedule Ainv src_e is formed before the
//       wait for upwind data;
//   3D: the block B_f itself (Nf x Nf, row-major, at fblk + slot Nf^2; C_f would add 27 x 9
//       entries per face to 27 x 27, too much memory at the largest sizes).
// SN_PREC_FP64_INV keeps doubles and applies them in FP64; SN_PREC_DS_INV keeps (hi, lo) FP32
// pairs of the same FP64 values and applies them in double-single arithmetic on the FP32 pipe.
// The code is written for an element policy El (node counts, face count, face-node maps), so the
// same bodies serve quadrilaterals / hexahedra (TensorEl), triangles (TriEl) and tetrahedra
// (TetEl).
#pragma once

namespace sn {

// ---- element policies
// N, NF: unknowns per element and per face; W: lanes per system (power of two >= N), SPW systems
// per warp; NFC: faces; face_node(f, i): face-node index of volume node i on face f, or -1;
// vol_node(f, fj): volume index of face node fj; trace_node(fn, oc, fj): volume index, in the
// neighbour's numbering, of our face node fj seen through the neighbour's face fn with
// orientation code oc; SLOTS / slot(f): registers for inflow block rows kept across the wait (a
// node lies on at most one face of each slot); AFFINE_TRACE: trace_node is c0 + ci I + cj J in
// the face node's coordinates (I, J) (tensor elements).
template <int DIM, int P_>
struct TensorEl {
  using S = Shape<DIM, P_>;
  static constexpr int DIMV = DIM, N = S::N, NF = S::NF, W = S::W, SPW = S::SPW, NFC = 2 * DIM, NP1 = P_ + 1;
  static constexpr int SLOTS = DIM;
  static constexpr bool AFFINE_TRACE = true;
  __host__ __device__ static constexpr int slot(int f) { return f >> 1; }
  __device__ static int face_node(int f, int i) { return on_face<DIM, P_>(f, i); }
  __host__ __device__ static constexpr int vol_node(int f, int fj) { return fvi<DIM, P_>(f, fj); }
  __device__ static int trace_node(int fn, int oc, int fj) {
    int c0, ci, cj;
    trace_affine<DIM, P_>(fn, oc, c0, ci, cj);
    return c0 + ci * (fj % NP1) + cj * (fj / NP1);
  }
  // all NF trace indices of one face at once (the face's constants computed once)
  __device__ static void trace_nodes(int fn, int oc, int (&t)[NF]) {
    int c0, ci, cj;
    trace_affine<DIM, P_>(fn, oc, c0, ci, cj);
#pragma unroll
    for (int fj = 0; fj < NF; ++fj) t[fj] = c0 + ci * (fj % NP1) + cj * (fj / NP1);
  }
};

// Triangles: faces f0 = v0 v1, f1 = v1 v2, f2 = v2 v0, face nodes in increasing face coordinate
// (tri_edge_node); a neighbour running the shared face the other way (oc = 1) sees face node fj
// as its node P_ - fj.
template <int P_>
struct TriEl {
  static constexpr int DIMV = 2, N = (P_ + 1) * (P_ + 2) / 2, NF = P_ + 1, NP1 = P_ + 1;
  static constexpr int W = N <= 4 ? 4 : (N <= 8 ? 8 : (N <= 16 ? 16 : 32)), SPW = 32 / W, NFC = 3;
  static constexpr int SLOTS = 3;
  static constexpr bool AFFINE_TRACE = false;
  __host__ __device__ static constexpr int slot(int f) { return f; }
  __device__ static int face_node(int f, int i) {
    int out = -1;
#pragma unroll
    for (int j = 0; j <= P_; ++j)
      if (tri_edge_node(P_, f, j) == i) out = j;
    return out;
  }
  __host__ __device__ static constexpr int vol_node(int f, int fj) { return tri_edge_node(P_, f, fj); }
  __device__ static int trace_node(int fn, int oc, int fj) { return tri_edge_node(P_, fn, (oc & 1) ? P_ - fj : fj); }
  __device__ static void trace_nodes(int fn, int oc, int (&t)[NF]) {
#pragma unroll
    for (int fj = 0; fj < NF; ++fj) t[fj] = trace_node(fn, oc, fj);
  }
};

// Straight-sided tetrahedra, P_1 / P_2 DG: face f opposite vertex f, face nodes the face's three
// vertices then (P_2) its edge midpoints (tet_face_node); the neighbour sees our face node fj as
// its face node tet_nbr_face_node(oc, fj).  A flat face is wholly inflow or wholly outflow, so
// no face is ever mixed and one slot per face costs nothing.  The node maps are evaluated at
// compile time into 4-bit fields: face_node(f, .) of a face f (a constant at every call site)
// is one 64-bit immediate, and the trace indices of a neighbour face (fn, oc), known only at
// run time, are one word of a 24-entry constant table -- evaluating the maps' nested selections
// per lane and face cost several hundred instructions per pair.
template <int P_>
struct TetTraceWords {
  uint32_t w[24];                      // [fn * 6 + oc], nibble fj = the trace's volume node
};
template <int P_>
__host__ __device__ constexpr TetTraceWords<P_> tet_trace_words() {
  TetTraceWords<P_> t{};
  for (int fn = 0; fn < 4; ++fn)
    for (int oc = 0; oc < 6; ++oc) {
      uint32_t w = 0;
      for (int fj = 0; fj < (P_ == 1 ? 3 : 6); ++fj)
        w |= (uint32_t)tet_face_node(P_, fn, tet_nbr_face_node(oc, fj)) << (4 * fj);
      t.w[fn * 6 + oc] = w;
    }
  return t;
}
static __constant__ TetTraceWords<1> c_tet_trace1 = tet_trace_words<1>();
static __constant__ TetTraceWords<2> c_tet_trace2 = tet_trace_words<2>();

template <int P_>
struct TetEl {
  static constexpr int DIMV = 3, N = P_ == 1 ? 4 : 10, NF = P_ == 1 ? 3 : 6, NP1 = P_ + 1;
  static constexpr int W = N <= 4 ? 4 : 16, SPW = 32 / W, NFC = 4;
  static constexpr int SLOTS = 4;
  static constexpr bool AFFINE_TRACE = false;
  __host__ __device__ static constexpr int slot(int f) { return f; }
  // nibble i: the face-node index of volume node i on face f, 15 if i is not on f
  __host__ __device__ static constexpr uint64_t face_node_word(int f) {
    uint64_t w = ~0ull;
    for (int j = 0; j < NF; ++j) {
      const int i = tet_face_node(P_, f, j);
      w = (w & ~(15ull << (4 * i))) | ((uint64_t)j << (4 * i));
    }
    return w;
  }
  __device__ static int face_node(int f, int i) {
    const int v = (int)((face_node_word(f) >> (4 * (i & 15))) & 15ull);
    return v == 15 ? -1 : v;
  }
  __host__ __device__ static constexpr int vol_node(int f, int fj) { return tet_face_node(P_, f, fj); }
  __device__ static uint32_t trace_word(int fn, int oc) {
    if constexpr (P_ == 1) return c_tet_trace1.w[fn * 6 + oc];
    else return c_tet_trace2.w[fn * 6 + oc];
  }
  __device__ static int trace_node(int fn, int oc, int fj) { return (int)((trace_word(fn, oc) >> (4 * fj)) & 15u); }
  __device__ static void trace_nodes(int fn, int oc, int (&t)[NF]) {
    const uint32_t w = trace_word(fn, oc);
#pragma unroll
    for (int fj = 0; fj < NF; ++fj) t[fj] = (int)((w >> (4 * fj)) & 15u);
  }
};

// FP64 inflow block row fi of face f: -Omega . FN_f (whole-inflow face) or the stored block of a
// partially-inflow face (slot).
template <class El>
__device__ __forceinline__ void brow_el(const double* blk, const SweepArgs& sa, uint32_t mode, int f, int fi,
                                        int slot, double om0, double om1, double om2, double* Brow) {
  constexpr int N = El::N, NF = El::NF, DIM = El::DIMV;
  if (mode == MODE_PURE) {
    const double* fnm = blk + (DIM + 1) * N * N + f * DIM * NF * NF + fi * NF;
#pragma unroll
    for (int fj = 0; fj < NF; ++fj) {
      double v = om0 * __ldg(fnm + fj);
      v = fma(om1, __ldg(fnm + NF * NF + fj), v);
      if (DIM == 3) v = fma(om2, __ldg(fnm + 2 * NF * NF + fj), v);
      Brow[fj] = -v;
    }
  } else {
    const double* mb = sa.mixedB + (int64_t)slot * NF * NF + fi * NF;
#pragma unroll
    for (int fj = 0; fj < NF; ++fj) Brow[fj] = __ldg(mb + fj);
  }
}

// b += B_f trace_f (FP64) for one inflow face row: the upwind neighbour's trace (new iterate, or
// the previous one through a lagged arc) or the incident flux on the domain boundary.
template <class El, bool DF>
__device__ __forceinline__ void face_rhs_el(const DevProblem& Pb, const SweepArgs& sa, uint32_t code, int f,
                                            int64_t e, int d, const double* Brow, double& b) {
  constexpr int N = El::N, NF = El::NF, NFC = El::NFC;
  const int64_t nb = Pb.nbr[e * NFC + f];
  if (nb >= 0) {
    const bool lag = face_lagged(code, f);
    const double* ps = lag ? sa.psi_old : sa.psi_new;
    const int fn = Pb.nbr_face[e * NFC + f], oc = Pb.orient[e * NFC + f];
    const double* pnb = ps + ((int64_t)d * Pb.E + nb) * N;
    int tix[NF];
    El::trace_nodes(fn, oc, tix);
#pragma unroll
    for (int fj = 0; fj < NF; ++fj) {
      const double* pt = pnb + tix[fj];
      b = fma(Brow[fj], lag ? __ldg(pt) : trace_load<DF>(pt), b);
    }
  } else if (Pb.psi_inc != nullptr) {
    const double* pin = Pb.psi_inc + ((int64_t)d * Pb.n_bdr + Pb.bdr_index[e * NFC + f]) * NF;
#pragma unroll
    for (int fj = 0; fj < NF; ++fj) b = fma(Brow[fj], __ldg(pin + fj), b);
  }
}

// Inverse and inflow blocks of one pair, formed in FP64 by Gauss-Jordan elimination with partial
// pivoting (row-per-lane; see gj32 for the bookkeeping of V in pivot-step order).  A is assembled
// as in body64.  DSOUT: store (hi, lo) FP32 pairs instead of doubles.  2D: after the inverse is
// stored, every lane forms its rows of C_f = Ainv B_f from its stored row of Ainv and the block
// rows held by the face lanes.
template <class El, bool DSOUT>
__device__ __forceinline__ void invert_pair(const DevProblem& Pb, const SweepArgs& sa, int64_t q, bool valid,
                                            int lane) {
  constexpr int N = El::N, NF = El::NF, W = El::W, DIM = El::DIMV, NFC = El::NFC;
  constexpr bool FOLD = DIM == 2;
  constexpr unsigned FULL = 0xffffffffu;
  const int i = lane % W;
  const int64_t E = Pb.E;
  const int d = valid ? (int)(q / E) : 0;
  const int64_t e = valid ? q % E : 0;
  const bool row = valid && (i < N);
  const double om0 = Pb.omega[d * 3 + 0], om1 = Pb.omega[d * 3 + 1], om2 = Pb.omega[d * 3 + 2];
  const double* blk = Pb.elem + e * Pb.blk;
  auto put = [&](int64_t idx, double x, double* base) {
    if constexpr (DSOUT) {
      float2 v;
      ds_split(x, v.x, v.y);
      reinterpret_cast<float2*>(base)[idx] = v;
    } else {
      base[idx] = x;
    }
  };
  auto get = [&](int64_t idx, const double* base) -> double {
    if constexpr (DSOUT) {
      const float2 v = reinterpret_cast<const float2*>(base)[idx];
      return (double)v.x + (double)v.y;
    } else {
      return base[idx];
    }
  };
  double a[N];
  if (row) {
    const double st = Pb.sig_t[e];
    static_for<0, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      double v = om0 * __ldg(blk + j * N + i);
      v = fma(om1, __ldg(blk + N * N + j * N + i), v);
      if (DIM == 3) v = fma(om2, __ldg(blk + 2 * N * N + j * N + i), v);
      a[j] = fma(st, __ldg(blk + DIM * N * N + j * N + i), v);
    });
  } else {
    static_for<0, N>([&](auto jconst) { a[decltype(jconst)::value] = 0.0; });
  }
  const uint32_t code = valid ? sa.facecode[q] : 0u;
  const int mbase = (valid && (code & 0xAAAu)) ? sa.mixed_off[q] : 0;
  const int64_t bidx = valid ? sa.fidx[q] : 0;
  double Bkeep[FOLD ? NFC : 1][NF];       // 2D: this lane's block row of each inflow face (else 0)
  if constexpr (FOLD)
    static_for<0, NFC>([&](auto fconst) {
      static_for<0, NF>([&](auto jconst) { Bkeep[decltype(fconst)::value][decltype(jconst)::value] = 0.0; });
    });
  int mrank = 0, rank = 0;
  static_for<0, NFC>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    const uint32_t mode = face_mode(code, f);
    const int fi = row ? El::face_node(f, i) : -1;
    if (mode != MODE_NONE && fi >= 0) {
      double Brow[NF];
      brow_el<El>(blk, sa, mode, f, fi, mbase + mrank, om0, om1, om2, Brow);
      const int64_t o = (bidx + rank) * (NF * NF) + fi * NF;
      static_for<0, NF>([&](auto jconst) {
        constexpr int fj = decltype(jconst)::value;
        a[El::vol_node(f, fj)] += Brow[fj];
        if constexpr (FOLD) Bkeep[f][fj] = Brow[fj];
        else put(o + fj, Brow[fj], sa.fblk);
      });
    }
    if (mode == MODE_MIXED) ++mrank;
    if (mode != MODE_NONE) ++rank;
  });
  double v[N];
  int plk[N];
  bool used = !row;
  double myinv = 0.0;
  int myk = -1;
  static_for<0, N>([&](auto jconst) { v[decltype(jconst)::value] = 0.0; });
  static_for<0, N>([&](auto kconst) {
    constexpr int k = decltype(kconst)::value;
    const unsigned hw = (unsigned)((unsigned long long)__double_as_longlong(a[k]) >> 32);
    const unsigned key = used ? 0u : ((hw & 0x7fffffe0u) | (unsigned)(31 - lane));
    const int pl = seg_argmax_key<W>(key, lane);
    plk[k] = pl;
    const double inv = nr_rcp(__shfl_sync(FULL, a[k], pl, W));
    const bool me = (lane == pl);
    if (me) {
      used = true;
      myk = k;
      myinv = inv;
      v[k] = 1.0;
    }
    const double l = me ? 0.0 : a[k] * inv;
    static_for<k + 1, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      a[j] = fma(-l, __shfl_sync(FULL, a[j], pl, W), a[j]);
    });
    static_for<0, k + 1>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      v[j] = fma(-l, __shfl_sync(FULL, v[j], pl, W), v[j]);
    });
  });
  // the lane of step k holds row k of the inverse: Ainv[k][row of plk[m]] = v[m] / pivot
  if (row && myk >= 0) {
    const int64_t o = q * (N * N) + myk;
    static_for<0, N>([&](auto mconst) {
      constexpr int m = decltype(mconst)::value;
      put(o + (plk[m] % W) * N, v[m] * myinv, sa.inv);
    });
  }
  if constexpr (FOLD) {
    __syncwarp();                        // the segment's stored rows are visible to all its lanes
    int r2 = 0;
    static_for<0, NFC>([&](auto fconst) {
      constexpr int f = decltype(fconst)::value;
      const uint32_t mode = face_mode(code, f);
      // block rows of face f from the face lanes (exchanged by every lane, used if f is inflow)
      double bsh[NF][NF];
      static_for<0, NF>([&](auto iconst) {
        constexpr int fi = decltype(iconst)::value;
        static_for<0, NF>([&](auto jconst) {
          constexpr int fj = decltype(jconst)::value;
          bsh[fi][fj] = __shfl_sync(FULL, Bkeep[f][fj], El::vol_node(f, fi), W);
        });
      });
      if (row && mode != MODE_NONE) {
        double arow[NF];
        static_for<0, NF>([&](auto iconst) {
          constexpr int fi = decltype(iconst)::value;
          arow[fi] = get(q * (N * N) + El::vol_node(f, fi) * N + i, sa.inv);
        });
        const int64_t o = (bidx + r2) * (N * NF) + i;
        static_for<0, NF>([&](auto jconst) {
          constexpr int fj = decltype(jconst)::value;
          double c = 0.0;
          static_for<0, NF>([&](auto iconst) {
            constexpr int fi = decltype(iconst)::value;
            c = fma(arow[fi], bsh[fi][fj], c);
          });
          put(o + fj * N, c, sa.fblk);
        });
      }
      if (mode != MODE_NONE) ++r2;
    });
  }
}

// ------------------------------------------------------------------ FP64 application, stored blocks (3D)
template <class El, bool DF>
__device__ __forceinline__ void bodyinv_blocks(const DevProblem& Pb, const SweepArgs& sa, int32_t pr, bool valid,
                                               int lane) {
  constexpr int N = El::N, NF = El::NF, W = El::W, DIM = El::DIMV;
  constexpr unsigned FULL = 0xffffffffu;
  constexpr bool BPRE = DIM == 2;      // inflow block rows held in registers across the wait (2D)
  const int i = lane % W;
  const int M = Pb.M;
  const int64_t E = Pb.E;
  const int64_t e = pr / M;
  const int d = pr % M;
  const int64_t q = (int64_t)d * E + e;
  const bool row = valid && (i < N);
  double ainv[N];
  double b = 0.0;
  if (row) {
    const double* ai = sa.inv + q * (N * N) + i;
    static_for<0, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      ainv[j] = __ldcs(ai + j * N);      // read once per sweep: streamed past the caches
    });
    if (Pb.q_dir != nullptr) {
      const double* blk = Pb.elem + e * Pb.blk;
      const double* qd = Pb.q_dir + q * N;
#pragma unroll
      for (int j = 0; j < N; ++j) b = fma(__ldg(blk + DIM * N * N + i * N + j), qd[j], b);
    }
  } else {
    static_for<0, N>([&](auto jconst) { ainv[decltype(jconst)::value] = 0.0; });
  }
  const uint32_t code = valid ? sa.facecode[q] : 0u;
  const int64_t bidx = valid ? sa.fidx[q] : 0;
  double Bax[BPRE ? El::SLOTS : 1][NF];
  if constexpr (BPRE) {
    int rank = 0;
    static_for<0, El::NFC>([&](auto fconst) {
      constexpr int f = decltype(fconst)::value;
      const uint32_t mode = face_mode(code, f);
      const int fi = row ? El::face_node(f, i) : -1;
      if (mode != MODE_NONE && fi >= 0) {
        const double* br = sa.fblk + (bidx + rank) * (NF * NF) + fi * NF;
        static_for<0, NF>([&](auto jconst) {
          Bax[El::slot(f)][decltype(jconst)::value] = __ldcs(br + decltype(jconst)::value);
        });
      }
      if (mode != MODE_NONE) ++rank;
    });
  }
  if constexpr (DF) wait_upwind_n<El::NFC>(Pb, sa, code, e, d, valid);
  else {
    pdl_wait();                          // sources and upwind traces come from earlier launches
    pdl_launch_dependents();
  }
  if (row) b += sa.src[e * N + i];
  int rank = 0;
  static_for<0, El::NFC>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    const uint32_t mode = face_mode(code, f);
    const int fi = row ? El::face_node(f, i) : -1;
    if (mode != MODE_NONE && fi >= 0) {
      if constexpr (BPRE) {
        face_rhs_el<El, DF>(Pb, sa, code, f, e, d, Bax[El::slot(f)], b);
      } else {
        double Brow[NF];
        const double* br = sa.fblk + (bidx + rank) * (NF * NF) + fi * NF;
        static_for<0, NF>([&](auto jconst) { Brow[decltype(jconst)::value] = __ldcs(br + decltype(jconst)::value); });
        face_rhs_el<El, DF>(Pb, sa, code, f, e, d, Brow, b);
      }
    }
    if (mode != MODE_NONE) ++rank;
  });
  // psi_i = sum_j Ainv[i][j] b_j, b_j from lane j of the segment; two accumulation chains
  double x0 = 0.0, x1 = 0.0;
  static_for<0, N>([&](auto jconst) {
    constexpr int j = decltype(jconst)::value;
    const double bj = __shfl_sync(FULL, b, j, W);
    if (j & 1) x1 = fma(ainv[j], bj, x1);
    else x0 = fma(ainv[j], bj, x0);
  });
  if (row) {
    const double x = x0 + x1;
    const int64_t o = q * N + i;
    sa.psi_new[o] = x;
    if (sa.psi_new_h != nullptr) {
      const float h = (float)x;
      sa.psi_new_h[o] = h;
      sa.psi_new_l[o] = (float)(x - (double)h);
    }
  }
  publish<DF, W>(Pb, sa, e, d, valid, i);
}

// ------------------------------------------------------------------ double-single application, stored blocks (3D)
// The right-hand side is accumulated and the inverse applied in double-single arithmetic
// (error-free FP32 products and sums, ~2^-48 relative), from the (hi, lo) splits of the stored
// FP64 inverse and blocks, of the source and of the upwind traces; no FP64 instruction on the
// solve path except the final psi = hi + lo.
template <class El, bool DF>
__device__ __forceinline__ void bodydsinv_blocks(const DevProblem& Pb, const SweepArgs& sa, int32_t pr, bool valid,
                                                 int lane) {
  constexpr int N = El::N, NF = El::NF, W = El::W, DIM = El::DIMV, NFC = El::NFC;
  constexpr unsigned FULL = 0xffffffffu;
  constexpr bool BPRE = DIM == 2;
  const int i = lane % W;
  const int M = Pb.M;
  const int64_t E = Pb.E;
  const int64_t e = pr / M;
  const int d = pr % M;
  const int64_t q = (int64_t)d * E + e;
  const bool row = valid && (i < N);
  const float2* inv2 = reinterpret_cast<const float2*>(sa.inv);
  const float2* fb2 = reinterpret_cast<const float2*>(sa.fblk);
  float2 A[N];
  float rbh = 0.0f, rbl = 0.0f;
  if (row) {
    const float2* ai = inv2 + q * (N * N) + i;
    static_for<0, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      A[j] = __ldcs(ai + j * N);
    });
    if (Pb.q_dir != nullptr) {           // direction-dependent source (tests): FP64, then split
      const double* blk = Pb.elem + e * Pb.blk;
      const double* qd = Pb.q_dir + q * N;
      double qb = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) qb = fma(__ldg(blk + DIM * N * N + i * N + j), qd[j], qb);
      ds_split(qb, rbh, rbl);
    }
  } else {
    static_for<0, N>([&](auto jconst) { A[decltype(jconst)::value] = make_float2(0.0f, 0.0f); });
  }
  const uint32_t code = valid ? sa.facecode[q] : 0u;
  const int64_t bidx = valid ? sa.fidx[q] : 0;
  int64_t nbv[NFC];
  int fov[NFC];
  static_for<0, NFC>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    nbv[f] = valid ? Pb.nbr[e * NFC + f] : -1;
    fov[f] = valid ? (Pb.nbr_face[e * NFC + f] | (Pb.orient[e * NFC + f] << 8)) : 0;
  });
  float2 Bax[BPRE ? El::SLOTS : 1][NF];
  if constexpr (BPRE) {
    int rank = 0;
    static_for<0, NFC>([&](auto fconst) {
      constexpr int f = decltype(fconst)::value;
      const uint32_t mode = face_mode(code, f);
      const int fi = row ? El::face_node(f, i) : -1;
      if (mode != MODE_NONE && fi >= 0) {
        const float2* br = fb2 + (bidx + rank) * (NF * NF) + fi * NF;
        static_for<0, NF>([&](auto jconst) {
          Bax[El::slot(f)][decltype(jconst)::value] = __ldcs(br + decltype(jconst)::value);
        });
      }
      if (mode != MODE_NONE) ++rank;
    });
  }
  if constexpr (DF) {
    wait_upwind_n<NFC>(Pb, sa, code, e, d, valid);
  } else {
    pdl_wait();                          // sources and upwind traces come from earlier launches
    pdl_launch_dependents();
  }
  if (row) ds_add(rbh, rbl, sa.src_h[e * N + i], sa.src_l[e * N + i]);
  float sh2 = 0.0f, sl2 = 0.0f;          // second accumulation chain for the face terms
  int rank = 0;
  static_for<0, NFC>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    const uint32_t mode = face_mode(code, f);
    const int fi = row ? El::face_node(f, i) : -1;
    const int64_t nb = nbv[f];
    if (mode != MODE_NONE && fi >= 0 && (nb >= 0 || Pb.psi_inc != nullptr)) {
      float2 B[NF];
      if constexpr (BPRE) {
        static_for<0, NF>([&](auto jconst) { B[decltype(jconst)::value] = Bax[El::slot(f)][decltype(jconst)::value]; });
      } else {
        const float2* br = fb2 + (bidx + rank) * (NF * NF) + fi * NF;
        static_for<0, NF>([&](auto jconst) { B[decltype(jconst)::value] = __ldcs(br + decltype(jconst)::value); });
      }
      if (nb >= 0) {                     // upwind neighbour's (hi, lo) split of the trace
        const bool lag = face_lagged(code, f);
        // hexahedra: the trace index is affine in the face node, c0 + ci I + cj J, with three
        // registers instead of a table of NF; tetrahedra: the table
        int c0 = 0;
        [[maybe_unused]] int ci = 0, cj = 0;
        [[maybe_unused]] int tix[El::AFFINE_TRACE ? 1 : NF];
        if constexpr (El::AFFINE_TRACE) trace_affine<DIM, El::NP1 - 1>(fov[f] & 0xff, fov[f] >> 8, c0, ci, cj);
        else El::trace_nodes(fov[f] & 0xff, fov[f] >> 8, tix);
        const int64_t base = ((int64_t)d * E + nb) * N + c0;
        const float* ph_ = (lag ? sa.psi_old_h : sa.psi_new_h) + base;
        const float* pl_ = (lag ? sa.psi_old_l : sa.psi_new_l) + base;
#pragma unroll
        for (int fj = 0; fj < NF; ++fj) {
          int o;
          if constexpr (El::AFFINE_TRACE) o = ci * (fj % El::NP1) + cj * (fj / El::NP1);
          else o = tix[fj];
          float th, tl, qh, ql;
          if (!lag && DF) {
            th = __ldcg(ph_ + o);
            tl = __ldcg(pl_ + o);
          } else {
            th = __ldg(ph_ + o);
            tl = __ldg(pl_ + o);
          }
          ds_mul(B[fj].x, B[fj].y, th, tl, qh, ql);
          if (fj & 1) ds_add(sh2, sl2, qh, ql);
          else ds_add(rbh, rbl, qh, ql);
        }
      } else {                           // incident flux on the domain boundary
        const double* pin = Pb.psi_inc + ((int64_t)d * Pb.n_bdr + Pb.bdr_index[e * NFC + f]) * NF;
#pragma unroll
        for (int fj = 0; fj < NF; ++fj) {
          float th, tl, qh, ql;
          ds_split(__ldg(pin + fj), th, tl);
          ds_mul(B[fj].x, B[fj].y, th, tl, qh, ql);
          ds_add(rbh, rbl, qh, ql);
        }
      }
    }
    if (mode != MODE_NONE) ++rank;
  });
  ds_add(rbh, rbl, sh2, sl2);
  // psi_i = sum_j Ainv[i][j] b_j in double-single, four independent chains
  float xh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, xl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  static_for<0, N>([&](auto jconst) {
    constexpr int j = decltype(jconst)::value;
    const float bjh = __shfl_sync(FULL, rbh, j, W);
    const float bjl = __shfl_sync(FULL, rbl, j, W);
    float ph, pl;
    ds_mul(A[j].x, A[j].y, bjh, bjl, ph, pl);
    ds_add(xh[j & 3], xl[j & 3], ph, pl);
  });
  ds_add(xh[0], xl[0], xh[1], xl[1]);
  ds_add(xh[2], xl[2], xh[3], xl[3]);
  ds_add(xh[0], xl[0], xh[2], xl[2]);
  if (row) {
    const int64_t o = q * N + i;
    sa.psi_new_h[o] = xh[0];
    sa.psi_new_l[o] = xl[0];
    sa.psi_new[o] = (double)xh[0] + (double)xl[0];
  }
  publish<DF, W>(Pb, sa, e, d, valid, i);
}

// ------------------------------------------------------------------ folded blocks (2D)
// psi_i = sum_j Ainv[i][j] src_j + sum_{inflow f} sum_fj C_f[i][fj] trace_f[fj]: every lane loads
// the face traces itself (the same addresses across the segment) and applies its rows of C_f; the
// source part needs the segment's right-hand side values (exchanged by shuffles) and, in the
// dataflow schedule, is formed before the wait (the source was written by an earlier launch).
template <class El, bool DF>
__device__ __forceinline__ void bodyinv_fold(const DevProblem& Pb, const SweepArgs& sa, int32_t pr, bool valid,
                                             int lane) {
  constexpr int N = El::N, NF = El::NF, W = El::W, DIM = El::DIMV, NFC = El::NFC;
  constexpr unsigned FULL = 0xffffffffu;
  const int i = lane % W;
  const int M = Pb.M;
  const int64_t E = Pb.E;
  const int64_t e = pr / M;
  const int d = pr % M;
  const int64_t q = (int64_t)d * E + e;
  const bool row = valid && (i < N);
  const uint32_t code = valid ? sa.facecode[q] : 0u;
  const int64_t bidx = valid ? sa.fidx[q] : 0;
  double ainv[N];
  double Cf[NFC][NF];
  double bs = 0.0;
  if (row) {
    const double* ai = sa.inv + q * (N * N) + i;
    static_for<0, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      ainv[j] = __ldcs(ai + j * N);      // read once per sweep: streamed past the caches
    });
    if (Pb.q_dir != nullptr) {
      const double* blk = Pb.elem + e * Pb.blk;
      const double* qd = Pb.q_dir + q * N;
#pragma unroll
      for (int j = 0; j < N; ++j) bs = fma(__ldg(blk + DIM * N * N + i * N + j), qd[j], bs);
    }
  } else {
    static_for<0, N>([&](auto jconst) { ainv[decltype(jconst)::value] = 0.0; });
  }
  int rank = 0;
  static_for<0, NFC>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    const uint32_t mode = face_mode(code, f);
    const double* cf = sa.fblk + (bidx + rank) * (N * NF) + i;
    static_for<0, NF>([&](auto jconst) {
      constexpr int fj = decltype(jconst)::value;
      Cf[f][fj] = (row && mode != MODE_NONE) ? __ldcs(cf + fj * N) : 0.0;
    });
    if (mode != MODE_NONE) ++rank;
  });
  int64_t nbv[NFC];
  int fov[NFC];
  static_for<0, NFC>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    nbv[f] = valid ? Pb.nbr[e * NFC + f] : -1;
    fov[f] = valid ? (Pb.nbr_face[e * NFC + f] | (Pb.orient[e * NFC + f] << 8)) : 0;
  });
  double y0 = 0.0, y1 = 0.0;
  auto apply_src = [&]() {
    if (row) bs += sa.src[e * N + i];
    static_for<0, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      const double bj = __shfl_sync(FULL, bs, j, W);
      if (j & 1) y1 = fma(ainv[j], bj, y1);
      else y0 = fma(ainv[j], bj, y0);
    });
  };
  if constexpr (DF) {
    apply_src();
    wait_upwind_n<NFC>(Pb, sa, code, e, d, valid);
  } else {
    pdl_wait();                          // sources and upwind traces come from earlier launches
    pdl_launch_dependents();
    apply_src();
  }
  double x = y0 + y1;
  static_for<0, NFC>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    const uint32_t mode = face_mode(code, f);
    const int64_t nb = nbv[f];
    if (row && mode != MODE_NONE) {
      if (nb >= 0) {
        const bool lag = face_lagged(code, f);
        const double* pnb = (lag ? sa.psi_old : sa.psi_new) + ((int64_t)d * E + nb) * N;
        int tix[NF];
        El::trace_nodes(fov[f] & 0xff, fov[f] >> 8, tix);
#pragma unroll
        for (int fj = 0; fj < NF; ++fj) {
          const double* pt = pnb + tix[fj];
          x = fma(Cf[f][fj], lag ? __ldg(pt) : trace_load<DF>(pt), x);
        }
      } else if (Pb.psi_inc != nullptr) {
        const double* pin = Pb.psi_inc + ((int64_t)d * Pb.n_bdr + Pb.bdr_index[e * NFC + f]) * NF;
#pragma unroll
        for (int fj = 0; fj < NF; ++fj) x = fma(Cf[f][fj], __ldg(pin + fj), x);
      }
    }
  });
  if (row) {
    const int64_t o = q * N + i;
    sa.psi_new[o] = x;
    if (sa.psi_new_h != nullptr) {
      const float h = (float)x;
      sa.psi_new_h[o] = h;
      sa.psi_new_l[o] = (float)(x - (double)h);
    }
  }
  publish<DF, W>(Pb, sa, e, d, valid, i);
}

template <class El, bool DF>
__device__ __forceinline__ void bodydsinv_fold(const DevProblem& Pb, const SweepArgs& sa, int32_t pr, bool valid,
                                               int lane) {
  constexpr int N = El::N, NF = El::NF, W = El::W, DIM = El::DIMV, NFC = El::NFC;
  constexpr unsigned FULL = 0xffffffffu;
  const int i = lane % W;
  const int M = Pb.M;
  const int64_t E = Pb.E;
  const int64_t e = pr / M;
  const int d = pr % M;
  const int64_t q = (int64_t)d * E + e;
  const bool row = valid && (i < N);
  const uint32_t code = valid ? sa.facecode[q] : 0u;
  const int64_t bidx = valid ? sa.fidx[q] : 0;
  const float2* inv2 = reinterpret_cast<const float2*>(sa.inv);
  const float2* fb2 = reinterpret_cast<const float2*>(sa.fblk);
  float2 A[N];
  float2 Cf[NFC][NF];
  float bh = 0.0f, bl = 0.0f;
  if (row) {
    const float2* ai = inv2 + q * (N * N) + i;
    static_for<0, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      A[j] = __ldcs(ai + j * N);
    });
    if (Pb.q_dir != nullptr) {           // direction-dependent source (tests): FP64, then split
      const double* blk = Pb.elem + e * Pb.blk;
      const double* qd = Pb.q_dir + q * N;
      double qb = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) qb = fma(__ldg(blk + DIM * N * N + i * N + j), qd[j], qb);
      ds_split(qb, bh, bl);
    }
  } else {
    static_for<0, N>([&](auto jconst) { A[decltype(jconst)::value] = make_float2(0.0f, 0.0f); });
  }
  int rank = 0;
  static_for<0, NFC>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    const uint32_t mode = face_mode(code, f);
    const float2* cf = fb2 + (bidx + rank) * (N * NF) + i;
    static_for<0, NF>([&](auto jconst) {
      constexpr int fj = decltype(jconst)::value;
      Cf[f][fj] = (row && mode != MODE_NONE) ? __ldcs(cf + fj * N) : make_float2(0.0f, 0.0f);
    });
    if (mode != MODE_NONE) ++rank;
  });
  int64_t nbv[NFC];
  int fov[NFC];
  static_for<0, NFC>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    nbv[f] = valid ? Pb.nbr[e * NFC + f] : -1;
    fov[f] = valid ? (Pb.nbr_face[e * NFC + f] | (Pb.orient[e * NFC + f] << 8)) : 0;
  });
  // y = Ainv src in double-single, four independent chains
  float xh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, xl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  auto apply_src = [&]() {
    if (row) ds_add(bh, bl, sa.src_h[e * N + i], sa.src_l[e * N + i]);
    static_for<0, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      const float bjh = __shfl_sync(FULL, bh, j, W);
      const float bjl = __shfl_sync(FULL, bl, j, W);
      float ph, pl;
      ds_mul(A[j].x, A[j].y, bjh, bjl, ph, pl);
      ds_add(xh[j & 3], xl[j & 3], ph, pl);
    });
  };
  if constexpr (DF) {
    apply_src();
    wait_upwind_n<NFC>(Pb, sa, code, e, d, valid);
  } else {
    pdl_wait();                          // sources and upwind traces come from earlier launches
    pdl_launch_dependents();
    apply_src();
  }
  // faces: C_f trace_f into chains 2 and 3 (even / odd face nodes)
  static_for<0, NFC>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    const uint32_t mode = face_mode(code, f);
    const int64_t nb = nbv[f];
    if (row && mode != MODE_NONE) {
      if (nb >= 0) {
        const bool lag = face_lagged(code, f);
        const int64_t base = ((int64_t)d * E + nb) * N;
        const float* ph_ = (lag ? sa.psi_old_h : sa.psi_new_h) + base;
        const float* pl_ = (lag ? sa.psi_old_l : sa.psi_new_l) + base;
        int tix[NF];
        El::trace_nodes(fov[f] & 0xff, fov[f] >> 8, tix);
#pragma unroll
        for (int fj = 0; fj < NF; ++fj) {
          const int o = tix[fj];
          float th, tl, qh, ql;
          if (!lag && DF) {
            th = __ldcg(ph_ + o);
            tl = __ldcg(pl_ + o);
          } else {
            th = __ldg(ph_ + o);
            tl = __ldg(pl_ + o);
          }
          ds_mul(Cf[f][fj].x, Cf[f][fj].y, th, tl, qh, ql);
          ds_add(xh[2 + (fj & 1)], xl[2 + (fj & 1)], qh, ql);
        }
      } else if (Pb.psi_inc != nullptr) {
        const double* pin = Pb.psi_inc + ((int64_t)d * Pb.n_bdr + Pb.bdr_index[e * NFC + f]) * NF;
#pragma unroll
        for (int fj = 0; fj < NF; ++fj) {
          float th, tl, qh, ql;
          ds_split(__ldg(pin + fj), th, tl);
          ds_mul(Cf[f][fj].x, Cf[f][fj].y, th, tl, qh, ql);
          ds_add(xh[2 + (fj & 1)], xl[2 + (fj & 1)], qh, ql);
        }
      }
    }
  });
  ds_add(xh[0], xl[0], xh[1], xl[1]);
  ds_add(xh[2], xl[2], xh[3], xl[3]);
  ds_add(xh[0], xl[0], xh[2], xl[2]);
  if (row) {
    const int64_t o = q * N + i;
    sa.psi_new_h[o] = xh[0];
    sa.psi_new_l[o] = xl[0];
    sa.psi_new[o] = (double)xh[0] + (double)xl[0];
  }
  publish<DF, W>(Pb, sa, e, d, valid, i);
}

// The two application forms: folded blocks in 2D, stored blocks in 3D.
template <class El, bool DF>
__device__ __forceinline__ void bodyinv(const DevProblem& Pb, const SweepArgs& sa, int32_t pr, bool valid, int lane) {
  if constexpr (El::DIMV == 2) bodyinv_fold<El, DF>(Pb, sa, pr, valid, lane);
  else bodyinv_blocks<El, DF>(Pb, sa, pr, valid, lane);
}

template <class El, bool DF>
__device__ __forceinline__ void bodydsinv(const DevProblem& Pb, const SweepArgs& sa, int32_t pr, bool valid,
                                          int lane) {
  if constexpr (El::DIMV == 2) bodydsinv_fold<El, DF>(Pb, sa, pr, valid, lane);
  else bodydsinv_blocks<El, DF>(Pb, sa, pr, valid, lane);
}
}  // namespace sn
