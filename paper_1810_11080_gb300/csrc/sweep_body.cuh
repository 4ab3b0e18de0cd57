// Device code of one (element, direction) solve, shared by the single-problem sweep kernels
// (sweep.cu) and the batched kernels (batch.cu).  See sweep.cu for the method.
#pragma once
#include <type_traits>
#include "devmath.cuh"

namespace sn {

template <int I, int END, class F>
__device__ __forceinline__ void static_for(F&& fn) {
  if constexpr (I < END) {
    fn(std::integral_constant<int, I>{});
    static_for<I + 1, END>(fn);
  }
}

// 1/x by Newton-Raphson (r <- r + r (1 - x r), two steps) from the hardware reciprocal
// approximation: relative error below 2^-52 for normal x, at a third of the FP64 pipe slots of
// an IEEE division.
__device__ __forceinline__ double nr_rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// Volume node index of face node fj of face f (compile-time).
template <int DIM, int P_>
__host__ __device__ constexpr int fvi(int f, int fj) {
  return face_vol_index(DIM, P_, f, fj % (P_ + 1), fj / (P_ + 1));
}

template <int DIM, int P_>
struct Shape {
  static constexpr int NP1 = P_ + 1;
  static constexpr int N = ipow(NP1, DIM);
  static constexpr int NF = ipow(NP1, DIM - 1);
  static constexpr int W = N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : 32;
  static constexpr int SPW = 32 / W;
  // Double-single form: inflow face blocks enter the matrix before the wait (and are formed
  // again after it for the right-hand side) in 2D; in 3D (6 faces of up to 9 nodes) forming them
  // twice costs more than it saves, and all face work follows the wait.
  static constexpr bool FACES_PRE = DIM == 2;
};

// Resident 128-thread blocks per SM the sweep kernels are compiled for, i.e. a register budget
// of 65536 / (128 minb) per thread.  Double-single form: 96 registers hold a 2D row without
// spills; the 3D p = 2 row (N = 27) gets 128 (a few spilled values), which measured faster than
// 168 without spills because the next level's blocks then fit beside the current level's.  The
// FP64 and FP64-residual forms get budgets without spills.
template <int DIM, int P_, int PREC>
constexpr int sweep_minb() {
  if (PREC == SN_PREC_FP64_INV) return DIM == 2 ? 5 : 3;
  if (PREC == SN_PREC_DS_INV) return DIM == 2 ? 5 : 4;
  if (DIM == 3 && P_ == 2) return PREC == SN_PREC_MIXED_DS ? 4 : (PREC == SN_PREC_FP64 ? 3 : 2);
  if (PREC == SN_PREC_FP64) return DIM == 2 ? 6 : 5;
  return PREC == SN_PREC_MIXED ? 4 : 5;
}

// Face-node index of volume node i on local face f, or -1.
template <int DIM, int P_>
__device__ __forceinline__ int on_face(int f, int i) {
  constexpr int n = P_ + 1;
  const int t0 = i % n, t1 = (i / n) % n, t2 = (DIM == 3) ? i / (n * n) : 0;
  const int axis = f >> 1, side = f & 1;
  const int ta = axis == 0 ? t0 : (axis == 1 ? t1 : t2);
  if (ta != side * P_) return -1;
  const int o0 = axis == 0 ? t1 : t0;
  const int o1 = axis == 2 ? t1 : t2;
  return DIM == 2 ? o0 : o0 + n * o1;
}

// Volume index, in the neighbour's node numbering, of face node fj = I + (p+1) J of our face,
// written as c0 + ci I + cj J for the neighbour's face fn and orientation code oc (bit 2 swaps
// the face axes, bit 0 flips the first, bit 1 the second): the same map as orient_map_idx
// followed by face_vol_index, with the per-face constants computed once.
template <int DIM, int P_>
__device__ __forceinline__ void trace_affine(int fn, int oc, int& c0, int& ci, int& cj) {
  constexpr int n = P_ + 1;
  const int axis = fn >> 1, side = fn & 1;
  if constexpr (DIM == 2) {
    const int A = axis == 0 ? side * P_ : n * side * P_;
    const int B = axis == 0 ? n : 1;
    const bool flip = oc & 1;
    c0 = flip ? A + B * P_ : A;
    ci = flip ? -B : B;
    cj = 0;
  } else {
    // neighbour face coordinates (t0, t1) -> volume index A + B0 t0 + B1 t1
    const int A = axis == 0 ? side * P_ : (axis == 1 ? n * side * P_ : n * n * side * P_);
    const int B0 = axis == 0 ? n : 1;
    const int B1 = axis == 2 ? n : n * n;
    const bool f0 = oc & 1, f1 = oc & 2, sw = oc & 4;
    // t0 = f0 ? p - u0 : u0, t1 = f1 ? p - u1 : u1, (u0, u1) = sw ? (J, I) : (I, J)
    const int b0 = f0 ? -B0 : B0, b1 = f1 ? -B1 : B1;
    c0 = A + (f0 ? B0 * P_ : 0) + (f1 ? B1 * P_ : 0);
    ci = sw ? b1 : b0;
    cj = sw ? b0 : b1;
  }
}

// ---- double-single (FP32 pair) arithmetic: error-free transformations (Knuth two-sum,
// fma-based two-product), ~2^-48 relative precision on the FP32 pipe.
__device__ __forceinline__ void ds_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (ph, pl) = (xh + xl)(yh + yl) to first order in the low parts.
__device__ __forceinline__ void ds_mul(float xh, float xl, float yh, float yl, float& ph, float& pl) {
  ph = xh * yh;
  pl = fmaf(xh, yh, -ph);
  pl = fmaf(xh, yl, pl);
  pl = fmaf(xl, yh, pl);
}
// (sh, sl) += (ph, pl), renormalised.
__device__ __forceinline__ void ds_add(float& sh, float& sl, float ph, float pl) {
  float t, e;
  ds_two_sum(sh, ph, t, e);
  e += sl + pl;
  sh = t + e;
  sl = e - (sh - t);
}
__device__ __forceinline__ void ds_split(double x, float& h, float& l) {
  h = (float)x;
  l = (float)(x - (double)h);
}

// ---- programmatic dependent launch (per-level schedule): the next level's grid may start as
// soon as every CTA of this one has begun; it waits for this grid's completion (and memory
// flush) only where it first reads data produced by earlier launches.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---- dataflow synchronisation
constexpr long long SPIN_LIMIT = 1LL << 20;     // default: ~0.1-1 s of polling before giving up

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <bool DF>
__device__ __forceinline__ double trace_load(const double* p) {
  if constexpr (DF) return __ldcg(p);      // written during this launch: bypass the incoherent L1
  else return __ldg(p);
}

// Wait until every kept upwind neighbour of (e, d) has published its angular flux.  A wait that
// exceeds its poll limit (sa.spin_limit, or SPIN_LIMIT when that is <= 0) sets *err and gives up
// (the result is then wrong and the host reports SN_ETIMEOUT); it never traps.
template <int NFC>
__device__ void wait_upwind_n(const DevProblem& Pb, const SweepArgs& sa, uint32_t code, int64_t e, int d,
                              bool valid) {
  if (!valid) return;
  const long long limit = sa.spin_limit > 0 ? sa.spin_limit : SPIN_LIMIT;
#pragma unroll
  for (int f = 0; f < NFC; ++f) {
    if (face_mode(code, f) == MODE_NONE || face_lagged(code, f)) continue;
    const int64_t nb = Pb.nbr[e * NFC + f];
    if (nb < 0) continue;
    const int* flag = sa.done + (int64_t)d * Pb.E + nb;
    long long spins = 0;
    while (ld_acquire(flag) == 0) {
      if (++spins > limit) {
        atomicExch(sa.err, 1);
        break;
      }
      if ((spins & 255) == 0 && *(volatile int*)sa.err) break;   // another wait gave up: stop
      __nanosleep(64);
    }
  }
}

template <int DIM>
__device__ __forceinline__ void wait_upwind(const DevProblem& Pb, const SweepArgs& sa, uint32_t code, int64_t e,
                                            int d, bool valid) {
  wait_upwind_n<2 * DIM>(Pb, sa, code, e, d, valid);
}

// Publish (e, d): every lane's flux store is made visible device-wide before the flag.
template <bool DF, int W>
__device__ __forceinline__ void publish(const DevProblem& Pb, const SweepArgs& sa, int64_t e, int d, bool valid,
                                        int i) {
  if constexpr (DF) {
    __threadfence();
    __syncwarp();
    if (valid && i == 0) st_release(sa.done + (int64_t)d * Pb.E + e, 1);
  }
}

// b += B_f trace_f for one inflow face row (FP64): neighbour trace or incident flux.
template <int DIM, int P_, bool DF>
__device__ __forceinline__ void face_rhs(const DevProblem& Pb, const SweepArgs& sa, uint32_t code, int f, int64_t e,
                                         int d, const double* Brow, double& b) {
  constexpr int NF = Shape<DIM, P_>::NF, NP1 = P_ + 1, N = Shape<DIM, P_>::N;
  const int64_t nb = Pb.nbr[e * 2 * DIM + f];
  if (nb >= 0) {
    const bool lag = face_lagged(code, f);
    const double* ps = lag ? sa.psi_old : sa.psi_new;
    const int fn = Pb.nbr_face[e * 2 * DIM + f], oc = Pb.orient[e * 2 * DIM + f];
    const double* pnb = ps + ((int64_t)d * Pb.E + nb) * N;
#pragma unroll
    for (int fj = 0; fj < NF; ++fj) {
      int t0, t1;
      orient_map_idx(DIM, oc, P_, fj % NP1, fj / NP1, t0, t1);
      const double* pt = pnb + face_vol_index(DIM, P_, fn, t0, t1);
      b = fma(Brow[fj], lag ? __ldg(pt) : trace_load<DF>(pt), b);
    }
  } else if (Pb.psi_inc != nullptr) {
    const double* pin = Pb.psi_inc + ((int64_t)d * Pb.n_bdr + Pb.bdr_index[e * 2 * DIM + f]) * NF;
#pragma unroll
    for (int fj = 0; fj < NF; ++fj) b = fma(Brow[fj], __ldg(pin + fj), b);
  }
}

// FP64 inflow block row fi of face f: -Omega . FN_f (whole-inflow) or the stored block.
template <int DIM, int P_>
__device__ __forceinline__ void brow64(const double* blk, const SweepArgs& sa, uint32_t mode, int f, int fi,
                                       int slot, double om0, double om1, double om2, double* Brow) {
  constexpr int NF = Shape<DIM, P_>::NF, N = Shape<DIM, P_>::N;
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

// ---- latency-oriented FP32 solve: Gauss-Jordan inverse with partial pivoting.
// Pivot search: one integer max per segment over key = (bits(|a|) with the 5 low mantissa bits
// cleared) | (31 - lane): the largest |a| (to 2^-18 relative) wins, ties go to the lowest lane.
template <int W>
__device__ __forceinline__ int seg_argmax_key(unsigned key, int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  if constexpr (W == 32) {
    return 31 - (int)(__reduce_max_sync(FULL, key) & 31u);
  } else if constexpr (W == 16) {
    const unsigned m0 = __reduce_max_sync(FULL, lane < 16 ? key : 0u);
    const unsigned m1 = __reduce_max_sync(FULL, lane < 16 ? 0u : key);
    return 31 - (int)((lane < 16 ? m0 : m1) & 31u);
  } else {
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) key = max(key, __shfl_xor_sync(FULL, key, off, W));
    return 31 - (int)(key & 31u);
  }
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Row-per-lane Gauss-Jordan on the segment, [A | V] with V = I at the start.  All rows are
// updated at every step, so there are N dependent steps and no triangular solves.  Pivot rows
// are not scaled during the elimination (row i -= (a_ik / a_pk) row p for i != p, one
// multiply-add per entry); V is scaled by 1/a_pk once at the end.  V's columns are kept in
// pivot-step order: column m holds the identity column of the row chosen at step m.  Before
// step k the pivot row's V part is nonzero only in columns 0..k-1 plus its own identity entry,
// which enters column k at that step, so step k updates V's columns 0..k only (k + 1 shuffles
// instead of N).  On return the lane chosen at step k (plk[k], myk == k) holds row k of A^{-1}
// in step order: x_k = sum_m v[m] b_{plk[m]}.
template <int N, int W>
__device__ __forceinline__ void gj32(float (&a)[N], float (&v)[N], int lane, bool row, int (&plk)[N], int& myk) {
  constexpr unsigned FULL = 0xffffffffu;
  bool used = !row;
  float myinv = 0.0f;
  myk = -1;
  static_for<0, N>([&](auto jconst) { v[decltype(jconst)::value] = 0.0f; });
  static_for<0, N>([&](auto kconst) {
    constexpr int k = decltype(kconst)::value;
    const unsigned key = used ? 0u : ((__float_as_uint(a[k]) & 0x7fffffe0u) | (unsigned)(31 - lane));
    const float own_inv = rcp_approx(a[k]);      // every lane, while the pivot search runs
    const int pl = seg_argmax_key<W>(key, lane);
    plk[k] = pl;
    const float inv = __shfl_sync(FULL, own_inv, pl, W);
    const bool me = (lane == pl);
    if (me) {
      used = true;
      myk = k;
      myinv = inv;
      v[k] = 1.0f;                               // the pivot row's identity entry, in column k
    }
    const float l = me ? 0.0f : a[k] * inv;
    static_for<k + 1, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      a[j] = fmaf(-l, __shfl_sync(FULL, a[j], pl, W), a[j]);
    });
    static_for<0, k + 1>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      v[j] = fmaf(-l, __shfl_sync(FULL, v[j], pl, W), v[j]);
    });
  });
  static_for<0, N>([&](auto jconst) { v[decltype(jconst)::value] *= myinv; });
}

// y_k = sum_m v[m] r_{plk[m]} on the pivot lane of step k; r_j lives on lane j of the segment.
template <int N, int W>
__device__ __forceinline__ float gj_apply(const float (&v)[N], float r, const int (&plk)[N]) {
  constexpr unsigned FULL = 0xffffffffu;
  float s0 = 0.0f, s1 = 0.0f;
  static_for<0, N>([&](auto jconst) {
    constexpr int j = decltype(jconst)::value;
    const float rj = __shfl_sync(FULL, r, plk[j], W);
    if (j & 1) s1 = fmaf(v[j], rj, s1);
    else s0 = fmaf(v[j], rj, s0);
  });
  return s0 + s1;
}

// ------------------------------------------------------------------ FP64 form
template <int DIM, int P_, bool DF>
__device__ __forceinline__ void body64(const DevProblem& Pb, const SweepArgs& sa, int32_t pr, bool valid, int lane) {
  using S = Shape<DIM, P_>;
  constexpr int N = S::N, NF = S::NF, W = S::W;
  constexpr unsigned FULL = 0xffffffffu;
  const int i = lane % W;
  const int M = Pb.M;
  const int64_t E = Pb.E;
  const int64_t e = pr / M;
  const int d = pr % M;
  const bool row = valid && (i < N);
  const double om0 = Pb.omega[d * 3 + 0], om1 = Pb.omega[d * 3 + 1], om2 = Pb.omega[d * 3 + 2];
  const double* blk = Pb.elem + e * Pb.blk;
  double a[N];
  double b = 0.0;
  if (row) {
    const double st = Pb.sig_t[e];
    static_for<0, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      double v = om0 * __ldg(blk + j * N + i);
      v = fma(om1, __ldg(blk + N * N + j * N + i), v);
      if (DIM == 3) v = fma(om2, __ldg(blk + 2 * N * N + j * N + i), v);
      a[j] = fma(st, __ldg(blk + DIM * N * N + j * N + i), v);
    });
    if (Pb.q_dir != nullptr) {
      const double* qd = Pb.q_dir + ((int64_t)d * E + e) * N;
#pragma unroll
      for (int j = 0; j < N; ++j) b = fma(__ldg(blk + DIM * N * N + i * N + j), qd[j], b);
    }
  } else {
    static_for<0, N>([&](auto jconst) { a[decltype(jconst)::value] = 0.0; });
  }
  const uint32_t code = valid ? sa.facecode[(int64_t)d * E + e] : 0u;
  const int mbase = (valid && (code & 0xAAAu)) ? sa.mixed_off[(int64_t)d * E + e] : 0;
  if constexpr (DF) wait_upwind<DIM>(Pb, sa, code, e, d, valid);
  else {
    pdl_wait();                          // sources and upwind traces come from earlier launches
    pdl_launch_dependents();             // ... and only then may the next level start: one level ahead
  }
  if (row) b += sa.src[e * N + i];
  int mrank = 0;
  static_for<0, 2 * DIM>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    const uint32_t mode = face_mode(code, f);
    const int fi = row ? on_face<DIM, P_>(f, i) : -1;
    if (mode != MODE_NONE && fi >= 0) {
      double Brow[NF];
      brow64<DIM, P_>(blk, sa, mode, f, fi, mbase + mrank, om0, om1, om2, Brow);
      static_for<0, NF>([&](auto jconst) {
        constexpr int fj = decltype(jconst)::value;
        a[fvi<DIM, P_>(f, fj)] += Brow[fj];
      });
      face_rhs<DIM, P_, DF>(Pb, sa, code, f, e, d, Brow, b);
    }
    if (mode == MODE_MIXED) ++mrank;
  });
  // LU with partial pivoting; argmax |a[k]| on the bit pattern (integer pipe)
  bool used = !row;
  int myk = -1;
  double myinv = 0.0;
  int plk[N];
  static_for<0, N>([&](auto kconst) {
    constexpr int k = decltype(kconst)::value;
    // key: high word of |a[k]| (sign cleared, 5 low bits replaced by the lane): integer max
    const unsigned hw = (unsigned)((unsigned long long)__double_as_longlong(a[k]) >> 32);
    const unsigned key = used ? 0u : ((hw & 0x7fffffe0u) | (unsigned)(31 - lane));
    const int pl = seg_argmax_key<W>(key, lane);
    plk[k] = pl;
    const double piv = __shfl_sync(FULL, a[k], pl, W);
    const double inv = nr_rcp(piv);
    if (lane == pl && !used) {
      used = true;
      myk = k;
      myinv = inv;
    }
    const bool elim = !used;
    const double l = a[k] * inv;
    static_for<k + 1, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      const double u = __shfl_sync(FULL, a[j], pl, W);
      if (elim) a[j] = fma(-l, u, a[j]);
    });
    const double ub = __shfl_sync(FULL, b, pl, W);
    if (elim) b = fma(-l, ub, b);
  });
  double x = 0.0;
  static_for<0, N>([&](auto jconst) {
    constexpr int j = N - 1 - decltype(jconst)::value;
    const bool mine = (myk == j);
    const double xl = mine ? b * myinv : 0.0;
    const double xj = __shfl_sync(FULL, xl, plk[j], W);
    if (mine) x = xj;
    if (myk >= 0 && myk < j) b = fma(-a[j], xj, b);
  });
  if (row && myk >= 0) {
    const int64_t o = ((int64_t)d * E + e) * N + myk;
    sa.psi_new[o] = x;
    if (sa.psi_new_h != nullptr) {       // keep the double-single split of the iterate current
      const float h = (float)x;
      sa.psi_new_h[o] = h;
      sa.psi_new_l[o] = (float)(x - (double)h);
    }
  }
  publish<DF, W>(Pb, sa, e, d, valid, i);
}

// ------------------------------------------------------------------ mixed form, FP64 residual
//   A32 = fl32 assembly of A from the FP32 factor copy; b in FP64;
//   xhat = A32^{-1} fl32(b); r = b - A64 xhat (FP64 row); psi = xhat + A32^{-1} fl32(r).
template <int DIM, int P_, bool DF>
__device__ __forceinline__ void bodymx(const DevProblem& Pb, const SweepArgs& sa, int32_t pr, bool valid, int lane) {
  using S = Shape<DIM, P_>;
  constexpr int N = S::N, NF = S::NF, W = S::W;
  constexpr unsigned FULL = 0xffffffffu;
  const int i = lane % W;
  const int M = Pb.M;
  const int64_t E = Pb.E;
  const int64_t e = pr / M;
  const int d = pr % M;
  const bool row = valid && (i < N);
  const double om0 = Pb.omega[d * 3 + 0], om1 = Pb.omega[d * 3 + 1], om2 = Pb.omega[d * 3 + 2];
  const float fo0 = (float)om0, fo1 = (float)om1, fo2 = (float)om2;
  const double* blk = Pb.elem + e * Pb.blk;
  const float* blk32 = Pb.elem32 + e * Pb.blk;
  float a[N];
  double a64[N];
  double b = 0.0;
  if (row) {
    const double st = Pb.sig_t[e];
    const float st32 = (float)st;
    static_for<0, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      float v = fo0 * __ldg(blk32 + j * N + i);
      v = fmaf(fo1, __ldg(blk32 + N * N + j * N + i), v);
      if (DIM == 3) v = fmaf(fo2, __ldg(blk32 + 2 * N * N + j * N + i), v);
      a[j] = fmaf(st32, __ldg(blk32 + DIM * N * N + j * N + i), v);
      double w = om0 * __ldg(blk + j * N + i);
      w = fma(om1, __ldg(blk + N * N + j * N + i), w);
      if (DIM == 3) w = fma(om2, __ldg(blk + 2 * N * N + j * N + i), w);
      a64[j] = fma(st, __ldg(blk + DIM * N * N + j * N + i), w);
    });
    if (Pb.q_dir != nullptr) {
      const double* qd = Pb.q_dir + ((int64_t)d * E + e) * N;
#pragma unroll
      for (int j = 0; j < N; ++j) b = fma(__ldg(blk + DIM * N * N + i * N + j), qd[j], b);
    }
  } else {
    static_for<0, N>([&](auto jconst) {
      a[decltype(jconst)::value] = 0.0f;
      a64[decltype(jconst)::value] = 0.0;
    });
  }
  const uint32_t code = valid ? sa.facecode[(int64_t)d * E + e] : 0u;
  const int mbase = (valid && (code & 0xAAAu)) ? sa.mixed_off[(int64_t)d * E + e] : 0;
  if constexpr (DF) wait_upwind<DIM>(Pb, sa, code, e, d, valid);
  else {
    pdl_wait();                          // sources and upwind traces come from earlier launches
    pdl_launch_dependents();             // ... and only then may the next level start: one level ahead
  }
  if (row) b += sa.src[e * N + i];
  int mrank = 0;
  static_for<0, 2 * DIM>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    const uint32_t mode = face_mode(code, f);
    const int fi = row ? on_face<DIM, P_>(f, i) : -1;
    if (mode != MODE_NONE && fi >= 0) {
      double Brow[NF];
      brow64<DIM, P_>(blk, sa, mode, f, fi, mbase + mrank, om0, om1, om2, Brow);
      static_for<0, NF>([&](auto jconst) {
        constexpr int fj = decltype(jconst)::value;
        a64[fvi<DIM, P_>(f, fj)] += Brow[fj];
        a[fvi<DIM, P_>(f, fj)] += (float)Brow[fj];
      });
      face_rhs<DIM, P_, DF>(Pb, sa, code, f, e, d, Brow, b);
    }
    if (mode == MODE_MIXED) ++mrank;
  });
  int plk[N], myk;
  float v[N];
  gj32<N, W>(a, v, lane, row, plk, myk);
  const float xhat = gj_apply<N, W>(v, (float)b, plk);     // on the pivot lane of step myk
  const double xh64 = (double)xhat;
  double r = b;
  static_for<0, N>([&](auto jconst) {
    constexpr int j = decltype(jconst)::value;
    const double xj = __shfl_sync(FULL, xh64, plk[j], W);
    r = fma(-a64[j], xj, r);
  });
  const float dx = gj_apply<N, W>(v, (float)r, plk);
  if (row && myk >= 0) {
    const int64_t o = ((int64_t)d * E + e) * N + myk;
    const double x = xh64 + (double)dx;
    sa.psi_new[o] = x;
    if (sa.psi_new_h != nullptr) {       // keep the double-single split of the iterate current
      const float h = (float)x;
      sa.psi_new_h[o] = h;
      sa.psi_new_l[o] = (float)(x - (double)h);
    }
  }
  publish<DF, W>(Pb, sa, e, d, valid, i);
}

// ------------------------------------------------------------------ mixed form, double-single residual
// The row of A is assembled once in double-single from the (hi, lo) FP32 split of the element
// factors; its hi part is the FP32 matrix that is inverted; r = b - A xhat is accumulated in
// double-single.  The volume part of A (and in 2D its inflow face blocks) depends only on the
// element, the direction and the face modes, not on upwind fluxes: it is assembled before the
// wait for upwind data, overlapping the previous level; the right-hand side, the inverse and
// its two applications follow the wait.

// Inflow block row fi of face f in double-single: -(Omega . FN_f) for a whole-inflow face, the
// stored block for a partially-inflow one (slot o_mixed).  NC: read-only cache loads.
template <int DIM, int P_, bool NC>
__device__ __forceinline__ void ds_block_row(const float* bh, const float* bl, const SweepArgs& sa, uint32_t mode,
                                             int f, int fi, int64_t o_mixed, const float (&oh)[3],
                                             const float (&ol)[3], float (&Bh)[Shape<DIM, P_>::NF],
                                             float (&Bl)[Shape<DIM, P_>::NF]) {
  using S = Shape<DIM, P_>;
  constexpr int N = S::N, NF = S::NF;
  auto ld = [](const float* p) { return NC ? __ldg(p) : *p; };
  if (mode == MODE_PURE) {
    const int o = (DIM + 1) * N * N + f * DIM * NF * NF + fi * NF;
#pragma unroll
    for (int fj = 0; fj < NF; ++fj) {
      float h, l, ph, pl;
      ds_mul(oh[0], ol[0], ld(bh + o + fj), ld(bl + o + fj), h, l);
      ds_mul(oh[1], ol[1], ld(bh + o + NF * NF + fj), ld(bl + o + NF * NF + fj), ph, pl);
      ds_add(h, l, ph, pl);
      if (DIM == 3) {
        ds_mul(oh[2], ol[2], ld(bh + o + 2 * NF * NF + fj), ld(bl + o + 2 * NF * NF + fj), ph, pl);
        ds_add(h, l, ph, pl);
      }
      Bh[fj] = -h;
      Bl[fj] = -l;
    }
  } else {
    const int64_t o = o_mixed * NF * NF + fi * NF;
#pragma unroll
    for (int fj = 0; fj < NF; ++fj) {
      Bh[fj] = ld(sa.mixedBh + o + fj);
      Bl[fj] = ld(sa.mixedBl + o + fj);
    }
  }
}

template <int DIM, int P_, bool DF>
__device__ __forceinline__ void bodyds(const DevProblem& Pb, const SweepArgs& sa, int32_t pr, bool valid, int lane) {
  using S = Shape<DIM, P_>;
  constexpr int N = S::N, NF = S::NF, W = S::W, NP1 = S::NP1;
  constexpr unsigned FULL = 0xffffffffu;
  const int i = lane % W;
  const int M = Pb.M;
  const int64_t E = Pb.E;
  const int64_t e = pr / M;
  const int d = pr % M;
  const bool row = valid && (i < N);
  float oh[3], ol[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    oh[k] = Pb.om32[d * 6 + 2 * k];
    ol[k] = Pb.om32[d * 6 + 2 * k + 1];
  }
  const float* bh = Pb.elem32 + e * Pb.blk;
  const float* bl = Pb.elem32lo + e * Pb.blk;
  float ah[N], al[N];
  float a[N];
  float rbh = 0.0f, rbl = 0.0f;                 // right-hand side in double-single
  if (row) {
    const float sh = Pb.st32[2 * e], sl = Pb.st32[2 * e + 1];
    static_for<0, N>([&](auto jconst) {
      constexpr int j = decltype(jconst)::value;
      float h, l, ph, pl;
      ds_mul(oh[0], ol[0], __ldg(bh + j * N + i), __ldg(bl + j * N + i), h, l);
      ds_mul(oh[1], ol[1], __ldg(bh + N * N + j * N + i), __ldg(bl + N * N + j * N + i), ph, pl);
      ds_add(h, l, ph, pl);
      if (DIM == 3) {
        ds_mul(oh[2], ol[2], __ldg(bh + 2 * N * N + j * N + i), __ldg(bl + 2 * N * N + j * N + i), ph, pl);
        ds_add(h, l, ph, pl);
      }
      ds_mul(sh, sl, __ldg(bh + DIM * N * N + j * N + i), __ldg(bl + DIM * N * N + j * N + i), ph, pl);
      ds_add(h, l, ph, pl);
      ah[j] = h;
      al[j] = l;
    });
    if (Pb.q_dir != nullptr) {           // direction-dependent source (tests): FP64, then split
      const double* blk = Pb.elem + e * Pb.blk;
      const double* qd = Pb.q_dir + ((int64_t)d * E + e) * N;
      double qb = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) qb = fma(__ldg(blk + DIM * N * N + i * N + j), qd[j], qb);
      ds_split(qb, rbh, rbl);
    }
  } else {
    static_for<0, N>([&](auto jconst) {
      ah[decltype(jconst)::value] = 0.0f;
      al[decltype(jconst)::value] = 0.0f;
    });
  }
  const uint32_t code = valid ? sa.facecode[(int64_t)d * E + e] : 0u;
  const int mbase = (valid && (code & 0xAAAu)) ? sa.mixed_off[(int64_t)d * E + e] : 0;
  // inflow face blocks into the matrix; in 2D the block rows are also kept in shared memory
  // ([face][entry][hi, lo][lane] per warp of a 128-thread block) for the right-hand side after
  // the wait
  float* bsave = nullptr;
  if constexpr (S::FACES_PRE) {
    __shared__ float bsave_all[4][2 * DIM][NF][2][32];
    bsave = &bsave_all[(threadIdx.x >> 5) & 3][0][0][0][0];
    int mrank = 0;
    static_for<0, 2 * DIM>([&](auto fconst) {
      constexpr int f = decltype(fconst)::value;
      const uint32_t mode = face_mode(code, f);
      const int fi = row ? on_face<DIM, P_>(f, i) : -1;
      if (mode != MODE_NONE && fi >= 0) {
        float Bh[NF], Bl[NF];
        ds_block_row<DIM, P_, true>(bh, bl, sa, mode, f, fi, mbase + mrank, oh, ol, Bh, Bl);
        static_for<0, NF>([&](auto jconst) {
          constexpr int fj = decltype(jconst)::value;
          constexpr int c = fvi<DIM, P_>(f, fj);
          ds_add(ah[c], al[c], Bh[fj], Bl[fj]);
          bsave[((f * NF + fj) * 2 + 0) * 32 + lane] = Bh[fj];
          bsave[((f * NF + fj) * 2 + 1) * 32 + lane] = Bl[fj];
        });
      }
      if (mode == MODE_MIXED) ++mrank;
    });
  }
  // mesh connectivity of the faces (static data)
  int64_t nbv[2 * DIM];
  int fov[2 * DIM];
  static_for<0, 2 * DIM>([&](auto fconst) {
    constexpr int f = decltype(fconst)::value;
    nbv[f] = valid ? Pb.nbr[e * 2 * DIM + f] : -1;
    fov[f] = valid ? (Pb.nbr_face[e * 2 * DIM + f] | (Pb.orient[e * 2 * DIM + f] << 8)) : 0;
  });
  // Dataflow schedule with the whole matrix formed before the wait (2D): the inverse depends only
  // on the element and the direction, so it is computed while the upwind pairs are still running
  // and only the right-hand side, the two inverse applications and the residual follow the wait.
  // (On per-level launches only one level runs ahead, and a longer pre-wait half bounds the level.)
  constexpr bool GJ_PRE = DF && S::FACES_PRE;
  int plk[N], myk;
  float v[N];
  if constexpr (GJ_PRE) {
    static_for<0, N>([&](auto jconst) { a[decltype(jconst)::value] = ah[decltype(jconst)::value]; });
    gj32<N, W>(a, v, lane, row, plk, myk);
  }
  if constexpr (DF) {
    wait_upwind<DIM>(Pb, sa, code, e, d, valid);
  } else {
    pdl_wait();                          // sources and upwind traces come from earlier launches
    pdl_launch_dependents();             // ... and only then may the next level start: one level ahead
  }
  if (row) ds_add(rbh, rbl, sa.src_h[e * N + i], sa.src_l[e * N + i]);
  {
    int mrank = 0;
    static_for<0, 2 * DIM>([&](auto fconst) {
      constexpr int f = decltype(fconst)::value;
      const uint32_t mode = face_mode(code, f);
      const int fi = row ? on_face<DIM, P_>(f, i) : -1;
      const int64_t nb = nbv[f];
      const bool has_trace = nb >= 0 || Pb.psi_inc != nullptr;
      if (mode != MODE_NONE && fi >= 0 && (!S::FACES_PRE || has_trace)) {
        float Bh[NF], Bl[NF];
        if constexpr (!S::FACES_PRE) {
          ds_block_row<DIM, P_, true>(bh, bl, sa, mode, f, fi, mbase + mrank, oh, ol, Bh, Bl);
          static_for<0, NF>([&](auto jconst) {
            constexpr int fj = decltype(jconst)::value;
            constexpr int c = fvi<DIM, P_>(f, fj);
            ds_add(ah[c], al[c], Bh[fj], Bl[fj]);
          });
        }
        if (nb >= 0) {                   // upwind neighbour's (hi, lo) split of the trace
          const bool lag = face_lagged(code, f);
          int c0, ci, cj;
          trace_affine<DIM, P_>(fov[f] & 0xff, fov[f] >> 8, c0, ci, cj);
          const int64_t base = ((int64_t)d * E + nb) * N + c0;
          const float* ph_ = (lag ? sa.psi_old_h : sa.psi_new_h) + base;
          const float* pl_ = (lag ? sa.psi_old_l : sa.psi_new_l) + base;
          float th[NF], tl[NF];
#pragma unroll
          for (int fj = 0; fj < NF; ++fj) {
            const int o = ci * (fj % NP1) + cj * (fj / NP1);
            if (!lag && DF) {
              th[fj] = __ldcg(ph_ + o);
              tl[fj] = __ldcg(pl_ + o);
            } else {
              th[fj] = __ldg(ph_ + o);
              tl[fj] = __ldg(pl_ + o);
            }
          }
          if constexpr (S::FACES_PRE) {
#pragma unroll
            for (int fj = 0; fj < NF; ++fj) {
              Bh[fj] = bsave[((f * NF + fj) * 2 + 0) * 32 + lane];
              Bl[fj] = bsave[((f * NF + fj) * 2 + 1) * 32 + lane];
            }
          }
          float sh2 = 0.0f, sl2 = 0.0f;  // second accumulator: two independent chains
#pragma unroll
          for (int fj = 0; fj < NF; ++fj) {
            float qh, ql;
            ds_mul(Bh[fj], Bl[fj], th[fj], tl[fj], qh, ql);
            if (fj & 1) ds_add(sh2, sl2, qh, ql);
            else ds_add(rbh, rbl, qh, ql);
          }
          ds_add(rbh, rbl, sh2, sl2);
        } else if (Pb.psi_inc != nullptr) {  // incident flux on the domain boundary
          if constexpr (S::FACES_PRE) {
#pragma unroll
            for (int fj = 0; fj < NF; ++fj) {
              Bh[fj] = bsave[((f * NF + fj) * 2 + 0) * 32 + lane];
              Bl[fj] = bsave[((f * NF + fj) * 2 + 1) * 32 + lane];
            }
          }
          const double* pin = Pb.psi_inc + ((int64_t)d * Pb.n_bdr + Pb.bdr_index[e * 2 * DIM + f]) * NF;
#pragma unroll
          for (int fj = 0; fj < NF; ++fj) {
            float th, tl, qh, ql;
            ds_split(__ldg(pin + fj), th, tl);
            ds_mul(Bh[fj], Bl[fj], th, tl, qh, ql);
            ds_add(rbh, rbl, qh, ql);
          }
        }
      }
      if (mode == MODE_MIXED) ++mrank;
    });
  }
  if constexpr (!GJ_PRE) {
    static_for<0, N>([&](auto jconst) { a[decltype(jconst)::value] = ah[decltype(jconst)::value]; });
    gj32<N, W>(a, v, lane, row, plk, myk);
  }
  const float xhat = gj_apply<N, W>(v, rbh, plk);        // on the pivot lane of step myk
  // r = b - A xhat in double-single, four independent accumulation chains
  float rh[4] = {rbh, 0.0f, 0.0f, 0.0f}, rl[4] = {rbl, 0.0f, 0.0f, 0.0f};
  static_for<0, N>([&](auto jconst) {
    constexpr int j = decltype(jconst)::value;
    const float xj = __shfl_sync(FULL, xhat, plk[j], W);
    float ph = ah[j] * xj;
    float pl = fmaf(ah[j], xj, -ph);
    pl = fmaf(al[j], xj, pl);
    ds_add(rh[j & 3], rl[j & 3], -ph, -pl);
  });
  ds_add(rh[0], rl[0], rh[1], rl[1]);
  ds_add(rh[2], rl[2], rh[3], rl[3]);
  ds_add(rh[0], rl[0], rh[2], rl[2]);
  const float dx = gj_apply<N, W>(v, rh[0] + rl[0], plk);
  if (row && myk >= 0) {
    float oh2, ol2;
    ds_two_sum(xhat, dx, oh2, ol2);
    const int64_t o = ((int64_t)d * E + e) * N + myk;
    sa.psi_new_h[o] = oh2;
    sa.psi_new_l[o] = ol2;
    sa.psi_new[o] = (double)oh2 + (double)ol2;
  }
  publish<DF, W>(Pb, sa, e, d, valid, i);
}

}  // namespace sn

#include "inverse_body.cuh"

namespace sn {

template <int DIM, int P_, int PREC, bool DF>
__device__ __forceinline__ void solve_item(const DevProblem& Pb, const SweepArgs& sa, int32_t pr, bool valid,
                                           int lane) {
  if constexpr (PREC == SN_PREC_FP64) body64<DIM, P_, DF>(Pb, sa, pr, valid, lane);
  else if constexpr (PREC == SN_PREC_FP64_INV) bodyinv<TensorEl<DIM, P_>, DF>(Pb, sa, pr, valid, lane);
  else if constexpr (PREC == SN_PREC_DS_INV) bodydsinv<TensorEl<DIM, P_>, DF>(Pb, sa, pr, valid, lane);
  else if constexpr (PREC == SN_PREC_MIXED) bodymx<DIM, P_, DF>(Pb, sa, pr, valid, lane);
  else bodyds<DIM, P_, DF>(Pb, sa, pr, valid, lane);
}


}  // namespace sn
