// Diffusion synthetic acceleration (DSA) of source iteration on the device.  The paper names DSA
// as the follow-up for scattering-dominated problems (Sec. 4 opening, conclusions) without printing
// its equations; this is the project's reading: after the sweep and its moment phi_half, the
// correction dphi solves, on the transport's own DG space,
//
//   a(dphi, v) = int sigma_s (phi_half - phi_prev) v,
//   a(u, v) = sum_K int_K (D grad u . grad v + sigma_a u v)
//           + sum_{interior F} int_F (kappa [[u]][[v]] - {{D grad u . n}}[[v]] - [[u]]{{D grad v . n}})
//           + sum_{boundary F} int_F (kappa u v - 1/2 (D grad u . n) v - 1/2 u (D grad v . n)),
//
// D = 1/(3 sigma_t), sigma_a = sigma_t - sigma_s, [[u]] = u_owner - u_other (owner = the lower element
// id), n the owner's outward normal, kappa = max(kappa_IP, 1/4) with kappa_IP = (c/2)(D_o/h_o + D_t/h_t)
// inside and c D/h on the boundary, c = 2 p (p + 1), h = |K| / |F|; and phi <- phi_half + dphi.
//
// Matrix: per element a diagonal block (volume + its faces' self terms) and per (element, face) the
// block coupling it to the neighbour, all N x N and stored column-major ([j][i]: lane i of a warp
// reads consecutive addresses).  Solver: conjugate gradients preconditioned by the inverses of the
// diagonal blocks, to a relative residual tolerance; the scalars stay on the device (three-slot
// ring: no host synchronisation inside an iteration) and the host checks convergence every 8
// iterations.
#include "devmath.cuh"

namespace sn {

namespace {

// DG basis values and reference gradients at reference point xi (tensor GLL Lagrange).
__device__ inline void basis_at(int dim, int p, const double* gll, const double* xi, double* val, double* gref) {
  const int n = p + 1;
  const int N = dim == 2 ? n * n : n * n * n;
  for (int m = 0; m < N; ++m) {
    const int id[3] = {m % n, (m / n) % n, dim == 3 ? m / (n * n) : 0};
    double v = 1.0;
    for (int k = 0; k < dim; ++k) v = v * dlagrange(gll, n, id[k], xi[k]);
    val[m] = v;
    for (int a = 0; a < dim; ++a) {
      double g = 1.0;
      for (int k = 0; k < dim; ++k) g = g * (k == a ? dlagrange_deriv(gll, n, id[k], xi[k]) : dlagrange(gll, n, id[k], xi[k]));
      gref[m * dim + a] = g;
    }
  }
}

// Jacobian of the Q_r map at reference point xi, its cofactor matrix and determinant.
__device__ inline double jac_cof(int dim, int r, const double* geo, const double* ctrl, const double* xi,
                                 double (*C)[3]) {
  const int n1 = r + 1;
  const int Nv = dim == 2 ? n1 * n1 : n1 * n1 * n1;
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int mv = 0; mv < Nv; ++mv) {
    const int id[3] = {mv % n1, (mv / n1) % n1, dim == 3 ? mv / (n1 * n1) : 0};
    for (int j = 0; j < dim; ++j) {
      double g = 1.0;
      for (int k = 0; k < dim; ++k) g = g * (k == j ? dlagrange_deriv(geo, n1, id[k], xi[k]) : dlagrange(geo, n1, id[k], xi[k]));
      for (int i = 0; i < dim; ++i) J[i][j] += ctrl[mv * dim + i] * g;
    }
  }
  if (dim == 2) {
    C[0][0] = J[1][1];
    C[0][1] = -J[1][0];
    C[1][0] = -J[0][1];
    C[1][1] = J[0][0];
    return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
      C[i][j] = J[r0][c0] * J[r1][c1] - J[r0][c1] * J[r1][c0];
    }
  return J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
}

// Volume part of the diagonal blocks: D K + sigma_a M, K_ij = sum_q w_q / |J| (C grad_ref u_i).(C
// grad_ref u_j); also |K| = sum_q w_q |J|.  One block of threads per element.
__global__ void dsa_volume_kernel(DevProblem P, double* __restrict__ diag, double* __restrict__ vol) {
  extern __shared__ double sh[];
  const int64_t e = blockIdx.x;
  const int N = P.N, Q = P.Q, Nv = P.Nv, dim = P.dim;
  double* G = sh;                      // [Q][dim][dim]: w C^T C / |J|
  double* wd = G + Q * 9;              // [Q]: w |J|
  const double* wq = tabp(P, P.off_wq);
  const double* dB = tabp(P, P.off_dB);
  const double* dV = tabp(P, P.off_dV);
  const double* ctrl = P.ctrl + e * Nv * dim;
  for (int q = threadIdx.x; q < Q; q += blockDim.x) {
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int m = 0; m < Nv; ++m)
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) J[i][j] += ctrl[m * dim + i] * dV[((size_t)q * Nv + m) * dim + j];
    double C[3][3];
    double det;
    if (dim == 2) {
      C[0][0] = J[1][1];
      C[0][1] = -J[1][0];
      C[1][0] = -J[0][1];
      C[1][1] = J[0][0];
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    } else {
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          const int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
          C[i][j] = J[r0][c0] * J[r1][c1] - J[r0][c1] * J[r1][c0];
        }
      det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    }
    wd[q] = wq[q] * det;
    // (C^T C)_ab = sum_k C[k][a] C[k][b]: grad u = C grad_ref u / |J|
    for (int a = 0; a < dim; ++a)
      for (int b = 0; b < dim; ++b) {
        double s = 0.0;
        for (int k = 0; k < dim; ++k) s += C[k][a] * C[k][b];
        G[(q * 3 + a) * 3 + b] = wq[q] * s / det;
      }
  }
  __syncthreads();
  const double D = 1.0 / (3.0 * P.sig_t[e]);
  const double sa = P.sig_t[e] - P.sig_s[e];
  const double* M = P.elem + e * P.blk + (int64_t)dim * N * N;
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    const int i = t / N, j = t % N;
    double k = 0.0;
    for (int q = 0; q < Q; ++q)
      for (int a = 0; a < dim; ++a) {
        const double gi = dB[((size_t)q * N + i) * dim + a];
        for (int b = 0; b < dim; ++b) k += G[(q * 3 + a) * 3 + b] * gi * dB[((size_t)q * N + j) * dim + b];
      }
    diag[(e * N + j) * N + i] = D * k + sa * M[i * N + j];          // column-major
  }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < Q; ++q) s += wd[q];
    vol[e] = s;
  }
}

// Face terms of element e through its face f, from e's side: the self block (added to e's
// diagonal later) and the block coupling e's test functions to the neighbour's trial functions.
// One warp per (element, face).  Points: the face rule without kink splitting in the owner's face
// coordinates (2D n_f GL points, 3D the K x K composite of n_f x n_f points).
__global__ void dsa_face_kernel(DevProblem P, const double* __restrict__ vol, double* __restrict__ selfb,
                                double* __restrict__ offb, int shm_per_warp) {
  extern __shared__ double sh[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int nfc = 2 * P.dim;
  if (item >= P.E * nfc) return;
  const int64_t e = item / nfc;
  const int f = (int)(item % nfc);
  const int dim = P.dim, N = P.N, nf = P.nf, r = P.r, p = P.p, Nv = P.Nv;
  const int K = dim == 3 ? P.K : 1;
  const int np = dim == 2 ? nf : K * K * nf * nf;
  const int64_t nb = P.nbr[e * nfc + f];
  const bool bdr = nb < 0;
  const bool e_owner = bdr || e < nb;
  const int64_t own = e_owner ? e : nb, oth = e_owner ? nb : e;
  const int fo = e_owner ? f : P.nbr_face[e * nfc + f];
  const int ft = bdr ? -1 : (e_owner ? P.nbr_face[e * nfc + f] : f);
  const int code = bdr ? 0 : P.orient[own * nfc + fo];
  const double* geo = tabp(P, P.off_geo);
  const double* gll = tabp(P, P.off_gll);
  const double* t = tabp(P, P.off_glf_t);
  const double* wt = tabp(P, P.off_glf_w);
  // per point: [w, w|n|, u_e[N], dn_e[N], u_x[N], dn_x[N]]  (dn = grad u . n~, n~ the owner's scaled normal)
  const int stride = 2 + 4 * N;
  double* pts = sh + (size_t)wib * shm_per_warp;
  for (int q = lane; q < np; q += 32) {
    double s0, s1 = 0.0, w;
    if (dim == 2) {
      s0 = t[q];
      w = wt[q];
    } else {
      const int i = q % nf, j = (q / nf) % nf, u = (q / (nf * nf)) % K, v = q / (nf * nf * K);
      s0 = ((double)u + t[i]) / (double)K;
      s1 = ((double)v + t[j]) / (double)K;
      w = (wt[i] / (double)K) * (wt[j] / (double)K);
    }
    double nt[3];
    face_normal(dim, r, geo, P.ctrl + own * Nv * dim, fo, s0, s1, nt);
    double nn = 0.0;
    for (int k = 0; k < dim; ++k) nn += nt[k] * nt[k];
    double* o = pts + q * stride;
    o[0] = w;
    o[1] = w * sqrt(nn);
    for (int side = 0; side < (bdr ? 1 : 2); ++side) {
      // side 0: element e itself, side 1: the other element of the face
      const bool is_owner = (side == 0) == e_owner;
      const int64_t el = is_owner ? own : oth;
      double xi[3];
      if (is_owner) {
        face_ref(dim, fo, s0, s1, xi);
      } else {
        double t0, t1;
        orient_map(dim, code, s0, s1, t0, t1);
        face_ref(dim, ft, t0, t1, xi);
      }
      double C[3][3];
      const double det = jac_cof(dim, r, geo, P.ctrl + el * Nv * dim, xi, C);
      double val[32], gref[32 * 3];
      basis_at(dim, p, gll, xi, val, gref);
      double* uo = o + 2 + side * 2 * N;
      for (int m = 0; m < N; ++m) {
        double dn = 0.0;
        for (int k = 0; k < dim; ++k) {
          double g = 0.0;
          for (int a = 0; a < dim; ++a) g += C[k][a] * gref[m * dim + a];
          dn += g * nt[k];
        }
        uo[m] = val[m];
        uo[N + m] = dn / det;
      }
    }
  }
  __syncwarp();
  double area = 0.0;
  for (int q = 0; q < np; ++q) area += pts[q * stride + 1];
  const double c_ip = 2.0 * p * (p + 1);
  const double De = 1.0 / (3.0 * P.sig_t[e]);
  double kap;
  double Dx = 0.0, sg_e = e_owner ? 1.0 : -1.0, sg_x = -sg_e;
  if (bdr) {
    kap = fmax(c_ip * De / (vol[e] / area), 0.25);
  } else {
    Dx = 1.0 / (3.0 * P.sig_t[nb]);
    const double Do = e_owner ? De : Dx, Dt = e_owner ? Dx : De;
    const double ho = vol[own] / area, ht = vol[oth] / area;
    kap = fmax(0.5 * c_ip * (Do / ho + Dt / ht), 0.25);
  }
  double* sb = selfb + (e * nfc + f) * N * N;
  double* ob = offb + (e * nfc + f) * N * N;
  for (int t2 = lane; t2 < N * N; t2 += 32) {
    const int i = t2 % N, j = t2 / N;            // test i (element e), trial j; column-major store [j][i]
    double s_self = 0.0, s_off = 0.0;
    for (int q = 0; q < np; ++q) {
      const double* o = pts + q * stride;
      const double w = o[0], wa = o[1];
      const double ve = o[2 + i], dve = o[2 + N + i];
      const double ue = o[2 + j], due = o[2 + N + j];
      if (bdr) {
        s_self += kap * wa * ue * ve - 0.5 * De * w * (due * ve + ue * dve);
      } else {
        const double ux = o[2 + 2 * N + j], dux = o[2 + 3 * N + j];
        s_self += sg_e * sg_e * kap * wa * ue * ve - sg_e * 0.5 * De * w * due * ve - sg_e * 0.5 * De * w * ue * dve;
        s_off += sg_x * sg_e * kap * wa * ux * ve - sg_e * 0.5 * Dx * w * dux * ve - sg_x * 0.5 * De * w * ux * dve;
      }
    }
    sb[j * N + i] = s_self;
    ob[j * N + i] = s_off;
  }
}

// Diagonal block = volume part + self face blocks (face order), and its inverse (Gauss-Jordan with
// partial pivoting), both column-major.  One thread per element.
__global__ void dsa_diag_kernel(int64_t E, int N, int nfc, const double* __restrict__ selfb, double* __restrict__ diag,
                                double* __restrict__ inv, int* bad) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  double A[27 * 27], V[27 * 27];
  for (int t = 0; t < N * N; ++t) {
    double s = diag[e * N * N + t];
    for (int f = 0; f < nfc; ++f) s += selfb[(e * nfc + f) * N * N + t];
    diag[e * N * N + t] = s;
    A[t] = s;                               // A[j*N + i] = entry (i, j)
    V[t] = 0.0;
  }
  for (int i = 0; i < N; ++i) V[i * N + i] = 1.0;
  for (int k = 0; k < N; ++k) {
    int pv = k;
    double best = fabs(A[k * N + k]);
    for (int i = k + 1; i < N; ++i)
      if (fabs(A[k * N + i]) > best) {
        best = fabs(A[k * N + i]);
        pv = i;
      }
    if (!(best > 0.0)) {
      atomicOr(bad, 1);
      return;
    }
    if (pv != k)
      for (int j = 0; j < N; ++j) {
        double a = A[j * N + k];
        A[j * N + k] = A[j * N + pv];
        A[j * N + pv] = a;
        a = V[j * N + k];
        V[j * N + k] = V[j * N + pv];
        V[j * N + pv] = a;
      }
    const double ip = 1.0 / A[k * N + k];
    for (int j = 0; j < N; ++j) {
      A[j * N + k] *= ip;
      V[j * N + k] *= ip;
    }
    for (int i = 0; i < N; ++i) {
      if (i == k) continue;
      const double l = A[k * N + i];
      if (l == 0.0) continue;
      for (int j = 0; j < N; ++j) {
        A[j * N + i] -= l * A[j * N + k];
        V[j * N + i] -= l * V[j * N + k];
      }
    }
  }
  for (int t = 0; t < N * N; ++t) inv[e * N * N + t] = V[t];
}

// ---------------------------------------------------------------- right-hand side and CG
// b_e = sigma_s,e M_e (phi_half - phi_prev)_e; also x = 0 and bb = b . b.  Thread per (element, node).
__global__ void dsa_rhs_kernel(DevProblem P, const double* __restrict__ half, const double* __restrict__ prev,
                               double* __restrict__ b, double* __restrict__ x, double* sc) {
  const int N = P.N;
  const int64_t n = P.E * N;
  double acc = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / N;
    const int m = (int)(t % N);
    const double* M = P.elem + e * P.blk + (int64_t)P.dim * N * N + (int64_t)m * N;
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += M[k] * (half[e * N + k] - prev[e * N + k]);
    s *= P.sig_s[e];
    b[t] = s;
    x[t] = 0.0;
    acc += s * s;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(sc + 0, acc);
}

// y_e = Minv_e v_e (block, column-major inverse): warp per element, lane = row.
__device__ inline double block_apply(const double* __restrict__ blk, const double* __restrict__ v, int N, int i) {
  double s = 0.0;
  for (int j = 0; j < N; ++j) s += blk[j * N + i] * v[j];
  return s;
}

// r = b; z = Minv r; p = z; rz = r . z into ring slot 2 (the "previous iteration").
__global__ void dsa_cg_init_kernel(DevProblem P, const double* __restrict__ inv, const double* __restrict__ b,
                                   double* __restrict__ r, double* __restrict__ z, double* __restrict__ pv, double* sc) {
  const int N = P.N, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  double acc = 0.0;
  if (e < P.E) {
    const double* be = b + e * N;
    double zi = 0.0;
    if (lane < N) {
      r[e * N + lane] = be[lane];
      zi = block_apply(inv + e * N * N, be, N, lane);
      z[e * N + lane] = zi;
      pv[e * N + lane] = zi;
      acc = be[lane] * zi;
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0 && acc != 0.0) atomicAdd(sc + 1 + 3 * 2 + 1, acc);
}

// Scalar ring: sc[1 + 3 s + 0] = p.q, [1] = r.z (new), [2] = r.r of iteration k with slot s = k % 3.
// q = A p and p.q (warp per element, lane = row)
__global__ void dsa_spmv_kernel(DevProblem P, const double* __restrict__ diag, const double* __restrict__ offb,
                                const double* __restrict__ pv, double* __restrict__ q, double* sc, int slot) {
  const int N = P.N, lane = threadIdx.x & 31, nfc = 2 * P.dim;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  double acc = 0.0;
  if (e < P.E && lane < N) {
    double s = block_apply(diag + e * N * N, pv + e * N, N, lane);
    for (int f = 0; f < nfc; ++f) {
      const int64_t nb = P.nbr[e * nfc + f];
      if (nb >= 0) s += block_apply(offb + (e * nfc + f) * N * N, pv + nb * N, N, lane);
    }
    q[e * N + lane] = s;
    acc = s * pv[e * N + lane];
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0 && acc != 0.0) atomicAdd(sc + 1 + 3 * slot + 0, acc);
}

// alpha = rz_prev / pq; x += alpha p; r -= alpha q; z = Minv r; rz_new, rr
__global__ void dsa_update_kernel(DevProblem P, const double* __restrict__ inv, const double* __restrict__ pv,
                                  const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
                                  double* __restrict__ z, double* sc, int slot, int prev) {
  const int N = P.N, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const double pq = sc[1 + 3 * slot + 0], rz = sc[1 + 3 * prev + 1];
  const double alpha = pq != 0.0 ? rz / pq : 0.0;
  double arz = 0.0, arr = 0.0;
  if (e < P.E) {
    double ri = 0.0;
    if (lane < N) {
      const int64_t o = e * N + lane;
      x[o] += alpha * pv[o];
      ri = r[o] - alpha * q[o];
      r[o] = ri;
    }
    __syncwarp();
    if (lane < N) {
      const double zi = block_apply(inv + e * N * N, r + e * N, N, lane);
      z[e * N + lane] = zi;
      arz = ri * zi;
      arr = ri * ri;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    arz += __shfl_xor_sync(0xffffffffu, arz, off);
    arr += __shfl_xor_sync(0xffffffffu, arr, off);
  }
  if (lane == 0 && (arz != 0.0 || arr != 0.0)) {
    atomicAdd(sc + 1 + 3 * slot + 1, arz);
    atomicAdd(sc + 1 + 3 * slot + 2, arr);
  }
}

// beta = rz_new / rz_prev; p = z + beta p; clear the slot of the next iteration
__global__ void dsa_pupdate_kernel(int64_t n, const double* __restrict__ z, double* __restrict__ pv, double* sc,
                                   int slot, int prev, int next) {
  const double rzn = sc[1 + 3 * slot + 1], rzp = sc[1 + 3 * prev + 1];
  const double beta = rzp != 0.0 ? rzn / rzp : 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    pv[t] = z[t] + beta * pv[t];
  if (blockIdx.x == 0 && threadIdx.x < 3) sc[1 + 3 * next + threadIdx.x] = 0.0;
}

// phi_new = phi_half + x; residual maxima |phi_new - phi_prev|, |phi_new|; source M (q + sigma_s
// phi_new / (4 pi)) and its (hi, lo) split.  Block = whole elements: threads (element slot, node).
__global__ void dsa_accept_kernel(DevProblem P, const double* __restrict__ half, const double* __restrict__ x,
                                  const double* __restrict__ prev, double* __restrict__ phi_new, double* __restrict__ src,
                                  float* __restrict__ src_h, float* __restrict__ src_l, unsigned long long* red) {
  extern __shared__ double sphi[];
  const int N = P.N;
  const int epb = blockDim.x / N;
  const int le = threadIdx.x / N, m = threadIdx.x % N;
  const int64_t e = (int64_t)blockIdx.x * epb + le;
  const bool ok = le < epb && e < P.E;
  double phi = 0.0, diff = 0.0, mag = 0.0;
  if (ok) {
    phi = half[e * N + m] + x[e * N + m];
    phi_new[e * N + m] = phi;
    diff = fabs(phi - prev[e * N + m]);
    mag = fabs(phi);
  }
  for (int off = 16; off > 0; off >>= 1) {
    diff = fmax(diff, __shfl_xor_sync(0xffffffffu, diff, off));
    mag = fmax(mag, __shfl_xor_sync(0xffffffffu, mag, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(red + 0, (unsigned long long)__double_as_longlong(diff));
    atomicMax(red + 1, (unsigned long long)__double_as_longlong(mag));
  }
  sphi[threadIdx.x] = phi;
  __syncthreads();
  if (ok && src != nullptr) {
    const double* Mm = P.elem + e * P.blk + (int64_t)P.dim * N * N + (int64_t)m * N;
    const double c = P.sig_s[e] * (1.0 / (4.0 * 3.14159265358979323846));
    const double* qe = P.q + e * N;
    double s = 0.0;
    for (int n2 = 0; n2 < N; ++n2) s = fma(Mm[n2], fma(c, sphi[le * N + n2], qe[n2]), s);
    src[e * N + m] = s;
    if (src_h != nullptr) {
      const float h = (float)s;
      src_h[e * N + m] = h;
      src_l[e * N + m] = (float)(s - (double)h);
    }
  }
}

}  // namespace

cudaError_t dsa_assemble(const DevProblem& P, DsaState& D, cudaStream_t s) {
  const int N = P.N, nfc = 2 * P.dim;
  const size_t shv = sizeof(double) * ((size_t)P.Q * 10);
  dsa_volume_kernel<<<(unsigned)P.E, 128, shv, s>>>(P, D.diag, D.vol);
  const int np = P.dim == 2 ? P.nf : P.K * P.K * P.nf * P.nf;
  const int spw = np * (2 + 4 * N);
  int warps = 4;
  while (warps > 1 && (size_t)warps * spw * sizeof(double) > 96 * 1024) warps >>= 1;
  const size_t shf = (size_t)warps * spw * sizeof(double);
  cudaFuncSetAttribute(dsa_face_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shf);
  const int64_t items = P.E * nfc;
  dsa_face_kernel<<<(unsigned)((items + warps - 1) / warps), warps * 32, shf, s>>>(P, D.vol, D.selfb, D.offb, spw);
  dsa_diag_kernel<<<(unsigned)((P.E + 63) / 64), 64, 0, s>>>(P.E, N, nfc, D.selfb, D.diag, D.inv, D.bad);
  return cudaGetLastError();
}

// One DSA correction: half = phi_half, prev = phi_prev; on return phi_new = half + dphi, the residual
// maxima in red[0..1] and the source for the next sweep.  *cg_iters receives the iterations run.
cudaError_t dsa_apply(const DevProblem& P, DsaState& D, const double* half, const double* prev, double* phi_new,
                      double* src, float* src_h, float* src_l, unsigned long long* red, double rtol, int max_iter,
                      int* cg_iters, int64_t* launches, cudaStream_t s) {
  const int N = P.N;
  const int64_t n = P.E * N;
  const unsigned gw = (unsigned)((P.E + 3) / 4);          // warp per element, 4 per block
  cudaError_t e = cudaMemsetAsync(D.sc, 0, 10 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  dsa_rhs_kernel<<<1216, 256, 0, s>>>(P, half, prev, D.b, D.x, D.sc);
  dsa_cg_init_kernel<<<gw, 128, 0, s>>>(P, D.inv, D.b, D.r, D.z, D.p, D.sc);
  *launches += 2;
  double bb = 0.0;
  int it = 0;
  e = cudaMemcpyAsync(&bb, D.sc, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (bb > 0.0) {
    const double target = rtol * rtol * bb;
    for (it = 0; it < max_iter;) {
      for (int k = 0; k < 8 && it < max_iter; ++k, ++it) {
        const int slot = it % 3, prevs = (it + 2) % 3, next = (it + 1) % 3;
        dsa_spmv_kernel<<<gw, 128, 0, s>>>(P, D.diag, D.offb, D.p, D.q, D.sc, slot);
        dsa_update_kernel<<<gw, 128, 0, s>>>(P, D.inv, D.p, D.q, D.x, D.r, D.z, D.sc, slot, prevs);
        dsa_pupdate_kernel<<<1216, 256, 0, s>>>(n, D.z, D.p, D.sc, slot, prevs, next);
        *launches += 3;
      }
      double rr = 0.0;
      e = cudaMemcpyAsync(&rr, D.sc + 1 + 3 * ((it - 1) % 3) + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return e;
      if (rr <= target) break;
    }
  }
  *cg_iters = it;
  const unsigned th = (unsigned)((256 / N) * N);
  const int64_t epb = th / N;
  dsa_accept_kernel<<<(unsigned)((P.E + epb - 1) / epb), th, th * sizeof(double), s>>>(P, half, D.x, prev, phi_new, src,
                                                                                      src_h, src_l, red);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace sn
