// Geometric factors of the curved elements (Sec. 2, eqs. 1, 11-16), once per problem.
// One CTA per element:
//   J(xi_q) = sum_m x_m grad v_m (eq. 14) at the tensor Gauss-Legendre volume points,
//   M_mn    = sum_q w_q |J_q| u_m u_n                          (mass, eqs. 12-13 without sigma)
//   S^k_mn  = sum_q w_q (cof(J_q) grad u_m)_k u_n = int du_m/dx_k u_n dx   (eq. 11 per axis)
//   FN[f][k]_ij = sum over face f's GL points of w (cof(J) n_hat)_k phi_i phi_j
// The sweep assembles G^(d) + F^(d) + M_t from these on the fly for every direction.
#include "devmath.cuh"

namespace sn {

template <int DIM>
__global__ void geometry_kernel(DevProblem P, double* __restrict__ elem, int* bad) {
  extern __shared__ double sh[];
  const int64_t e = blockIdx.x;
  const int N = P.N, Nf = P.Nf, Q = P.Q, Nv = P.Nv, p = P.p, r = P.r;
  double* sctrl = sh;                          // [Nv][DIM]
  double* wdet = sctrl + Nv * DIM;             // [Q]
  double* cofw = wdet + Q;                     // [Q][DIM][DIM]
  double* gradw = cofw + Q * DIM * DIM;        // [Q][N][DIM]
  const double* wq = tabp(P, P.off_wq);
  const double* B = tabp(P, P.off_B);
  const double* dB = tabp(P, P.off_dB);
  const double* dV = tabp(P, P.off_dV);
  for (int t = threadIdx.x; t < Nv * DIM; t += blockDim.x) sctrl[t] = P.ctrl[e * Nv * DIM + t];
  __syncthreads();
  for (int q = threadIdx.x; q < Q; q += blockDim.x) {
    double J[DIM][DIM];
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) J[i][j] = 0.0;
    for (int m = 0; m < Nv; ++m)
      for (int i = 0; i < DIM; ++i)
        for (int j = 0; j < DIM; ++j) J[i][j] += sctrl[m * DIM + i] * dV[((size_t)q * Nv + m) * DIM + j];
    double C[DIM][DIM];
    double det;
    if (DIM == 2) {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      C[0][0] = J[1][1];
      C[0][1] = -J[1][0];
      C[1][0] = -J[0][1];
      C[1][1] = J[0][0];
    } else {
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
          C[i][j] = J[r0][c0] * J[r1][c1] - J[r0][c1] * J[r1][c0];   // cyclic minors carry the sign
        }
      det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    }
    if (!(det > 0.0)) atomicOr(bad, 1);
    wdet[q] = wq[q] * det;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) cofw[(q * DIM + i) * DIM + j] = wq[q] * C[i][j];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < Q * N; t += blockDim.x) {
    const int q = t / N, m = t % N;
    for (int k = 0; k < DIM; ++k) {
      double g = 0.0;
      for (int j = 0; j < DIM; ++j) g += cofw[(q * DIM + k) * DIM + j] * dB[((size_t)q * N + m) * DIM + j];
      gradw[(q * N + m) * DIM + k] = g;
    }
  }
  __syncthreads();
  double* out = elem + e * P.blk;
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    const int m = t / N, n = t % N;
    double mm = 0.0, s[DIM];
    for (int k = 0; k < DIM; ++k) s[k] = 0.0;
    for (int q = 0; q < Q; ++q) {
      const double bn = B[(size_t)q * N + n];
      mm += wdet[q] * B[(size_t)q * N + m] * bn;
      for (int k = 0; k < DIM; ++k) s[k] += gradw[(q * N + m) * DIM + k] * bn;
    }
    for (int k = 0; k < DIM; ++k) out[(size_t)k * N * N + t] = s[k];
    out[(size_t)DIM * N * N + t] = mm;
  }
  __syncthreads();
  // face matrices with the element's own outward normal, base GL rule n_f^(dim-1) points
  const int nf = P.nf;
  const int Pf = (DIM == 2) ? nf : nf * nf;
  const double* gt = tabp(P, P.off_glf_t);
  const double* gw = tabp(P, P.off_glf_w);
  const double* geo = tabp(P, P.off_geo);
  const double* gll = tabp(P, P.off_gll);
  double* wn = gradw;                          // reuse: [nfc][Pf][DIM]
  for (int t = threadIdx.x; t < P.nfc * Pf; t += blockDim.x) {
    const int f = t / Pf, q = t % Pf;
    const int qi = q % nf, qj = q / nf;
    const bool tet = DIM == 3 && P.simplex;          // collapsed triangle rule on a flat face
    const double s0 = gt[qi], s1 = (DIM == 3) ? (tet ? gt[qj] * (1.0 - gt[qi]) : gt[qj]) : 0.0;
    const double w = (DIM == 3) ? (tet ? (gw[qi] * gw[qj]) * (1.0 - gt[qi]) : gw[qi] * gw[qj]) : gw[qi];
    double nv[3];
    face_normal_el(P, geo, sctrl, f, s0, s1, nv);
    for (int k = 0; k < DIM; ++k) wn[(f * Pf + q) * DIM + k] = w * nv[k];
  }
  __syncthreads();
  const int np1 = p + 1;
  double* fnout = out + (size_t)(DIM + 1) * N * N;
  for (int t = threadIdx.x; t < P.nfc * Nf * Nf; t += blockDim.x) {
    const int f = t / (Nf * Nf), ij = t % (Nf * Nf), i = ij / Nf, j = ij % Nf;
    double acc[DIM];
    for (int k = 0; k < DIM; ++k) acc[k] = 0.0;
    for (int q = 0; q < Pf; ++q) {
      const int qi = q % nf, qj = q / nf;
      const bool tet = DIM == 3 && P.simplex;
      const double s0 = gt[qi], s1 = (DIM == 3) ? (tet ? gt[qj] * (1.0 - gt[qi]) : gt[qj]) : 0.0;
      const double pp = face_basis_el_one(P, gll, i, s0, s1) * face_basis_el_one(P, gll, j, s0, s1);
      for (int k = 0; k < DIM; ++k) acc[k] += wn[(f * Pf + q) * DIM + k] * pp;
    }
    for (int k = 0; k < DIM; ++k) fnout[((size_t)(f * DIM + k) * Nf + i) * Nf + j] = acc[k];
  }
}

cudaError_t launch_geometry(const DevProblem& P, double* elem, int* bad, cudaStream_t s) {
  const int nf = P.nf;
  const int Pf = (P.dim == 2) ? nf : nf * nf;
  size_t shmem = sizeof(double) * ((size_t)P.Nv * P.dim + P.Q + (size_t)P.Q * P.dim * P.dim +
                                   std::max((size_t)P.Q * P.N * P.dim, (size_t)P.nfc * Pf * P.dim));
  if (P.dim == 2) {
    auto k = geometry_kernel<2>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
    k<<<(unsigned)P.E, 128, shmem, s>>>(P, elem, bad);
  } else {
    auto k = geometry_kernel<3>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
    k<<<(unsigned)P.E, 128, shmem, s>>>(P, elem, bad);
  }
  return cudaGetLastError();
}

// FP32 split of the element factors: hi = fl32(x), lo = fl32(x - hi) (x = hi + lo to ~2^-48).
__global__ void to_fp32_kernel(const double* __restrict__ a, float* __restrict__ hi, float* __restrict__ lo,
                               int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float h = (float)a[i];
    hi[i] = h;
    lo[i] = (float)(a[i] - (double)h);
  }
}

cudaError_t launch_elem_to_fp32(const DevProblem& P, float* elem32, float* elem32lo, cudaStream_t s) {
  int64_t n = P.E * P.blk;
  to_fp32_kernel<<<1216, 256, 0, s>>>(P.elem, elem32, elem32lo, n);
  return cudaGetLastError();
}

}  // namespace sn

namespace sn {

// Volume quadrature points of every element and the squared L2 distance of a nodal field from
// given point values (for manufactured-solution errors): one CTA per element,
//   x_q = sum_m x_m v_m(xi_q),  err^2 += sum_q w_q |J_q| (sum_n u_n(xi_q) phi_n - exact_q)^2.
template <int DIM>
__global__ void volume_points_kernel(DevProblem P, const double* __restrict__ phi, const double* __restrict__ exact_q,
                                     double* __restrict__ xq, double* acc) {
  __shared__ double sctrl[64 * 3];
  __shared__ double part[4];
  const int64_t e = blockIdx.x;
  const int N = P.N, Q = P.Q, Nv = P.Nv;
  const double* wq = tabp(P, P.off_wq);
  const double* B = tabp(P, P.off_B);
  const double* dV = tabp(P, P.off_dV);
  const double* V = tabp(P, P.off_V);
  for (int t = threadIdx.x; t < Nv * DIM; t += blockDim.x) sctrl[t] = P.ctrl[e * Nv * DIM + t];
  __syncthreads();
  double local = 0.0;
  for (int q = threadIdx.x; q < Q; q += blockDim.x) {
    double J[DIM][DIM], x[DIM];
    for (int i = 0; i < DIM; ++i) {
      x[i] = 0.0;
      for (int j = 0; j < DIM; ++j) J[i][j] = 0.0;
    }
    for (int m = 0; m < Nv; ++m) {
      const double v = V[(size_t)q * Nv + m];
      for (int i = 0; i < DIM; ++i) {
        x[i] += sctrl[m * DIM + i] * v;
        for (int j = 0; j < DIM; ++j) J[i][j] += sctrl[m * DIM + i] * dV[((size_t)q * Nv + m) * DIM + j];
      }
    }
    if (xq != nullptr)
      for (int i = 0; i < DIM; ++i) xq[(e * Q + q) * DIM + i] = x[i];
    if (phi != nullptr) {
      double det;
      if (DIM == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      } else {
        det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
              J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      }
      double val = 0.0;
      for (int n = 0; n < N; ++n) val += B[(size_t)q * N + n] * phi[e * N + n];
      const double dlt = val - exact_q[e * Q + q];
      local += wq[q] * det * dlt * dlt;
    }
  }
  if (phi == nullptr) return;
  for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(acc, part[0] + part[1] + part[2] + part[3]);
}

cudaError_t launch_volume_points(const DevProblem& P, const double* phi, const double* exact_q, double* xq,
                                 double* acc, cudaStream_t s) {
  if (P.Nv * P.dim > 64 * 3) return cudaErrorInvalidValue;
  if (P.dim == 2) volume_points_kernel<2><<<(unsigned)P.E, 128, 0, s>>>(P, phi, exact_q, xq, acc);
  else volume_points_kernel<3><<<(unsigned)P.E, 128, 0, s>>>(P, phi, exact_q, xq, acc);
  return cudaGetLastError();
}

}  // namespace sn
