// Lagged transport sweep (Sec. 3, eq. 21) and scalar-flux moment / scattering source
// (eqs. 2 and 18) on the device.
//
// Every (element, direction) pair is one small dense system A psi_e = b solved by a W-lane
// segment of a warp (W = next power of two >= N; 32/W systems per warp).  Lane i owns row i
// of the system in registers:
//   A = sum_k Omega_k (S^k)^T + sigma_t M + sum_{inflow faces} B_f      (strong form of
//       G + F_e + M_t: int (Omega.grad u_n) u_m + sigma_t int u_m u_n + oint max(-Omega.n,0) u_m u_n)
//   b = src_e + sum_{inflow faces} B_f trace_f
// with B_f = -Omega . FN_f on whole-inflow faces and the stored block on partially-inflow
// faces; trace_f = the upwind neighbour's nodal values on the face (new iterate for kept
// arcs, previous iterate for lagged ones) or the incident flux on the domain boundary.
// Elimination: partial pivoting by a segment-wide argmax; rows are not moved, the pivot row is
// broadcast by shuffles; back substitution in pivot order.
//
// Three arithmetic forms (SN_PREC_*): FP64; FP32 LU + one refinement with an FP64 residual;
// FP32 LU + one refinement with the row and residual in double-single (FP32 pairs).
// Two schedules: one launch per wavefront level (pairs of a level are independent), or one
// persistent "dataflow" launch per sweep in which warps take pairs from a queue in level order
// and wait only for the completion flags of their kept upwind neighbours.
#include "sweep_kernels.cuh"

namespace sn {

// Template instance of the form and the problem's (dim, p); the stored-inverse forms live in
// sweep_inv.cu.
#define SN_CASE(FN, D, PP, ...)                                                                    \
  if (P.dim == D && P.p == PP) {                                                                   \
    if (precision == SN_PREC_FP64) return FN<D, PP, SN_PREC_FP64>(P, __VA_ARGS__);                 \
    if (precision == SN_PREC_MIXED) return FN<D, PP, SN_PREC_MIXED>(P, __VA_ARGS__);               \
    return FN<D, PP, SN_PREC_MIXED_DS>(P, __VA_ARGS__);                                            \
  }
#define SN_DISPATCH(FN, ...)                                                                       \
  do {                                                                                             \
    if (precision == SN_PREC_FP64_INV || precision == SN_PREC_DS_INV)                              \
      return FN##_inv(P, precision, __VA_ARGS__);                                                  \
    SN_CASE(FN, 2, 1, __VA_ARGS__)                                                                 \
    SN_CASE(FN, 2, 2, __VA_ARGS__)                                                                 \
    SN_CASE(FN, 2, 3, __VA_ARGS__)                                                                 \
    SN_CASE(FN, 3, 1, __VA_ARGS__)                                                                 \
    SN_CASE(FN, 3, 2, __VA_ARGS__)                                                                 \
    return cudaErrorInvalidValue;                                                                  \
  } while (0)

cudaError_t launch_sweep_level(const DevProblem& P, int precision, const int32_t* pairs, int64_t count,
                               const SweepArgs& sa, cudaStream_t s) {
  SN_DISPATCH(launch_level_t, sa, pairs, count, s);
}

cudaError_t launch_sweep_flow(const DevProblem& P, int precision, const int32_t* pairs, int64_t count,
                              const SweepArgs& sa, unsigned long long* head, int blocks_per_sm, cudaStream_t s) {
  SN_DISPATCH(launch_flow_t, sa, pairs, count, head, blocks_per_sm, s);
}

// ------------------------------------------------------------------ moment and source
__device__ inline void block_max2(double& a, double& b) {
  __shared__ double ra[32], rb[32];
  for (int off = 16; off > 0; off >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, off));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, off));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    ra[w] = a;
    rb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    a = l < nw ? ra[l] : 0.0;
    b = l < nw ? rb[l] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      a = fmax(a, __shfl_xor_sync(0xffffffffu, a, off));
      b = fmax(b, __shfl_xor_sync(0xffffffffu, b, off));
    }
  }
}

// phi = sum_d w_d psi_d (d ascending); residual maxima; src = M (q + sigma_s phi / (4 pi)).
// Block = whole elements: threads (element slot, node).
__global__ void moment_kernel(DevProblem P, const double* __restrict__ psi, const double* __restrict__ phi_prev,
                              double* __restrict__ phi_out, double* __restrict__ src, float* __restrict__ src_h,
                              float* __restrict__ src_l, unsigned long long* red) {
  extern __shared__ double sphi[];
  const int N = P.N;
  const int epb = blockDim.x / N;
  const int le = threadIdx.x / N, m = threadIdx.x % N;
  const int64_t e = (int64_t)blockIdx.x * epb + le;
  const bool ok = le < epb && e < P.E;
  double phi = 0.0;
  if (ok && psi != nullptr) {
    for (int d = 0; d < P.M; ++d) phi = fma(P.w[d], __ldg(psi + ((int64_t)d * P.E + e) * N + m), phi);
  } else if (ok) {
    phi = phi_prev ? phi_prev[e * N + m] : 0.0;
  }
  if (red != nullptr) {
    double diff = ok ? fabs(phi - (phi_prev ? phi_prev[e * N + m] : 0.0)) : 0.0;
    double mag = ok ? fabs(phi) : 0.0;
    block_max2(diff, mag);
    if (threadIdx.x == 0) {
      atomicMax(red + 0, (unsigned long long)__double_as_longlong(diff));
      atomicMax(red + 1, (unsigned long long)__double_as_longlong(mag));
    }
  }
  if (ok && phi_out != nullptr) phi_out[e * N + m] = phi;
  sphi[threadIdx.x] = phi;
  __syncthreads();
  if (ok && src != nullptr) {
    const double* Mm = P.elem + e * P.blk + (int64_t)P.dim * N * N + (int64_t)m * N;
    const double c = P.sig_s[e] * (1.0 / (4.0 * 3.14159265358979323846));
    const double* qe = P.q + e * N;
    double s = 0.0;
    for (int n = 0; n < N; ++n) s = fma(Mm[n], fma(c, sphi[le * N + n], qe[n]), s);
    src[e * N + m] = s;
    if (src_h != nullptr) {
      const float h = (float)s;
      src_h[e * N + m] = h;
      src_l[e * N + m] = (float)(s - (double)h);
    }
  }
}

static unsigned moment_threads(int N) { return (unsigned)((256 / N) * N); }

cudaError_t launch_moment(const DevProblem& P, const double* psi, const double* phi_prev, double* phi_out,
                          double* src, float* src_h, float* src_l, unsigned long long* red, cudaStream_t s) {
  const unsigned th = moment_threads(P.N);
  const int64_t epb = th / P.N;
  const int64_t blocks = (P.E + epb - 1) / epb;
  moment_kernel<<<(unsigned)blocks, th, th * sizeof(double), s>>>(P, psi, phi_prev, phi_out, src, src_h, src_l, red);
  return cudaGetLastError();
}

cudaError_t launch_source(const DevProblem& P, const double* phi, double* src, float* src_h, float* src_l,
                          cudaStream_t s) {
  return launch_moment(P, nullptr, phi, nullptr, src, src_h, src_l, nullptr, s);
}

// x = h + l with h = fl32(x), l = fl32(x - h).
__global__ void split_kernel(const double* __restrict__ x, float* __restrict__ h, float* __restrict__ l, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float a = (float)x[i];
    h[i] = a;
    l[i] = (float)(x[i] - (double)a);
  }
}

cudaError_t launch_split(const double* x, float* h, float* l, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  split_kernel<<<1216, 256, 0, s>>>(x, h, l, n);
  return cudaGetLastError();
}

}  // namespace sn
