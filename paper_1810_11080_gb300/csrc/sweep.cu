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
#include "sweep_body.cuh"

namespace sn {

// One wavefront level: pairs[0, count) are mutually independent.
template <int DIM, int P_, int PREC>
__global__ void __launch_bounds__(128, (sweep_minb<DIM, P_, PREC>())) sweep_level_kernel(DevProblem Pb, SweepArgs sa, const int32_t* __restrict__ pairs,
                                                          int64_t count) {
  using S = Shape<DIM, P_>;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t item = gwarp * S::SPW + lane / S::W;
  const int32_t pr = item < count ? pairs[item] : -1;
  solve_item<DIM, P_, PREC, false>(Pb, sa, pr < 0 ? 0 : pr, pr >= 0, lane);
}

// Whole sweep in one launch (one resident block per SM less than the level kernel: the queue
// loop holds a few more values): warps take S::SPW consecutive pairs of the level-ordered list from
// the queue head; a pair waits only for its kept upwind neighbours (always handed out earlier,
// hence held by running warps: no deadlock whatever the grid size).
template <int DIM, int P_, int PREC>
__global__ void __launch_bounds__(128, (sweep_minb<DIM, P_, PREC>() > 2 ? sweep_minb<DIM, P_, PREC>() - 1 : 2)) sweep_flow_kernel(DevProblem Pb, SweepArgs sa, const int32_t* __restrict__ pairs,
                                                         int64_t count, unsigned long long* head) {
  using S = Shape<DIM, P_>;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  while (true) {
    long long t = 0;
    if (lane == 0) t = (*(volatile int*)sa.err) ? count : (long long)atomicAdd(head, (unsigned long long)S::SPW);
    t = __shfl_sync(FULL, t, 0);
    if (t >= count) break;
    const int64_t item = t + lane / S::W;
    const int32_t pr = item < count ? pairs[item] : -1;
    solve_item<DIM, P_, PREC, true>(Pb, sa, pr < 0 ? 0 : pr, pr >= 0, lane);
  }
}

template <int DIM, int P_, int PREC>
static cudaError_t launch_level_t(const DevProblem& P, const SweepArgs& sa, const int32_t* pairs, int64_t count,
                                  cudaStream_t s) {
  using S = Shape<DIM, P_>;
  const int threads = 128;
  const int64_t per_block = (threads / 32) * S::SPW;
  const int64_t blocks = (count + per_block - 1) / per_block;
  if (blocks == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(threads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  // The FP64 form is bound by the FP64 pipe: an overlapped next level would only compete for it.
  cfg.attrs = attr;
  cfg.numAttrs = (PREC == SN_PREC_FP64) ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, sweep_level_kernel<DIM, P_, PREC>, P, sa, pairs, count);
}

template <int DIM, int P_, int PREC>
static cudaError_t launch_flow_t(const DevProblem& P, const SweepArgs& sa, const int32_t* pairs, int64_t count,
                                 unsigned long long* head, int blocks_per_sm, cudaStream_t s) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sweep_flow_kernel<DIM, P_, PREC>, 128, 0);
  if (occ < 1) occ = 1;
  const int bps = blocks_per_sm > 0 ? std::min(blocks_per_sm, occ) : occ;
  sweep_flow_kernel<DIM, P_, PREC><<<(unsigned)(sms * bps), 128, 0, s>>>(P, sa, pairs, count, head);
  return cudaGetLastError();
}

#define SN_DISPATCH(FN, ...)                                                                        \
  do {                                                                                              \
    if (P.dim == 2 && P.p == 1) { if (precision == 0) return FN<2, 1, 0>(__VA_ARGS__); if (precision == 1) return FN<2, 1, 1>(__VA_ARGS__); return FN<2, 1, 2>(__VA_ARGS__); } \
    if (P.dim == 2 && P.p == 2) { if (precision == 0) return FN<2, 2, 0>(__VA_ARGS__); if (precision == 1) return FN<2, 2, 1>(__VA_ARGS__); return FN<2, 2, 2>(__VA_ARGS__); } \
    if (P.dim == 2 && P.p == 3) { if (precision == 0) return FN<2, 3, 0>(__VA_ARGS__); if (precision == 1) return FN<2, 3, 1>(__VA_ARGS__); return FN<2, 3, 2>(__VA_ARGS__); } \
    if (P.dim == 3 && P.p == 1) { if (precision == 0) return FN<3, 1, 0>(__VA_ARGS__); if (precision == 1) return FN<3, 1, 1>(__VA_ARGS__); return FN<3, 1, 2>(__VA_ARGS__); } \
    if (P.dim == 3 && P.p == 2) { if (precision == 0) return FN<3, 2, 0>(__VA_ARGS__); if (precision == 1) return FN<3, 2, 1>(__VA_ARGS__); return FN<3, 2, 2>(__VA_ARGS__); } \
    return cudaErrorInvalidValue;                                                                   \
  } while (0)

cudaError_t launch_sweep_level(const DevProblem& P, int precision, const int32_t* pairs, int64_t count,
                               const SweepArgs& sa, cudaStream_t s) {
  SN_DISPATCH(launch_level_t, P, sa, pairs, count, s);
}

cudaError_t launch_sweep_flow(const DevProblem& P, int precision, const int32_t* pairs, int64_t count,
                              const SweepArgs& sa, unsigned long long* head, int blocks_per_sm, cudaStream_t s) {
  SN_DISPATCH(launch_flow_t, P, sa, pairs, count, head, blocks_per_sm, s);
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
