// Lagged sweep with stored local inverses (SN_PREC_FP64_INV, SN_PREC_DS_INV): the inverse of
// every (direction, element) matrix G + F_e + M_t of eq. 21 and its inflow face blocks are formed
// once per problem by invert_kernel, and each sweep applies them (inverse_body.cuh).  The
// kernels are instantiated for the tensor elements (quadrilaterals, hexahedra) and for
// triangles.
#include "sweep_kernels.cuh"

namespace sn {

// All M E pairs at once (no dependencies between them): pair q = d E + e, El::SPW pairs per warp.
template <class El, bool DSOUT>
__global__ void __launch_bounds__(128) invert_kernel(DevProblem Pb, SweepArgs sa, int64_t count) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t q = gwarp * El::SPW + lane / El::W;
  invert_pair<El, DSOUT>(Pb, sa, q < count ? q : 0, q < count, lane);
}

template <class El>
static cudaError_t launch_invert_el(const DevProblem& P, int precision, const SweepArgs& sa, cudaStream_t s) {
  const int64_t count = (int64_t)P.M * P.E;
  const int64_t per_block = 4 * El::SPW;
  const int64_t blocks = (count + per_block - 1) / per_block;
  if (blocks == 0) return cudaSuccess;
  if (precision == SN_PREC_DS_INV) invert_kernel<El, true><<<(unsigned)blocks, 128, 0, s>>>(P, sa, count);
  else invert_kernel<El, false><<<(unsigned)blocks, 128, 0, s>>>(P, sa, count);
  return cudaGetLastError();
}

template <class El, int PREC, bool DF>
__device__ __forceinline__ void solve_el(const DevProblem& Pb, const SweepArgs& sa, int32_t pr, bool valid,
                                         int lane) {
  if constexpr (PREC == SN_PREC_DS_INV) bodydsinv<El, DF>(Pb, sa, pr, valid, lane);
  else bodyinv<El, DF>(Pb, sa, pr, valid, lane);
}

// Resident 128-thread blocks per SM the kernels are compiled for (register budget).
template <class El, int PREC>
constexpr int inv_minb() {
  if (El::N > 16) return PREC == SN_PREC_DS_INV ? 4 : 3;      // 3D p = 2 rows
  return 5;
}

// One wavefront level (see sweep_level_kernel) and the whole sweep in one persistent launch
// (see sweep_flow_kernel), for an element policy.
template <class El, int PREC>
__global__ void __launch_bounds__(128, (inv_minb<El, PREC>())) el_level_kernel(DevProblem Pb, SweepArgs sa,
                                                                                const int32_t* __restrict__ pairs,
                                                                                int64_t count) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t item = gwarp * El::SPW + lane / El::W;
  const int32_t pr = item < count ? pairs[item] : -1;
  solve_el<El, PREC, false>(Pb, sa, pr < 0 ? 0 : pr, pr >= 0, lane);
}

// Work-queue granularity of the dataflow kernel: a warp takes FLOW_CHUNK consecutive tasks
// (FLOW_CHUNK El::SPW pairs of the level-ordered list) per atomic on the queue head and solves
// them in order; the bodies here are light enough that one atomic per task would make the shared
// queue head the bottleneck.  Still deadlock-free: a pair waits only for pairs earlier in the
// list, which were handed out before it to running warps.
constexpr int FLOW_CHUNK = 2;

template <class El, int PREC>
__global__ void __launch_bounds__(128, (inv_minb<El, PREC>() > 2 ? inv_minb<El, PREC>() - 1 : 2))
    el_flow_kernel(DevProblem Pb, SweepArgs sa, const int32_t* __restrict__ pairs, int64_t count,
                   unsigned long long* head) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  while (true) {
    long long t = 0;
    if (lane == 0)
      t = (*(volatile int*)sa.err) ? count : (long long)atomicAdd(head, (unsigned long long)(FLOW_CHUNK * El::SPW));
    t = __shfl_sync(FULL, t, 0);
    if (t >= count) break;
#pragma unroll 1
    for (int c = 0; c < FLOW_CHUNK; ++c) {
      const int64_t item = t + c * El::SPW + lane / El::W;
      const int32_t pr = item < count ? pairs[item] : -1;
      solve_el<El, PREC, true>(Pb, sa, pr < 0 ? 0 : pr, pr >= 0, lane);
    }
  }
}

template <class El, int PREC>
static cudaError_t level_el(const DevProblem& P, const SweepArgs& sa, const int32_t* pairs, int64_t count,
                            cudaStream_t s) {
  const int threads = 128;
  const int64_t per_block = (threads / 32) * El::SPW;
  const int64_t blocks = (count + per_block - 1) / per_block;
  if (blocks == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(threads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, el_level_kernel<El, PREC>, P, sa, pairs, count);
}

template <class El, int PREC>
static cudaError_t flow_el(const DevProblem& P, const SweepArgs& sa, const int32_t* pairs, int64_t count,
                           unsigned long long* head, int blocks_per_sm, cudaStream_t s) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, el_flow_kernel<El, PREC>, 128, 0);
  if (occ < 1) occ = 1;
  const int bps = blocks_per_sm > 0 ? std::min(blocks_per_sm, occ) : occ;
  el_flow_kernel<El, PREC><<<(unsigned)(sms * bps), 128, 0, s>>>(P, sa, pairs, count, head);
  return cudaGetLastError();
}

// Element policy of the problem: triangles (P_p, p = 1..3), tetrahedra (p = 1, 2) or tensor
// elements (dim, p).
#define SN_DISPATCH_EL(FN, ...)                                                   \
  do {                                                                           \
    if (P.simplex && P.dim == 3) {                                               \
      if (P.p == 1) return FN<TetEl<1>>(__VA_ARGS__);                            \
      if (P.p == 2) return FN<TetEl<2>>(__VA_ARGS__);                            \
      return cudaErrorInvalidValue;                                              \
    }                                                                            \
    if (P.simplex) {                                                             \
      if (P.p == 1) return FN<TriEl<1>>(__VA_ARGS__);                            \
      if (P.p == 2) return FN<TriEl<2>>(__VA_ARGS__);                            \
      if (P.p == 3) return FN<TriEl<3>>(__VA_ARGS__);                            \
      return cudaErrorInvalidValue;                                              \
    }                                                                            \
    if (P.dim == 2 && P.p == 1) return FN<TensorEl<2, 1>>(__VA_ARGS__);          \
    if (P.dim == 2 && P.p == 2) return FN<TensorEl<2, 2>>(__VA_ARGS__);          \
    if (P.dim == 2 && P.p == 3) return FN<TensorEl<2, 3>>(__VA_ARGS__);          \
    if (P.dim == 3 && P.p == 1) return FN<TensorEl<3, 1>>(__VA_ARGS__);          \
    if (P.dim == 3 && P.p == 2) return FN<TensorEl<3, 2>>(__VA_ARGS__);          \
    return cudaErrorInvalidValue;                                                \
  } while (0)

template <class El>
static cudaError_t level_inv(const DevProblem& P, int precision, const SweepArgs& sa, const int32_t* pairs,
                             int64_t count, cudaStream_t s) {
  if (precision == SN_PREC_DS_INV) return level_el<El, SN_PREC_DS_INV>(P, sa, pairs, count, s);
  return level_el<El, SN_PREC_FP64_INV>(P, sa, pairs, count, s);
}

template <class El>
static cudaError_t flow_inv(const DevProblem& P, int precision, const SweepArgs& sa, const int32_t* pairs,
                            int64_t count, unsigned long long* head, int blocks_per_sm, cudaStream_t s) {
  if (precision == SN_PREC_DS_INV) return flow_el<El, SN_PREC_DS_INV>(P, sa, pairs, count, head, blocks_per_sm, s);
  return flow_el<El, SN_PREC_FP64_INV>(P, sa, pairs, count, head, blocks_per_sm, s);
}

cudaError_t launch_level_t_inv(const DevProblem& P, int precision, const SweepArgs& sa, const int32_t* pairs,
                               int64_t count, cudaStream_t s) {
  SN_DISPATCH_EL(level_inv, P, precision, sa, pairs, count, s);
}

cudaError_t launch_flow_t_inv(const DevProblem& P, int precision, const SweepArgs& sa, const int32_t* pairs,
                              int64_t count, unsigned long long* head, int blocks_per_sm, cudaStream_t s) {
  SN_DISPATCH_EL(flow_inv, P, precision, sa, pairs, count, head, blocks_per_sm, s);
}

cudaError_t launch_invert(const DevProblem& P, int precision, const SweepArgs& sa, cudaStream_t s) {
  SN_DISPATCH_EL(launch_invert_el, P, precision, sa, s);
}

}  // namespace sn
