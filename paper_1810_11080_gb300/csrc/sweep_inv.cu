// Lagged sweep with stored local inverses (SN_PREC_FP64_INV, SN_PREC_DS_INV): the inverse of
// every (direction, element) matrix G + F_e + M_t of eq. 21 and its inflow face blocks are formed
// once per problem by invert_kernel, and each sweep applies them (inverse_body.cuh).
#include "sweep_kernels.cuh"

namespace sn {

// All M E pairs at once (no dependencies between them): pair q = d E + e, S::SPW pairs per warp.
template <int DIM, int P_, bool DSOUT>
__global__ void __launch_bounds__(128) invert_kernel(DevProblem Pb, SweepArgs sa, int64_t count) {
  using S = Shape<DIM, P_>;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t q = gwarp * S::SPW + lane / S::W;
  invert_pair<DIM, P_, DSOUT>(Pb, sa, q < count ? q : 0, q < count, lane);
}

template <int DIM, int P_>
static cudaError_t launch_invert_t(const DevProblem& P, int precision, const SweepArgs& sa, cudaStream_t s) {
  using S = Shape<DIM, P_>;
  const int64_t count = (int64_t)P.M * P.E;
  const int64_t per_block = 4 * S::SPW;
  const int64_t blocks = (count + per_block - 1) / per_block;
  if (blocks == 0) return cudaSuccess;
  if (precision == SN_PREC_DS_INV) invert_kernel<DIM, P_, true><<<(unsigned)blocks, 128, 0, s>>>(P, sa, count);
  else invert_kernel<DIM, P_, false><<<(unsigned)blocks, 128, 0, s>>>(P, sa, count);
  return cudaGetLastError();
}

#define SN_DISPATCH_DP(FN, ...)                                                   \
  do {                                                                           \
    if (P.dim == 2 && P.p == 1) return FN<2, 1>(__VA_ARGS__);                    \
    if (P.dim == 2 && P.p == 2) return FN<2, 2>(__VA_ARGS__);                    \
    if (P.dim == 2 && P.p == 3) return FN<2, 3>(__VA_ARGS__);                    \
    if (P.dim == 3 && P.p == 1) return FN<3, 1>(__VA_ARGS__);                    \
    if (P.dim == 3 && P.p == 2) return FN<3, 2>(__VA_ARGS__);                    \
    return cudaErrorInvalidValue;                                                \
  } while (0)

template <int DIM, int P_>
static cudaError_t level_inv(const DevProblem& P, int precision, const SweepArgs& sa, const int32_t* pairs,
                             int64_t count, cudaStream_t s) {
  if (precision == SN_PREC_DS_INV) return launch_level_t<DIM, P_, SN_PREC_DS_INV>(P, sa, pairs, count, s);
  return launch_level_t<DIM, P_, SN_PREC_FP64_INV>(P, sa, pairs, count, s);
}

template <int DIM, int P_>
static cudaError_t flow_inv(const DevProblem& P, int precision, const SweepArgs& sa, const int32_t* pairs,
                            int64_t count, unsigned long long* head, int blocks_per_sm, cudaStream_t s) {
  if (precision == SN_PREC_DS_INV)
    return launch_flow_t<DIM, P_, SN_PREC_DS_INV>(P, sa, pairs, count, head, blocks_per_sm, s);
  return launch_flow_t<DIM, P_, SN_PREC_FP64_INV>(P, sa, pairs, count, head, blocks_per_sm, s);
}

cudaError_t launch_level_t_inv(const DevProblem& P, int precision, const SweepArgs& sa, const int32_t* pairs,
                               int64_t count, cudaStream_t s) {
  SN_DISPATCH_DP(level_inv, P, precision, sa, pairs, count, s);
}

cudaError_t launch_flow_t_inv(const DevProblem& P, int precision, const SweepArgs& sa, const int32_t* pairs,
                              int64_t count, unsigned long long* head, int blocks_per_sm, cudaStream_t s) {
  SN_DISPATCH_DP(flow_inv, P, precision, sa, pairs, count, head, blocks_per_sm, s);
}

cudaError_t launch_invert(const DevProblem& P, int precision, const SweepArgs& sa, cudaStream_t s) {
  SN_DISPATCH_DP(launch_invert_t, P, precision, sa, s);
}

}  // namespace sn
