// Sweep kernel templates (per-level and persistent dataflow schedules) and their launchers,
// instantiated for the FP64, mixed and double-single forms in sweep.cu and for the form with
// stored inverses in sweep_inv.cu.
#pragma once
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

}  // namespace sn

namespace sn {
// Stored-inverse forms (sweep_inv.cu), dispatched on the form and the problem's (dim, p).
cudaError_t launch_level_t_inv(const DevProblem& P, int precision, const SweepArgs& sa, const int32_t* pairs,
                               int64_t count, cudaStream_t s);
cudaError_t launch_flow_t_inv(const DevProblem& P, int precision, const SweepArgs& sa, const int32_t* pairs,
                              int64_t count, unsigned long long* head, int blocks_per_sm, cudaStream_t s);
}  // namespace sn
