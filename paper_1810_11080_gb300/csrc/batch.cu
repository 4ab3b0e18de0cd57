// Batched sweeps: many independent problems (uneven mesh sizes, DG orders, direction sets) in
// one persistent launch.  Work items are warp tasks -- up to 32/W pairs of one level of one
// problem -- ordered by level across all problems; warps take tasks from a queue (dataflow
// schedule: each pair waits only for its own problem's kept upwind neighbours) or one task per
// warp within a single level (level schedule).  A task selects the solve's template instance
// by its DG order p.
#include "sweep_body.cuh"

namespace sn {

template <int DIM, int P_, int PREC, bool DF>
__device__ __forceinline__ void batch_task(const DevProblem& Pb, const SweepArgs& sa, int off, int lane) {
  using S = Shape<DIM, P_>;
  const int64_t idx = (int64_t)off + lane / S::W;
  const int32_t pr = sa.pairs[idx];     // tasks never run past a problem's padded level
  solve_item<DIM, P_, PREC, DF>(Pb, sa, pr < 0 ? 0 : pr, pr >= 0, lane);
}

// Register budget of the largest body the kernel holds (2D p = 3; 3D p = 2 with one block per SM
// less, as every order's body shares the budget).
template <int DIM, int PREC>
constexpr int batch_minb() {
  return DIM == 2 ? sweep_minb<2, 3, PREC>() : (sweep_minb<3, 2, PREC>() > 2 ? sweep_minb<3, 2, PREC>() - 1 : 2);
}
template <int DIM, int PREC, bool DF>
__global__ void __launch_bounds__(128, (batch_minb<DIM, PREC>())) sweep_batch_kernel(const DevProblem* __restrict__ probs,
                                                          const SweepArgs* __restrict__ args,
                                                          const int4* __restrict__ tasks, int64_t ntasks,
                                                          unsigned long long* head, int* err) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  while (true) {
    if constexpr (DF) {
      long long tt = 0;
      if (lane == 0) tt = (*(volatile int*)err) ? ntasks : (long long)atomicAdd(head, 1ull);
      t = __shfl_sync(FULL, tt, 0);
    }
    if (t >= ntasks) break;
    const int4 task = tasks[t];
    const DevProblem& Pb = probs[task.x];
    const SweepArgs& sa = args[task.x];
    switch (task.y) {
      case 1:
        batch_task<DIM, 1, PREC, DF>(Pb, sa, task.z, lane);
        break;
      case 2:
        batch_task<DIM, 2, PREC, DF>(Pb, sa, task.z, lane);
        break;
      default:
        if constexpr (DIM == 2) batch_task<DIM, 3, PREC, DF>(Pb, sa, task.z, lane);
        break;
    }
    if constexpr (!DF) break;
  }
}

template <int DIM, int PREC, bool DF>
static cudaError_t launch_batch_t(const DevProblem* probs, const SweepArgs* args, const int4* tasks, int64_t ntasks,
                                  unsigned long long* head, int* err, int blocks_per_sm, cudaStream_t s) {
  if (ntasks == 0) return cudaSuccess;
  if constexpr (DF) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sweep_batch_kernel<DIM, PREC, DF>, 128, 0);
    if (occ < 1) occ = 1;
    const int bps = blocks_per_sm > 0 ? std::min(blocks_per_sm, occ) : occ;
    sweep_batch_kernel<DIM, PREC, DF><<<(unsigned)(sms * bps), 128, 0, s>>>(probs, args, tasks, ntasks, head, err);
  } else {
    const int64_t blocks = (ntasks + 3) / 4;
    sweep_batch_kernel<DIM, PREC, DF><<<(unsigned)blocks, 128, 0, s>>>(probs, args, tasks, ntasks, head, err);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_sweep(int dim, int precision, bool dataflow, const DevProblem* probs, const SweepArgs* args,
                               const int4* tasks, int64_t ntasks, unsigned long long* head, int* err,
                               int blocks_per_sm, cudaStream_t s) {
#define SN_BATCH_CASE(D, PR)                                                                           \
  if (dim == D && precision == PR)                                                                    \
    return dataflow ? launch_batch_t<D, PR, true>(probs, args, tasks, ntasks, head, err, blocks_per_sm, s) \
                    : launch_batch_t<D, PR, false>(probs, args, tasks, ntasks, head, err, blocks_per_sm, s);
  SN_BATCH_CASE(2, 0)
  SN_BATCH_CASE(2, 1)
  SN_BATCH_CASE(2, 2)
  SN_BATCH_CASE(3, 0)
  SN_BATCH_CASE(3, 1)
  SN_BATCH_CASE(3, 2)
  SN_BATCH_CASE(2, 3)
  SN_BATCH_CASE(3, 3)
  SN_BATCH_CASE(2, 4)
  SN_BATCH_CASE(3, 4)
#undef SN_BATCH_CASE
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ batched moment + source
// Block b belongs to the problem k with block_off[k] <= b < block_off[k+1]; inside a problem the
// block covers 256 / N whole elements, as moment_kernel does.
__global__ void moment_batch_kernel(const DevProblem* __restrict__ probs, const MomentArgs* __restrict__ margs,
                                    const int64_t* __restrict__ block_off, int nprob, unsigned long long* red) {
  __shared__ double sphi[256];
  __shared__ double ra[8], rb[8];
  int lo = 0, hi = nprob - 1;
  const int64_t b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (block_off[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const int k = lo;
  const DevProblem& P = probs[k];
  const MomentArgs& ma = margs[k];
  const int N = P.N;
  const int epb = 256 / N;
  const int le = threadIdx.x / N, m = threadIdx.x % N;
  const int64_t e = (b - block_off[k]) * epb + le;
  const bool ok = le < epb && e < P.E;
  double phi = 0.0, prev = 0.0;
  if (ok) {
    for (int d = 0; d < P.M; ++d) phi = fma(P.w[d], __ldg(ma.psi + ((int64_t)d * P.E + e) * N + m), phi);
    prev = ma.phi_prev[e * N + m];
    ma.phi_out[e * N + m] = phi;
  }
  double diff = ok ? fabs(phi - prev) : 0.0, mag = ok ? fabs(phi) : 0.0;
  for (int off = 16; off > 0; off >>= 1) {
    diff = fmax(diff, __shfl_xor_sync(0xffffffffu, diff, off));
    mag = fmax(mag, __shfl_xor_sync(0xffffffffu, mag, off));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    ra[w] = diff;
    rb[w] = mag;
  }
  sphi[threadIdx.x] = phi;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) {
      a = fmax(a, ra[j]);
      c = fmax(c, rb[j]);
    }
    atomicMax(red + 2 * k, (unsigned long long)__double_as_longlong(a));
    atomicMax(red + 2 * k + 1, (unsigned long long)__double_as_longlong(c));
  }
  if (ok) {
    const double* Mm = P.elem + e * P.blk + (int64_t)P.dim * N * N + (int64_t)m * N;
    const double cs = P.sig_s[e] * (1.0 / (4.0 * 3.14159265358979323846));
    const double* qe = P.q + e * N;
    double s = 0.0;
    for (int n = 0; n < N; ++n) s = fma(Mm[n], fma(cs, sphi[le * N + n], qe[n]), s);
    ma.src[e * N + m] = s;
    if (ma.src_h != nullptr) {
      const float h = (float)s;
      ma.src_h[e * N + m] = h;
      ma.src_l[e * N + m] = (float)(s - (double)h);
    }
  }
}

cudaError_t launch_batch_moment(const DevProblem* probs, const MomentArgs* margs, const int64_t* block_off,
                                int nprob, int64_t nblocks, unsigned long long* red, cudaStream_t s) {
  if (nblocks == 0) return cudaSuccess;
  moment_batch_kernel<<<(unsigned)nblocks, 256, 0, s>>>(probs, margs, block_off, nprob, red);
  return cudaGetLastError();
}

}  // namespace sn
