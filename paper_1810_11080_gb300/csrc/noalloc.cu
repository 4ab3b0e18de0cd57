// sn_moment_noalloc: the scalar-flux moment and relative-change computation of sn_moment,
// for callers that cannot allocate device memory.
//
// Who needs it: a caller that only holds raw device buffers handed to it by a host framework
// which owns all device memory through its own allocator (fixed memory budget, no side
// allocations), or that must not call cudaMalloc/cudaFree because those calls synchronise
// the whole device and stall the framework's other streams.  Such a caller cannot create an
// sn_ctx (which allocates its workspace) but can still call this function.
//
// Scratch: the residual reduction needs one (difference, magnitude) pair per thread block
// plus one final pair.  It lives in the file-scope device array below, sized for
// SN_NOALLOC_MAX_BLOCKS blocks (256 KiB + 16 B); every GPU that loads this library holds it
// until the process exits.  Host code cannot use the array's name as a device address: the
// address is looked up once per device with cudaGetSymbolAddress and passed to the kernels.
#include <cstring>
#include <mutex>
#include "common.h"

namespace sn {
namespace {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_BLOCKS = 16384;          // => at most 4,194,304 (element, node) values
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_BLOCKS + 2];

std::mutex g_mu;
double* g_scratch_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

// Block-level max of a pair, result valid in thread 0.
__device__ void block_max_pair(double& a, double& b) {
  __shared__ double sa[NOALLOC_THREADS / 32], sb[NOALLOC_THREADS / 32];
  for (int off = 16; off > 0; off >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, off));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, off));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = l < (int)(blockDim.x >> 5) ? sa[l] : 0.0;
    b = l < (int)(blockDim.x >> 5) ? sb[l] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      a = fmax(a, __shfl_xor_sync(0xffffffffu, a, off));
      b = fmax(b, __shfl_xor_sync(0xffffffffu, b, off));
    }
  }
}

// phi[i] = sum_d w_d psi[d][i] (d ascending, the order sn_moment uses); each block writes its
// (max |phi - phi_prev|, max |phi|) pair to scratch[2 blockIdx.x ..]: no accumulation, so
// nothing has to be cleared between calls.
__global__ void noalloc_moment_kernel(int n_dir, int64_t n, const double* __restrict__ w,
                                      const double* __restrict__ psi, const double* __restrict__ phi_prev,
                                      double* __restrict__ phi_out, double* scratch) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double diff = 0.0, mag = 0.0;
  if (i < n) {
    double phi = 0.0;
    for (int d = 0; d < n_dir; ++d) phi = fma(w[d], __ldg(psi + (int64_t)d * n + i), phi);
    phi_out[i] = phi;
    diff = fabs(phi - (phi_prev ? phi_prev[i] : 0.0));
    mag = fabs(phi);
  }
  block_max_pair(diff, mag);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = diff;
    scratch[2 * blockIdx.x + 1] = mag;
  }
}

// Reduce the per-block pairs into scratch[2 NOALLOC_MAX_BLOCKS ..] (overwritten every call).
__global__ void noalloc_finish_kernel(int nblocks, double* scratch) {
  double diff = 0.0, mag = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    diff = fmax(diff, scratch[2 * b]);
    mag = fmax(mag, scratch[2 * b + 1]);
  }
  block_max_pair(diff, mag);
  if (threadIdx.x == 0) {
    scratch[2 * NOALLOC_MAX_BLOCKS] = diff;
    scratch[2 * NOALLOC_MAX_BLOCKS + 1] = mag;
  }
}

// True for managed memory, or device memory that lives on `device` (a buffer on another GPU
// would be read without peer access by kernels launched on `device`).
bool on_device(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == device);
}

// Makes `device` current for the lifetime of the guard and gives the calling thread its
// previous current device back on every return path.
struct DeviceGuard {
  int prev = -1;
  cudaError_t set(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
    return cudaSetDevice(device);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Device address of the scratch array on `device` (which must be current); looked up on the
// first call for that device.
sn_status scratch_for(int device, double** out) {
  if (device < 0 || device >= NOALLOC_MAX_DEVICES) return SN_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[device]) {
    double* ptr = nullptr;
    if (cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return SN_ECUDA;
    }
    g_scratch_ptr[device] = ptr;
  }
  *out = g_scratch_ptr[device];
  return SN_OK;
}

}  // namespace
}  // namespace sn

extern "C" sn_status sn_moment_noalloc(int device, void* cuda_stream, int n_dir, int64_t n_elem, int n_dofs,
                                       const double* w, const double* psi, const double* phi_prev,
                                       double* phi_out, double* residual) {
  using namespace sn;
  if (n_dir < 1 || n_elem < 1 || n_dofs < 1) return SN_EINVAL;
  const int64_t n = n_elem * (int64_t)n_dofs;
  const int64_t blocks = (n + NOALLOC_THREADS - 1) / NOALLOC_THREADS;
  if (blocks > NOALLOC_MAX_BLOCKS) return SN_EINVAL;     // beyond the static scratch
  if (!w || !psi || !phi_out) return SN_EINVAL;
  DeviceGuard guard;
  if (guard.set(device) != cudaSuccess) {
    cudaGetLastError();
    return SN_ECUDA;
  }
  if (!on_device(w, device) || !on_device(psi, device) || !on_device(phi_out, device) ||
      (phi_prev && !on_device(phi_prev, device)))
    return SN_EINVAL;                                     // buffers of this device only: nothing is staged
  double* scratch = nullptr;
  sn_status st = scratch_for(device, &scratch);
  if (st != SN_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  noalloc_moment_kernel<<<(unsigned)blocks, NOALLOC_THREADS, 0, s>>>(n_dir, n, w, psi, phi_prev, phi_out, scratch);
  noalloc_finish_kernel<<<1, NOALLOC_THREADS, 0, s>>>((int)blocks, scratch);
  if (cudaGetLastError() != cudaSuccess) return SN_ECUDA;
  if (residual) {
    double pair[2];
    if (cudaMemcpyAsync(pair, scratch + 2 * NOALLOC_MAX_BLOCKS, sizeof(pair), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return SN_ECUDA;
    }
    *residual = pair[1] > 0.0 ? pair[0] / pair[1] : (pair[0] > 0.0 ? INFINITY : 0.0);
  }
  return SN_OK;
}
