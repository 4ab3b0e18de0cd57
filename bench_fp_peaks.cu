// FP64 / FP32 fused multiply-add throughput of one GPU: 8 independent FMA chains per thread,
// 16-way unrolled, on SMs x {4,8} blocks of 256 threads.  Used to measure the FP64 pipe peak
// that the sweep roofline is reported against (the measured peaks file has HBM and BF16 only).
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/fp_peaks bench_fp_peaks.cu && /tmp/fp_peaks
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_kernel(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <typename T>
void run(const char* name, int blocks, int threads, int iters) {
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for (int w = 0; w < 3; ++w) fma_kernel<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e0);
  fma_kernel<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1); cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
  printf("%s blocks=%d threads=%d iters=%d ms=%.3f TFLOP/s=%.3f err=%s\n", name, blocks, threads, iters, ms,
         flops / ms / 1e9, cudaGetErrorString(cudaGetLastError()));
  cudaFree(out);
}
int main() {
  int dev; cudaGetDevice(&dev); cudaDeviceProp p; cudaGetDeviceProperties(&p, dev);
  printf("%s SMs=%d cc=%d.%d l2=%d smem/blk optin=%zu regs/sm=%d\n", p.name, p.multiProcessorCount, p.major, p.minor,
         p.l2CacheSize, p.sharedMemPerBlockOptin, p.regsPerMultiprocessor);
  int sms = p.multiProcessorCount;
  run<double>("fp64", sms * 4, 256, 200);
  run<double>("fp64", sms * 8, 256, 200);
  run<float>("fp32", sms * 4, 256, 4000);
  run<float>("fp32", sms * 8, 256, 4000);
  return 0;
}
