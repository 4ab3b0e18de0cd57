// Internal declarations of the learned-predictor kernels (mlp.cu) and the MLP object.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include "common.h"

#ifndef SN_FEATURES
#define SN_FEATURES 16
#endif
#define MLP_HIDDEN 64
#define MLP_MAXW 64      // max layer width (inputs and outputs)

namespace sn {
cudaError_t mlp_launch_fwd(int64_t rows, int n_in, int n_out, const float* X, const __nv_bfloat16* W, const float* b,
                           float* Y, bool tanh_act, cudaStream_t s);
cudaError_t mlp_launch_bwd(int64_t rows, int n_in, int n_out, const float* X, const __nv_bfloat16* W, const float* Y,
                           const float* dY, float* dX, float* gW, float* gb, bool tanh_act, cudaStream_t s);
cudaError_t mlp_launch_mse(int64_t n, double scale, const float* y, const float* t, float* dy, double* loss,
                           cudaStream_t s);
cudaError_t mlp_launch_adam(int64_t n, float lr, float b1, float b2, float eps, int step, float* theta, const float* g,
                            float* m, float* v, cudaStream_t s);
cudaError_t mlp_launch_to_bf16(int64_t n, const float* a, __nv_bfloat16* b, cudaStream_t s);
cudaError_t launch_predictor_features(const DevProblem& P, const float* bb, float* feat, double* phi_ref,
                                      cudaStream_t s);
cudaError_t launch_predictor_scale(int64_t E, int N, const double* phi_ref, const double* phi, float* t, const float* y,
                                   double* phi_out, cudaStream_t s);
cudaError_t launch_predictor_corr_data(int64_t E, int N, const float* featn, const double* pa, const double* pb,
                                       const double* pc, const double* pinf, float* inputs, float* target,
                                       cudaStream_t s);
cudaError_t launch_predictor_apply_corr(int64_t E, int N, const float* y, const double* pb, double* pc, cudaStream_t s);
cudaError_t launch_predictor_normalise(int64_t rows, int n, const float* x, const float* mean, const float* istd,
                                       float* out, cudaStream_t s);
}  // namespace sn
