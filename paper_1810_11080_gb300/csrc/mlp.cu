// Learned flux predictor kernels (this project's addition; not in the paper):
//  - a per-element MLP x -> tanh(x W1 + b1) -> tanh(. W2 + b2) -> . W3 + b3 (width 64), weights
//    stored as BF16, all products accumulated in FP32, with forward, backward, MSE loss and Adam;
//  - per-element predictor data from a context: features (cross sections, source, geometry and
//    mesh-graph neighbour statistics), initial-guess targets, correction inputs and targets, and
//    the correction applied to the scalar flux.
// The GEMMs are rows x (n_in <= 64) x 64: a 48^3 mesh is ~1.5 GFLOP per inference, tens of
// microseconds on the FP32 pipe, so they run on CUDA cores with shared-memory tiles.
#include <cuda_bf16.h>
#include "devmath.cuh"
#include "mlp.h"

namespace sn {

namespace {
constexpr int RB = 32;          // rows per block
constexpr int TPB = 128;
}

// Y[r][j] = act(sum_i X[r][i] W[i][j] + b[j]), act = tanh if tanh_act.
__global__ void mlp_layer_fwd(int64_t rows, int n_in, int n_out, const float* __restrict__ X,
                              const __nv_bfloat16* __restrict__ W, const float* __restrict__ b, float* __restrict__ Y,
                              int tanh_act) {
  __shared__ float sW[MLP_MAXW * MLP_MAXW];
  __shared__ float sX[RB * MLP_MAXW];
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  for (int t = threadIdx.x; t < n_in * n_out; t += blockDim.x) sW[t] = __bfloat162float(W[t]);
  for (int t = threadIdx.x; t < RB * n_in; t += blockDim.x) {
    const int64_t r = r0 + t / n_in;
    sX[t] = r < rows ? X[r * n_in + t % n_in] : 0.0f;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < RB * n_out; t += blockDim.x) {
    const int rr = t / n_out, j = t % n_out;
    const int64_t r = r0 + rr;
    if (r >= rows) continue;
    float acc = b[j];
    for (int i = 0; i < n_in; ++i) acc = fmaf(sX[rr * n_in + i], sW[i * n_out + j], acc);
    Y[r * n_out + j] = tanh_act ? tanhf(acc) : acc;
  }
}

// Backward of one layer.  dY = dL/d(output after activation).  Accumulates dW, db into grad
// (FP32 atomics); writes dX (may be null for the first layer).
__global__ void mlp_layer_bwd(int64_t rows, int n_in, int n_out, const float* __restrict__ X,
                              const __nv_bfloat16* __restrict__ W, const float* __restrict__ Y,
                              const float* __restrict__ dY, float* __restrict__ dX, float* __restrict__ gW,
                              float* __restrict__ gb, int tanh_act) {
  __shared__ float sW[MLP_MAXW * MLP_MAXW];
  __shared__ float sX[RB * MLP_MAXW];
  __shared__ float sD[RB * MLP_MAXW];
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  for (int t = threadIdx.x; t < n_in * n_out; t += blockDim.x) sW[t] = __bfloat162float(W[t]);
  for (int t = threadIdx.x; t < RB * n_in; t += blockDim.x) {
    const int64_t r = r0 + t / n_in;
    sX[t] = r < rows ? X[r * n_in + t % n_in] : 0.0f;
  }
  for (int t = threadIdx.x; t < RB * n_out; t += blockDim.x) {
    const int64_t r = r0 + t / n_out;
    float dz = 0.0f;
    if (r < rows) {
      dz = dY[r * n_out + t % n_out];
      if (tanh_act) {
        const float y = Y[r * n_out + t % n_out];
        dz *= (1.0f - y * y);
      }
    }
    sD[t] = dz;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n_in * n_out; t += blockDim.x) {
    const int i = t / n_out, j = t % n_out;
    float acc = 0.0f;
    for (int rr = 0; rr < RB; ++rr) acc = fmaf(sX[rr * n_in + i], sD[rr * n_out + j], acc);
    atomicAdd(gW + t, acc);
  }
  for (int j = threadIdx.x; j < n_out; j += blockDim.x) {
    float acc = 0.0f;
    for (int rr = 0; rr < RB; ++rr) acc += sD[rr * n_out + j];
    atomicAdd(gb + j, acc);
  }
  if (dX != nullptr) {
    for (int t = threadIdx.x; t < RB * n_in; t += blockDim.x) {
      const int rr = t / n_in, i = t % n_in;
      const int64_t r = r0 + rr;
      if (r >= rows) continue;
      float acc = 0.0f;
      for (int j = 0; j < n_out; ++j) acc = fmaf(sD[rr * n_out + j], sW[i * n_out + j], acc);
      dX[r * n_in + i] = acc;
    }
  }
}

// dY = (y - t) / (rows n_out); loss += sum (y - t)^2 / (2 rows n_out) (FP64 accumulation).
__global__ void mlp_mse(int64_t n, double scale, const float* __restrict__ y, const float* __restrict__ t,
                        float* __restrict__ dy, double* loss) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float r = y[i] - t[i];
    dy[i] = (float)(r * scale);
    acc += 0.5 * (double)r * (double)r * scale;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// Adam on the FP32 master parameters; refresh the BF16 weight copies.
__global__ void mlp_adam(int64_t n, float lr, float b1, float b2, float eps, float c1, float c2,
                         float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                         float* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

__global__ void mlp_to_bf16(int64_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

cudaError_t mlp_launch_fwd(int64_t rows, int n_in, int n_out, const float* X, const __nv_bfloat16* W, const float* b,
                           float* Y, bool tanh_act, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  mlp_layer_fwd<<<(unsigned)((rows + RB - 1) / RB), TPB, 0, s>>>(rows, n_in, n_out, X, W, b, Y, tanh_act ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t mlp_launch_bwd(int64_t rows, int n_in, int n_out, const float* X, const __nv_bfloat16* W, const float* Y,
                           const float* dY, float* dX, float* gW, float* gb, bool tanh_act, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  mlp_layer_bwd<<<(unsigned)((rows + RB - 1) / RB), TPB, 0, s>>>(rows, n_in, n_out, X, W, Y, dY, dX, gW, gb,
                                                                 tanh_act ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t mlp_launch_mse(int64_t n, double scale, const float* y, const float* t, float* dy, double* loss,
                           cudaStream_t s) {
  mlp_mse<<<(unsigned)std::min<int64_t>(1216, (n + 255) / 256 + 1), 256, 0, s>>>(n, scale, y, t, dy, loss);
  return cudaGetLastError();
}

cudaError_t mlp_launch_adam(int64_t n, float lr, float b1, float b2, float eps, int step, float* theta, const float* g,
                            float* m, float* v, cudaStream_t s) {
  const float c1 = 1.0f / (1.0f - powf(b1, (float)step));
  const float c2 = 1.0f / (1.0f - powf(b2, (float)step));
  mlp_adam<<<(unsigned)std::min<int64_t>(1216, (n + 255) / 256 + 1), 256, 0, s>>>(n, lr, b1, b2, eps, c1, c2, theta, g,
                                                                                 m, v);
  return cudaGetLastError();
}

cudaError_t mlp_launch_to_bf16(int64_t n, const float* a, __nv_bfloat16* b, cudaStream_t s) {
  mlp_to_bf16<<<(unsigned)std::min<int64_t>(1216, (n + 255) / 256 + 1), 256, 0, s>>>(n, a, b);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ predictor data
// Per-element features (SN_FEATURES = 16):
//  0 sigma_t, 1 sigma_s, 2 sigma_a, 3 c = sigma_s/sigma_t, 4 mean nodal q, 5..7 mean control
//  point (x, y, z; 0 in 2D), 8 volume, 9 size h = volume^(1/dim), 10 distance of the mean
//  control point to the mesh bounding box, 11 boundary faces, 12 mean sigma_t over the faces
//  (0 across the boundary), 13 sigma_t h, 14 log sigma_t, 15 mean c over the faces.
// phi_ref = 4 pi max(mean q, 1e-12) / max(sigma_a, 1e-3 sigma_t) (infinite-medium scale).
__global__ void predictor_features(DevProblem P, float bb_lo0, float bb_lo1, float bb_lo2, float bb_hi0,
                                   float bb_hi1, float bb_hi2, float* __restrict__ feat, double* __restrict__ phi_ref) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= P.E) return;
  const int N = P.N, dim = P.dim, nfc = 2 * dim;
  const double st = P.sig_t[e], ss = P.sig_s[e], sa = st - ss;
  double qm = 0.0;
  for (int m = 0; m < N; ++m) qm += P.q[e * N + m];
  qm /= N;
  double c[3] = {0.0, 0.0, 0.0};
  for (int m = 0; m < P.Nv; ++m)
    for (int k = 0; k < dim; ++k) c[k] += P.ctrl[(e * P.Nv + m) * dim + k];
  for (int k = 0; k < dim; ++k) c[k] /= P.Nv;
  const double* Mm = P.elem + e * P.blk + (int64_t)dim * N * N;
  double vol = 0.0;
  for (int t = 0; t < N * N; ++t) vol += Mm[t];
  const double h = pow(vol, 1.0 / dim);
  const float lo[3] = {bb_lo0, bb_lo1, bb_lo2}, hi[3] = {bb_hi0, bb_hi1, bb_hi2};
  double dist = 1e30;
  for (int k = 0; k < dim; ++k) dist = fmin(dist, fmin(c[k] - lo[k], hi[k] - c[k]));
  int nb_bdr = 0;
  double nst = 0.0, nc = 0.0;
  for (int f = 0; f < nfc; ++f) {
    const int64_t nb = P.nbr[e * nfc + f];
    if (nb < 0) {
      ++nb_bdr;
      continue;
    }
    nst += P.sig_t[nb];
    nc += P.sig_s[nb] / P.sig_t[nb];
  }
  float* o = feat + e * SN_FEATURES;
  o[0] = (float)st;
  o[1] = (float)ss;
  o[2] = (float)sa;
  o[3] = (float)(ss / st);
  o[4] = (float)qm;
  o[5] = (float)c[0];
  o[6] = (float)c[1];
  o[7] = (float)c[2];
  o[8] = (float)vol;
  o[9] = (float)h;
  o[10] = (float)dist;
  o[11] = (float)nb_bdr;
  o[12] = (float)(nst / nfc);
  o[13] = (float)(st * h);
  o[14] = (float)log(st);
  o[15] = (float)(nc / nfc);
  phi_ref[e] = 4.0 * 3.14159265358979323846 * fmax(qm, 1e-12) / fmax(sa, 1e-3 * st);
}

// Initial-guess targets t[e][m] = phi[e][m] / phi_ref[e]; or the inverse (decode).
__global__ void predictor_scale(int64_t E, int N, const double* __restrict__ phi_ref, const double* __restrict__ phi,
                                float* __restrict__ t, const float* __restrict__ y, double* __restrict__ phi_out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= E * N) return;
  const int64_t e = i / N;
  if (t != nullptr) t[i] = (float)(phi[i] / phi_ref[e]);
  if (phi_out != nullptr) phi_out[i] = (double)y[i] * phi_ref[e];
}

// Correction data from three successive iterates phi_a (l-1), phi_b (l), phi_c (l+1):
// inputs[e] = (normalised features ..., rho = |c - b| / |b - a|, log10(|c - b| / |c|)) and, when
// phi_inf is given, target[e] = log1p(clip(<phi_inf - c, c - b> / <c - b, c - b>, 0, 500)).
__global__ void predictor_corr_data(int64_t E, int N, const float* __restrict__ featn, const double* __restrict__ pa,
                                    const double* __restrict__ pb, const double* __restrict__ pc,
                                    const double* __restrict__ pinf, float* __restrict__ inputs,
                                    float* __restrict__ target) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  double n1 = 0.0, n0 = 0.0, nc = 0.0, num = 0.0;
  for (int m = 0; m < N; ++m) {
    const int64_t i = e * N + m;
    const double d1 = pc[i] - pb[i], d0 = pb[i] - pa[i];
    n1 += d1 * d1;
    n0 += d0 * d0;
    nc += pc[i] * pc[i];
    if (pinf) num += (pinf[i] - pc[i]) * d1;
  }
  float* o = inputs + e * (SN_FEATURES + 2);
  for (int k = 0; k < SN_FEATURES; ++k) o[k] = featn[e * SN_FEATURES + k];
  o[SN_FEATURES] = (float)fmin(sqrt(n1 / fmax(n0, 1e-300)), 10.0);
  o[SN_FEATURES + 1] = (float)log10(sqrt(n1 / fmax(nc, 1e-300)) + 1e-30);
  if (target != nullptr) {
    const double g = n1 > 0.0 ? num / n1 : 0.0;
    target[e] = (float)log1p(fmin(fmax(g, 0.0), 500.0));
  }
}

// phi_c += expm1(clip(y)) (phi_c - phi_b), element by element.
__global__ void predictor_apply_corr(int64_t E, int N, const float* __restrict__ y, const double* __restrict__ pb,
                                    double* __restrict__ pc) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= E * N) return;
  const double g = expm1(fmin(fmax((double)y[i / N], 0.0), 6.0));
  pc[i] = pc[i] + g * (pc[i] - pb[i]);
}

// Feature normalisation x' = (x - mean) * istd.
__global__ void predictor_normalise(int64_t rows, int n, const float* __restrict__ x, const float* __restrict__ mean,
                                    const float* __restrict__ istd, float* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= rows * n) return;
  const int k = (int)(i % n);
  out[i] = (x[i] - mean[k]) * istd[k];
}

cudaError_t launch_predictor_features(const DevProblem& P, const float* bb, float* feat, double* phi_ref,
                                      cudaStream_t s) {
  predictor_features<<<(unsigned)((P.E + 127) / 128), 128, 0, s>>>(P, bb[0], bb[1], bb[2], bb[3], bb[4], bb[5], feat,
                                                                     phi_ref);
  return cudaGetLastError();
}
cudaError_t launch_predictor_scale(int64_t E, int N, const double* phi_ref, const double* phi, float* t, const float* y,
                                   double* phi_out, cudaStream_t s) {
  predictor_scale<<<(unsigned)((E * N + 255) / 256), 256, 0, s>>>(E, N, phi_ref, phi, t, y, phi_out);
  return cudaGetLastError();
}
cudaError_t launch_predictor_corr_data(int64_t E, int N, const float* featn, const double* pa, const double* pb,
                                       const double* pc, const double* pinf, float* inputs, float* target,
                                       cudaStream_t s) {
  predictor_corr_data<<<(unsigned)((E + 127) / 128), 128, 0, s>>>(E, N, featn, pa, pb, pc, pinf, inputs, target);
  return cudaGetLastError();
}
cudaError_t launch_predictor_apply_corr(int64_t E, int N, const float* y, const double* pb, double* pc, cudaStream_t s) {
  predictor_apply_corr<<<(unsigned)((E * N + 255) / 256), 256, 0, s>>>(E, N, y, pb, pc);
  return cudaGetLastError();
}
cudaError_t launch_predictor_normalise(int64_t rows, int n, const float* x, const float* mean, const float* istd,
                                       float* out, cudaStream_t s) {
  predictor_normalise<<<(unsigned)((rows * n + 255) / 256), 256, 0, s>>>(rows, n, x, mean, istd, out);
  return cudaGetLastError();
}

}  // namespace sn
