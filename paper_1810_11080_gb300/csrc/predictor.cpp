// Learned flux predictor (C ABI, include/snsweep.h): the per-element MLP object with its
// training loop, the predictor data calls, and source iteration with a predicted initial
// scalar flux and a learned post-sweep correction.  Plain source iteration stays the arbiter:
// a correction is kept only if the next plain residual is below the one before it, and
// convergence is only declared on a step whose input came from a plain step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>
#include <cuda_runtime.h>
#include "mlp.h"

using namespace sn;

struct sn_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n_in = 0, n_out = 0;
  int64_t P = 0;
  int64_t off[6] = {0};
  float *theta = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* w16 = nullptr;
  int64_t cap = 0;                       // activation rows allocated
  float *x = nullptr, *h1 = nullptr, *h2 = nullptr, *y = nullptr, *dy = nullptr, *dh2 = nullptr, *dh1 = nullptr,
        *t = nullptr;
  double* loss = nullptr;
  int step = 0;
  std::string err;
};

namespace {

bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#define SM_CUDA(obj, call)                                              \
  do {                                                                  \
    cudaError_t _e = (call);                                            \
    if (_e != cudaSuccess) {                                            \
      (obj)->err = std::string(#call) + ": " + cudaGetErrorString(_e);  \
      return SN_ECUDA;                                                  \
    }                                                                   \
  } while (0)

sn_status mlp_reserve(sn_mlp* m, int64_t rows) {
  if (rows <= m->cap) return SN_OK;
  cudaFree(m->x);
  cudaFree(m->h1);
  cudaFree(m->h2);
  cudaFree(m->y);
  cudaFree(m->dy);
  cudaFree(m->dh2);
  cudaFree(m->dh1);
  cudaFree(m->t);
  const size_t H = MLP_HIDDEN;
  SM_CUDA(m, cudaMalloc((void**)&m->x, rows * m->n_in * sizeof(float)));
  SM_CUDA(m, cudaMalloc((void**)&m->h1, rows * H * sizeof(float)));
  SM_CUDA(m, cudaMalloc((void**)&m->h2, rows * H * sizeof(float)));
  SM_CUDA(m, cudaMalloc((void**)&m->y, rows * m->n_out * sizeof(float)));
  SM_CUDA(m, cudaMalloc((void**)&m->dy, rows * m->n_out * sizeof(float)));
  SM_CUDA(m, cudaMalloc((void**)&m->dh2, rows * H * sizeof(float)));
  SM_CUDA(m, cudaMalloc((void**)&m->dh1, rows * H * sizeof(float)));
  SM_CUDA(m, cudaMalloc((void**)&m->t, rows * m->n_out * sizeof(float)));
  m->cap = rows;
  return SN_OK;
}

cudaError_t fwd(sn_mlp* m, int64_t rows, const float* x, float* y) {
  const int H = MLP_HIDDEN;
  cudaError_t e = mlp_launch_fwd(rows, m->n_in, H, x, m->w16 + m->off[0], m->theta + m->off[1], m->h1, true, m->stream);
  if (e == cudaSuccess)
    e = mlp_launch_fwd(rows, H, H, m->h1, m->w16 + m->off[2], m->theta + m->off[3], m->h2, true, m->stream);
  if (e == cudaSuccess)
    e = mlp_launch_fwd(rows, H, m->n_out, m->h2, m->w16 + m->off[4], m->theta + m->off[5], y, false, m->stream);
  return e;
}

// Gradient of sum (y - t)^2 * scale / 2 over the rows, accumulated into m->g.
cudaError_t fwd_bwd(sn_mlp* m, int64_t rows, const float* x, const float* t, double scale) {
  const int H = MLP_HIDDEN;
  cudaError_t e = fwd(m, rows, x, m->y);
  if (e == cudaSuccess) e = mlp_launch_mse(rows * m->n_out, scale, m->y, t, m->dy, m->loss, m->stream);
  if (e == cudaSuccess)
    e = mlp_launch_bwd(rows, H, m->n_out, m->h2, m->w16 + m->off[4], m->y, m->dy, m->dh2, m->g + m->off[4],
                       m->g + m->off[5], false, m->stream);
  if (e == cudaSuccess)
    e = mlp_launch_bwd(rows, H, H, m->h1, m->w16 + m->off[2], m->h2, m->dh2, m->dh1, m->g + m->off[2],
                       m->g + m->off[3], true, m->stream);
  if (e == cudaSuccess)
    e = mlp_launch_bwd(rows, m->n_in, H, x, m->w16 + m->off[0], m->h1, m->dh1, nullptr, m->g + m->off[0],
                       m->g + m->off[1], true, m->stream);
  return e;
}

}  // namespace

namespace {
// Device copies (or in-place device pointers) of caller arrays; freed by the destructor.
struct Staged {
  std::vector<void*> own;
  ~Staged() {
    for (void* p : own) cudaFree(p);
  }
  template <class T>
  T* in(const T* p, size_t n, cudaStream_t s) {
    if (!p) return nullptr;
    if (dev_ptr(p)) return const_cast<T*>(p);
    T* d = nullptr;
    if (cudaMalloc((void**)&d, n * sizeof(T)) != cudaSuccess) return nullptr;
    own.push_back(d);
    cudaMemcpyAsync(d, p, n * sizeof(T), cudaMemcpyHostToDevice, s);
    return d;
  }
  template <class T>
  T* out(T* p, size_t n) {
    if (!p) return nullptr;
    if (dev_ptr(p)) return p;
    T* d = nullptr;
    if (cudaMalloc((void**)&d, n * sizeof(T)) != cudaSuccess) return nullptr;
    own.push_back(d);
    return d;
  }
};
}  // namespace

extern "C" {

sn_status sn_mlp_create(sn_mlp** out, int device, void* cuda_stream, int n_in, int n_out, uint64_t seed) {
  if (!out || n_in < 1 || n_in > MLP_MAXW || n_out < 1 || n_out > MLP_MAXW) return SN_EINVAL;
  *out = nullptr;
  sn_mlp* m = new (std::nothrow) sn_mlp();
  if (!m) return SN_ENOMEM;
  m->device = device;
  m->stream = (cudaStream_t)cuda_stream;
  m->n_in = n_in;
  m->n_out = n_out;
  const int64_t H = MLP_HIDDEN;
  const int64_t sz[6] = {n_in * H, H, H * H, H, H * n_out, n_out};
  int64_t o = 0;
  for (int k = 0; k < 6; ++k) {
    m->off[k] = o;
    o += sz[k];
  }
  m->P = o;
  // Glorot-uniform weights, zero biases, from a seeded mt19937_64
  std::vector<float> th(m->P, 0.0f);
  std::mt19937_64 rng(seed);
  const int fan[3][2] = {{n_in, (int)H}, {(int)H, (int)H}, {(int)H, n_out}};
  for (int l = 0; l < 3; ++l) {
    const double a = std::sqrt(6.0 / (fan[l][0] + fan[l][1]));
    std::uniform_real_distribution<double> U(-a, a);
    for (int64_t i = 0; i < sz[2 * l]; ++i) th[m->off[2 * l] + i] = (float)U(rng);
  }
  auto fail = [&]() {
    sn_mlp_destroy(m);
    return SN_ENOMEM;
  };
  if (cudaSetDevice(device) != cudaSuccess) {
    delete m;
    return SN_ECUDA;
  }
  if (cudaMalloc((void**)&m->theta, m->P * 4) || cudaMalloc((void**)&m->g, m->P * 4) ||
      cudaMalloc((void**)&m->m, m->P * 4) || cudaMalloc((void**)&m->v, m->P * 4) ||
      cudaMalloc((void**)&m->w16, m->P * 2) || cudaMalloc((void**)&m->loss, 8))
    return fail();
  cudaMemcpy(m->theta, th.data(), m->P * 4, cudaMemcpyHostToDevice);
  cudaMemset(m->m, 0, m->P * 4);
  cudaMemset(m->v, 0, m->P * 4);
  if (mlp_launch_to_bf16(m->P, m->theta, m->w16, m->stream) != cudaSuccess) return fail();
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return fail();
  *out = m;
  return SN_OK;
}

void sn_mlp_destroy(sn_mlp* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  if (m->stream) cudaStreamSynchronize(m->stream);
  for (float* p : {m->theta, m->g, m->m, m->v, m->x, m->h1, m->h2, m->y, m->dy, m->dh2, m->dh1, m->t}) cudaFree(p);
  cudaFree(m->w16);
  cudaFree(m->loss);
  delete m;
}

int64_t sn_mlp_num_params(const sn_mlp* m) { return m ? m->P : 0; }

sn_status sn_mlp_params(sn_mlp* m, float* get, const float* set) {
  if (!m) return SN_EINVAL;
  cudaSetDevice(m->device);
  if (set) {
    SM_CUDA(m, cudaMemcpyAsync(m->theta, set, m->P * 4, cudaMemcpyDefault, m->stream));
    SM_CUDA(m, mlp_launch_to_bf16(m->P, m->theta, m->w16, m->stream));
    SM_CUDA(m, cudaMemsetAsync(m->m, 0, m->P * 4, m->stream));
    SM_CUDA(m, cudaMemsetAsync(m->v, 0, m->P * 4, m->stream));
    m->step = 0;
  }
  if (get) SM_CUDA(m, cudaMemcpyAsync(get, m->theta, m->P * 4, cudaMemcpyDefault, m->stream));
  SM_CUDA(m, cudaStreamSynchronize(m->stream));
  return SN_OK;
}

sn_status sn_mlp_forward(sn_mlp* m, int64_t rows, const float* x, float* y) {
  if (!m || rows < 0 || !x || !y) return SN_EINVAL;
  cudaSetDevice(m->device);
  const int64_t CH = 65536;
  sn_status st = mlp_reserve(m, std::min(rows, CH));
  if (st != SN_OK) return st;
  const bool xd = dev_ptr(x), yd = dev_ptr(y);
  for (int64_t r0 = 0; r0 < rows; r0 += CH) {
    const int64_t n = std::min(CH, rows - r0);
    const float* xs = x + r0 * m->n_in;
    if (!xd) {
      SM_CUDA(m, cudaMemcpyAsync(m->x, xs, n * m->n_in * 4, cudaMemcpyHostToDevice, m->stream));
      xs = m->x;
    }
    float* ys = yd ? y + r0 * m->n_out : m->t;
    SM_CUDA(m, fwd(m, n, xs, ys));
    if (!yd) SM_CUDA(m, cudaMemcpyAsync(y + r0 * m->n_out, m->t, n * m->n_out * 4, cudaMemcpyDeviceToHost, m->stream));
  }
  SM_CUDA(m, cudaStreamSynchronize(m->stream));
  return SN_OK;
}

sn_status sn_mlp_grad(sn_mlp* m, int64_t rows, const float* x, const float* t, float* loss, float* grad) {
  if (!m || rows < 1 || !x || !t) return SN_EINVAL;
  cudaSetDevice(m->device);
  const int64_t CH = 65536;
  sn_status st = mlp_reserve(m, std::min(rows, CH));
  if (st != SN_OK) return st;
  const bool xd = dev_ptr(x), td = dev_ptr(t);
  SM_CUDA(m, cudaMemsetAsync(m->g, 0, m->P * 4, m->stream));
  SM_CUDA(m, cudaMemsetAsync(m->loss, 0, 8, m->stream));
  const double scale = 1.0 / ((double)rows * m->n_out);
  for (int64_t r0 = 0; r0 < rows; r0 += CH) {
    const int64_t n = std::min(CH, rows - r0);
    const float* xs = x + r0 * m->n_in;
    const float* ts = t + r0 * m->n_out;
    if (!xd) {
      SM_CUDA(m, cudaMemcpyAsync(m->x, xs, n * m->n_in * 4, cudaMemcpyHostToDevice, m->stream));
      xs = m->x;
    }
    if (!td) {
      SM_CUDA(m, cudaMemcpyAsync(m->t, ts, n * m->n_out * 4, cudaMemcpyHostToDevice, m->stream));
      ts = m->t;
    }
    SM_CUDA(m, fwd_bwd(m, n, xs, ts, scale));
  }
  double L = 0.0;
  SM_CUDA(m, cudaMemcpyAsync(&L, m->loss, 8, cudaMemcpyDeviceToHost, m->stream));
  if (grad) SM_CUDA(m, cudaMemcpyAsync(grad, m->g, m->P * 4, cudaMemcpyDefault, m->stream));
  SM_CUDA(m, cudaStreamSynchronize(m->stream));
  if (loss) *loss = (float)L;
  return SN_OK;
}

sn_status sn_mlp_train(sn_mlp* m, int64_t rows, const float* x, const float* t, int epochs, int batch_rows, float lr,
                       uint64_t seed, float* loss_out) {
  if (!m || rows < 1 || !x || !t || epochs < 1 || batch_rows < 1 || !(lr > 0.0f)) return SN_EINVAL;
  cudaSetDevice(m->device);
  const int64_t B = std::min<int64_t>(batch_rows, rows);
  sn_status st = mlp_reserve(m, B);
  if (st != SN_OK) return st;
  // whole data set on the device
  float *dx = const_cast<float*>(x), *dt = const_cast<float*>(t);
  bool own_x = false, own_t = false;
  if (!dev_ptr(x)) {
    SM_CUDA(m, cudaMalloc((void**)&dx, rows * m->n_in * 4));
    own_x = true;
    SM_CUDA(m, cudaMemcpyAsync(dx, x, rows * m->n_in * 4, cudaMemcpyHostToDevice, m->stream));
  }
  if (!dev_ptr(t)) {
    SM_CUDA(m, cudaMalloc((void**)&dt, rows * m->n_out * 4));
    own_t = true;
    SM_CUDA(m, cudaMemcpyAsync(dt, t, rows * m->n_out * 4, cudaMemcpyHostToDevice, m->stream));
  }
  const int64_t nb = (rows + B - 1) / B;
  std::vector<int64_t> order(nb);
  for (int64_t i = 0; i < nb; ++i) order[i] = i;
  std::mt19937_64 rng(seed);
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(order.begin(), order.end(), rng);
    SM_CUDA(m, cudaMemsetAsync(m->loss, 0, 8, m->stream));
    for (int64_t bi : order) {
      const int64_t r0 = bi * B, n = std::min(B, rows - r0);
      SM_CUDA(m, cudaMemsetAsync(m->g, 0, m->P * 4, m->stream));
      SM_CUDA(m, fwd_bwd(m, n, dx + r0 * m->n_in, dt + r0 * m->n_out, 1.0 / ((double)n * m->n_out)));
      SM_CUDA(m, mlp_launch_adam(m->P, lr, 0.9f, 0.999f, 1e-8f, ++m->step, m->theta, m->g, m->m, m->v, m->stream));
      SM_CUDA(m, mlp_launch_to_bf16(m->P, m->theta, m->w16, m->stream));
    }
    double L = 0.0;
    SM_CUDA(m, cudaMemcpyAsync(&L, m->loss, 8, cudaMemcpyDeviceToHost, m->stream));
    SM_CUDA(m, cudaStreamSynchronize(m->stream));
    last = L / nb;
  }
  if (own_x) cudaFree(dx);
  if (own_t) cudaFree(dt);
  if (loss_out) *loss_out = (float)last;
  return SN_OK;
}

// ------------------------------------------------------------------ predictor data
sn_status sn_predictor_features(sn_ctx* c, float* feat, double* phi_ref) {
  if (!c || !feat) return SN_EINVAL;
  if (!c->graph_ready) {
    c->err = "sn_build_graph first";
    return SN_ESTATE;
  }
  if (c->simplex) {
    c->err = "flux predictor: quadrilateral and hexahedral meshes only";
    return SN_EINVAL;
  }
  cudaSetDevice(c->device);
  float bb[6] = {1e30f, 1e30f, 1e30f, -1e30f, -1e30f, -1e30f};
  for (size_t i = 0; i < c->h_ctrl.size(); ++i) {
    const int k = (int)(i % c->dim);
    bb[k] = std::min(bb[k], (float)c->h_ctrl[i]);
    bb[3 + k] = std::max(bb[3 + k], (float)c->h_ctrl[i]);
  }
  for (int k = c->dim; k < 3; ++k) bb[k] = bb[3 + k] = 0.0f;
  float* df = feat;
  double* dr = phi_ref;
  const bool fdev = dev_ptr(feat), rdev = dev_ptr(phi_ref);
  if (!fdev && cudaMalloc((void**)&df, c->E * SN_FEATURES * 4) != cudaSuccess) return SN_ENOMEM;
  if (!rdev && cudaMalloc((void**)&dr, c->E * 8) != cudaSuccess) return SN_ENOMEM;
  cudaError_t e = launch_predictor_features(c->dev(), bb, df, dr, c->stream);
  if (e == cudaSuccess && !fdev) e = cudaMemcpyAsync(feat, df, c->E * SN_FEATURES * 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && phi_ref && !rdev) e = cudaMemcpyAsync(phi_ref, dr, c->E * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (!fdev) cudaFree(df);
  if (!rdev) cudaFree(dr);
  if (e != cudaSuccess) {
    c->err = cudaGetErrorString(e);
    return SN_ECUDA;
  }
  return SN_OK;
}


sn_status sn_predictor_init_targets(sn_ctx* c, const double* phi, float* target) {
  if (!c || !phi || !target) return SN_EINVAL;
  if (!c->graph_ready) return SN_ESTATE;
  cudaSetDevice(c->device);
  Staged S;
  const size_t EN = (size_t)c->E * c->N;
  float* df = nullptr;
  double* dref = nullptr;
  if (cudaMalloc((void**)&df, c->E * SN_FEATURES * 4) != cudaSuccess) return SN_ENOMEM;
  S.own.push_back(df);
  if (cudaMalloc((void**)&dref, c->E * 8) != cudaSuccess) return SN_ENOMEM;
  S.own.push_back(dref);
  sn_status st = sn_predictor_features(c, df, dref);
  if (st != SN_OK) return st;
  const double* dphi = S.in(phi, EN, c->stream);
  float* dt = S.out(target, EN);
  if (!dphi || !dt) return SN_ENOMEM;
  if (launch_predictor_scale(c->E, c->N, dref, dphi, dt, nullptr, nullptr, c->stream) != cudaSuccess) return SN_ECUDA;
  if (dt != target) cudaMemcpyAsync(target, dt, EN * 4, cudaMemcpyDeviceToHost, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SN_ECUDA;
  return SN_OK;
}

sn_status sn_predictor_corr_data(sn_ctx* c, const double* phi_a, const double* phi_b, const double* phi_c,
                                 const double* phi_inf, float* inputs, float* target) {
  if (!c || !phi_a || !phi_b || !phi_c || !inputs) return SN_EINVAL;
  if (!c->graph_ready) return SN_ESTATE;
  cudaSetDevice(c->device);
  Staged S;
  const size_t EN = (size_t)c->E * c->N;
  float* df = nullptr;
  if (cudaMalloc((void**)&df, c->E * SN_FEATURES * 4) != cudaSuccess) return SN_ENOMEM;
  S.own.push_back(df);
  double* dref = nullptr;
  if (cudaMalloc((void**)&dref, c->E * 8) != cudaSuccess) return SN_ENOMEM;
  S.own.push_back(dref);
  sn_status st = sn_predictor_features(c, df, dref);
  if (st != SN_OK) return st;
  const double *a = S.in(phi_a, EN, c->stream), *b = S.in(phi_b, EN, c->stream), *cc = S.in(phi_c, EN, c->stream);
  const double* inf = S.in(phi_inf, EN, c->stream);
  float* din = S.out(inputs, (size_t)c->E * (SN_FEATURES + 2));
  float* dt = S.out(target, (size_t)c->E);
  if (!a || !b || !cc || !din || (phi_inf && !inf) || (target && !dt)) return SN_ENOMEM;
  if (launch_predictor_corr_data(c->E, c->N, df, a, b, cc, inf, din, dt, c->stream) != cudaSuccess) return SN_ECUDA;
  if (din != inputs) cudaMemcpyAsync(inputs, din, (size_t)c->E * (SN_FEATURES + 2) * 4, cudaMemcpyDeviceToHost, c->stream);
  if (target && dt != target) cudaMemcpyAsync(target, dt, (size_t)c->E * 4, cudaMemcpyDeviceToHost, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SN_ECUDA;
  return SN_OK;
}

sn_status sn_predictor_initial_phi(sn_ctx* c, sn_mlp* init_model, const sn_predictor_cfg* cfg, double* phi0) {
  if (!c || !init_model || !cfg || !phi0) return SN_EINVAL;
  if (!c->graph_ready) return SN_ESTATE;
  if (init_model->n_in != SN_FEATURES || init_model->n_out != c->N) return SN_EINVAL;
  cudaSetDevice(c->device);
  const int64_t E = c->E;
  const size_t EN = (size_t)E * c->N;
  cudaStream_t s = c->stream;
  Staged S;
  float *feat = nullptr, *featn = nullptr, *y = nullptr, *norm = nullptr;
  double* ref = nullptr;
  auto al = [&](auto*& p, size_t n) {
    if (cudaMalloc((void**)&p, n * sizeof(*p)) != cudaSuccess) return false;
    S.own.push_back(p);
    return true;
  };
  if (!al(feat, E * SN_FEATURES) || !al(featn, E * SN_FEATURES) || !al(y, EN) || !al(norm, 2 * SN_FEATURES) ||
      !al(ref, E))
    return SN_ENOMEM;
  float hn[2 * SN_FEATURES];
  std::memcpy(hn, cfg->init_mean, sizeof(cfg->init_mean));
  std::memcpy(hn + SN_FEATURES, cfg->init_istd, sizeof(cfg->init_istd));
  if (cudaMemcpyAsync(norm, hn, sizeof(hn), cudaMemcpyHostToDevice, s) != cudaSuccess) return SN_ECUDA;
  sn_status st = sn_predictor_features(c, feat, ref);
  if (st != SN_OK) return st;
  if (launch_predictor_normalise(E, SN_FEATURES, feat, norm, norm + SN_FEATURES, featn, s) != cudaSuccess)
    return SN_ECUDA;
  init_model->stream = s;
  if ((st = sn_mlp_forward(init_model, E, featn, y)) != SN_OK) return st;
  double* dout = S.out(phi0, EN);
  if (!dout) return SN_ENOMEM;
  if (launch_predictor_scale(E, c->N, ref, nullptr, nullptr, y, dout, s) != cudaSuccess) return SN_ECUDA;
  if (dout != phi0) cudaMemcpyAsync(phi0, dout, EN * 8, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return SN_ECUDA;
  return SN_OK;
}

sn_status sn_source_iterate_learned(sn_ctx* c, double tol, int max_iter, int precision, sn_mlp* init_model,
                                    sn_mlp* corr_model, const sn_predictor_cfg* cfg, double* phi_out,
                                    sn_si_stats* stats, int32_t* n_accepted, int32_t* n_rejected) {
  if (!c || !cfg || max_iter < 1 || !(tol > 0.0)) return SN_EINVAL;
  if (!c->graph_ready) return SN_ESTATE;
  if (init_model && (init_model->n_in != SN_FEATURES || init_model->n_out != c->N)) return SN_EINVAL;
  if (corr_model && (corr_model->n_in != SN_FEATURES + 2 || corr_model->n_out != 1)) return SN_EINVAL;
  cudaSetDevice(c->device);
  auto t0 = std::chrono::steady_clock::now();
  const int64_t E = c->E;
  const size_t EN = (size_t)E * c->N;
  cudaStream_t s = c->stream;
  Staged S;
  float *feat = nullptr, *featn = nullptr, *y = nullptr, *cin = nullptr, *cinn = nullptr, *norm = nullptr;
  double *ref = nullptr, *phi0 = nullptr, *hin = nullptr, *hprev = nullptr;
  auto al = [&](auto*& p, size_t n) {
    if (cudaMalloc((void**)&p, n * sizeof(*p)) != cudaSuccess) return false;
    S.own.push_back(p);
    return true;
  };
  if (!al(feat, E * SN_FEATURES) || !al(featn, E * SN_FEATURES) || !al(y, EN) || !al(cin, E * (SN_FEATURES + 2)) ||
      !al(cinn, E * (SN_FEATURES + 2)) || !al(norm, 2 * (2 * SN_FEATURES + 2)) || !al(ref, E) || !al(phi0, EN) ||
      !al(hin, EN) || !al(hprev, EN))
    return SN_ENOMEM;
  float hn[2 * (2 * SN_FEATURES + 2)];
  std::memcpy(hn, cfg->init_mean, sizeof(cfg->init_mean));
  std::memcpy(hn + SN_FEATURES, cfg->init_istd, sizeof(cfg->init_istd));
  std::memcpy(hn + 2 * SN_FEATURES, cfg->corr_mean, sizeof(cfg->corr_mean));
  std::memcpy(hn + 3 * SN_FEATURES + 2, cfg->corr_istd, sizeof(cfg->corr_istd));
  if (cudaMemcpyAsync(norm, hn, sizeof(hn), cudaMemcpyHostToDevice, s) != cudaSuccess) return SN_ECUDA;
  sn_status st = sn_predictor_features(c, feat, ref);
  if (st != SN_OK) return st;
  const double* start = nullptr;
  if (init_model) {
    if (launch_predictor_normalise(E, SN_FEATURES, feat, norm, norm + SN_FEATURES, featn, s) != cudaSuccess)
      return SN_ECUDA;
    init_model->stream = s;
    if ((st = sn_mlp_forward(init_model, E, featn, y)) != SN_OK) return st;
    if (launch_predictor_scale(E, c->N, ref, nullptr, nullptr, y, phi0, s) != cudaSuccess) return SN_ECUDA;
    start = phi0;
  }
  if ((st = sn_si_begin(c, start)) != SN_OK) return st;
  if (corr_model) corr_model->stream = s;
  bool corr_on = corr_model != nullptr;
  bool corrected_last = false;
  double res = INFINITY, res_before = INFINITY;
  int acc = 0, rej = 0, it = 0;
  bool conv = false;
  for (it = 1; it <= max_iter; ++it) {
    std::swap(hprev, hin);
    if (cudaMemcpyAsync(hin, c->d_phi, EN * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return SN_ECUDA;
    if ((st = sn_si_step(c, precision, &res, nullptr)) != SN_OK) return st;
    if (corrected_last) {
      if (res < res_before) ++acc;
      else {
        ++rej;
        corr_on = false;           // fall back to plain source iteration
      }
      corrected_last = false;
      continue;                    // never declare convergence right after a correction
    }
    if (res < tol) {
      conv = true;
      break;
    }
    if (corr_on && it >= std::max(3, cfg->corr_start) && (it - cfg->corr_start) % std::max(1, cfg->corr_every) == 0) {
      if (launch_predictor_corr_data(E, c->N, feat, hprev, hin, c->d_phi, nullptr, cin, nullptr, s) != cudaSuccess)
        return SN_ECUDA;
      if (launch_predictor_normalise(E, SN_FEATURES + 2, cin, norm + 2 * SN_FEATURES, norm + 3 * SN_FEATURES + 2, cinn,
                                     s) != cudaSuccess)
        return SN_ECUDA;
      if ((st = sn_mlp_forward(corr_model, E, cinn, y)) != SN_OK) return st;
      if (launch_predictor_apply_corr(E, c->N, y, hin, c->d_phi, s) != cudaSuccess) return SN_ECUDA;
      if (launch_source(c->dev(), c->d_phi, c->d_src, c->d_srch, c->d_srcl, s) != cudaSuccess) return SN_ECUDA;
      c->launches += 4;
      res_before = res;
      corrected_last = true;
    }
  }
  if (it > max_iter) it = max_iter;
  if ((st = sn_si_result(c, phi_out, nullptr)) != SN_OK) return st;
  if (stats) {
    stats->iters = it;
    stats->converged = conv ? 1 : 0;
    stats->residual = res;
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (n_accepted) *n_accepted = acc;
  if (n_rejected) *n_rejected = rej;
  if (!conv) {
    c->err = "learned source iteration did not reach tol within max_iter";
    return SN_ENOTCONVERGED;
  }
  return SN_OK;
}

}  // extern "C"
