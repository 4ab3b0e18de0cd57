// Batched source iteration over many independent problems (C ABI, include/snsweep.h): one
// persistent dataflow launch (or one launch per level) sweeps every problem, one kernel forms
// every problem's scalar flux, scattering source and residual; the step is captured as a CUDA
// graph.  Each problem keeps its own sn_ctx (factors, graph, flux buffers).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>
#include <cuda_runtime.h>
#include "common.h"

using namespace sn;

struct sn_batch {
  int n = 0;
  int device = 0;
  int dim = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  std::vector<sn_ctx*> ctx;
  std::vector<double*> phiA, phiB;
  int launch_mode = SN_LAUNCH_DATAFLOW;
  int blocks_per_sm = 0;
  int parity = 0;
  bool ready = false;
  int64_t updates = 0;
  // device tables
  DevProblem* d_probs = nullptr;
  SweepArgs* d_args[2] = {nullptr, nullptr};
  MomentArgs* d_margs[2] = {nullptr, nullptr};
  int4* d_tasks = nullptr;
  int64_t ntasks = 0;
  std::vector<int64_t> level_task_off;
  int64_t* d_block_off = nullptr;
  int64_t moment_blocks = 0;
  int* d_done = nullptr;
  size_t done_total = 0;
  unsigned long long* d_red = nullptr;   // [2n] residual maxima, [2n] error word, [2n+1] queue head
  std::vector<unsigned long long> h_red;
  std::map<int, cudaGraphExec_t> graphs;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::vector<SweepArgs> h_args[2];     // host copies of the argument tables
  bool inv_linked = false;              // d_args carry every problem's stored inverses
};

namespace {

#define SB_CUDA(b, call)                                                \
  do {                                                                  \
    cudaError_t _e = (call);                                            \
    if (_e != cudaSuccess) {                                            \
      (b)->err = std::string(#call) + ": " + cudaGetErrorString(_e);    \
      return SN_ECUDA;                                                  \
    }                                                                   \
  } while (0)

#define SB_REQ(b, cond, st, msg) \
  do {                           \
    if (!(cond)) {               \
      (b)->err = msg;            \
      return st;                 \
    }                            \
  } while (0)

void free_graphs(sn_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

// Sweep + moment of one step, enqueued on the batch stream (captured by the caller).
cudaError_t enqueue_step(sn_batch* b, int prec) {
  const int p = b->parity;
  int* errw = reinterpret_cast<int*>(b->d_red + 2 * b->n);
  unsigned long long* head = b->d_red + 2 * b->n + 1;
  cudaError_t e = cudaMemsetAsync(b->d_red, 0, (2 * (size_t)b->n + 2) * sizeof(unsigned long long), b->stream);
  if (e != cudaSuccess) return e;
  if (b->launch_mode == SN_LAUNCH_DATAFLOW) {
    e = cudaMemsetAsync(b->d_done, 0, b->done_total * sizeof(int), b->stream);
    if (e != cudaSuccess) return e;
    e = launch_batch_sweep(b->dim, prec, true, b->d_probs, b->d_args[p], b->d_tasks, b->ntasks, head, errw,
                           b->blocks_per_sm, b->stream);
  } else {
    for (size_t L = 0; L + 1 < b->level_task_off.size(); ++L) {
      const int64_t o = b->level_task_off[L], c = b->level_task_off[L + 1] - o;
      e = launch_batch_sweep(b->dim, prec, false, b->d_probs, b->d_args[p], b->d_tasks + o, c, head, errw, 0,
                             b->stream);
      if (e != cudaSuccess) return e;
    }
  }
  if (e != cudaSuccess) return e;
  return launch_batch_moment(b->d_probs, b->d_margs[p], b->d_block_off, b->n, b->moment_blocks, b->d_red, b->stream);
}

}  // namespace

extern "C" {

sn_status sn_batch_create(sn_batch** out, int n_problems, sn_ctx* const* problems, void* cuda_stream) {
  if (!out || n_problems < 1 || !problems) return SN_EINVAL;
  *out = nullptr;
  sn_batch* b = new (std::nothrow) sn_batch();
  if (!b) return SN_ENOMEM;
  auto fail = [&](sn_status st) {
    sn_batch_destroy(b);
    return st;
  };
  b->n = n_problems;
  b->stream = (cudaStream_t)cuda_stream;
  for (int k = 0; k < n_problems; ++k) {
    sn_ctx* c = problems[k];
    if (!c || !c->graph_ready) return fail(SN_ESTATE);
    if (c->simplex) return fail(SN_EINVAL);         // batches: quadrilateral and hexahedral problems
    if (k == 0) {
      b->device = c->device;
      b->dim = c->dim;
    }
    if (c->device != b->device || c->dim != b->dim) return fail(SN_EINVAL);
    b->ctx.push_back(c);
  }
  if (cudaSetDevice(b->device) != cudaSuccess) return fail(SN_ECUDA);
  const int n = n_problems;
  std::vector<DevProblem> probs(n);
  std::vector<SweepArgs> args0(n), args1(n);
  std::vector<MomentArgs> m0(n), m1(n);
  std::vector<int64_t> done_off(n + 1, 0), block_off(n + 1, 0);
  for (int k = 0; k < n; ++k) {
    sn_ctx* c = b->ctx[k];
    probs[k] = c->dev();
    done_off[k + 1] = done_off[k] + (int64_t)c->M * c->E;
    const int epb = 256 / c->N;
    block_off[k + 1] = block_off[k] + (c->E + epb - 1) / epb;
    b->phiA.push_back(c->d_phi);
    b->phiB.push_back(c->d_phi2);
    b->updates += (int64_t)c->M * c->E;
  }
  b->done_total = (size_t)done_off[n];
  b->moment_blocks = block_off[n];
  if (cudaMalloc((void**)&b->d_done, b->done_total * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&b->d_red, (2 * (size_t)n + 2) * sizeof(unsigned long long)) != cudaSuccess)
    return fail(SN_ENOMEM);
  int* errw = reinterpret_cast<int*>(b->d_red + 2 * n);
  for (int k = 0; k < n; ++k) {
    sn_ctx* c = b->ctx[k];
    SweepArgs base{c->d_facecode, c->d_mixed_off, c->d_mixedB, c->d_mixedB32, c->d_mixedB32lo, c->d_src,
                   nullptr, nullptr, b->d_done + done_off[k], errw, c->d_pairs,
                   c->d_srch, c->d_srcl, nullptr, nullptr, nullptr, nullptr, c->spin_limit};
    args0[k] = base;
    args0[k].psi_old = c->d_psi[0];
    args0[k].psi_new = c->d_psi[1];
    args0[k].psi_old_h = c->d_psih[0];
    args0[k].psi_old_l = c->d_psil[0];
    args0[k].psi_new_h = c->d_psih[1];
    args0[k].psi_new_l = c->d_psil[1];
    args1[k] = base;
    args1[k].psi_old = c->d_psi[1];
    args1[k].psi_new = c->d_psi[0];
    args1[k].psi_old_h = c->d_psih[1];
    args1[k].psi_old_l = c->d_psil[1];
    args1[k].psi_new_h = c->d_psih[0];
    args1[k].psi_new_l = c->d_psil[0];
    args0[k].inv = args1[k].inv = nullptr;
    args0[k].fblk = args1[k].fblk = nullptr;
    args0[k].fidx = args1[k].fidx = nullptr;
    m0[k] = MomentArgs{c->d_psi[1], b->phiA[k], b->phiB[k], c->d_src, c->d_srch, c->d_srcl};
    m1[k] = MomentArgs{c->d_psi[0], b->phiB[k], b->phiA[k], c->d_src, c->d_srch, c->d_srcl};
  }
  // tasks ordered by level across problems; each problem's levels are padded to its 32/W
  int Lmax = 0;
  for (auto* c : b->ctx) Lmax = std::max<int>(Lmax, (int)c->level_off.size() - 1);
  std::vector<int4> tasks;
  b->level_task_off.assign(1, 0);
  for (int L = 0; L < Lmax; ++L) {
    for (int k = 0; k < n; ++k) {
      sn_ctx* c = b->ctx[k];
      if (L + 1 >= (int)c->level_off.size()) continue;
      const int W = c->N <= 4 ? 4 : c->N <= 8 ? 8 : c->N <= 16 ? 16 : 32;
      const int spw = 32 / W;
      for (int64_t o = c->level_off[L]; o < c->level_off[L + 1]; o += spw) tasks.push_back(make_int4(k, c->p, (int)o, 0));
    }
    b->level_task_off.push_back((int64_t)tasks.size());
  }
  b->ntasks = (int64_t)tasks.size();
  auto up = [&](auto*& dst, const auto& v) -> bool {
    using T = typename std::remove_reference<decltype(v)>::type::value_type;
    if (cudaMalloc((void**)&dst, std::max<size_t>(1, v.size()) * sizeof(T)) != cudaSuccess) return false;
    return cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
  };
  if (!up(b->d_probs, probs) || !up(b->d_args[0], args0) || !up(b->d_args[1], args1) || !up(b->d_margs[0], m0) ||
      !up(b->d_margs[1], m1) || !up(b->d_tasks, tasks) || !up(b->d_block_off, block_off))
    return fail(SN_ENOMEM);
  if (cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess) return fail(SN_ECUDA);
  b->h_red.assign(2 * (size_t)n + 2, 0);
  b->h_args[0] = args0;
  b->h_args[1] = args1;
  *out = b;
  return SN_OK;
}

void sn_batch_destroy(sn_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_graphs(b);
  cudaFree(b->d_probs);
  cudaFree(b->d_args[0]);
  cudaFree(b->d_args[1]);
  cudaFree(b->d_margs[0]);
  cudaFree(b->d_margs[1]);
  cudaFree(b->d_tasks);
  cudaFree(b->d_block_off);
  cudaFree(b->d_done);
  cudaFree(b->d_red);
  if (b->ev[0]) cudaEventDestroy(b->ev[0]);
  if (b->ev[1]) cudaEventDestroy(b->ev[1]);
  delete b;
}

const char* sn_batch_last_error(const sn_batch* b) { return b ? b->err.c_str() : "null batch"; }

int64_t sn_batch_updates_per_sweep(const sn_batch* b) { return b ? b->updates : 0; }

sn_status sn_batch_set_launch(sn_batch* b, int mode, int blocks_per_sm) {
  if (!b) return SN_EINVAL;
  SB_REQ(b, mode == SN_LAUNCH_LEVELS || mode == SN_LAUNCH_DATAFLOW, SN_EINVAL, "unknown launch mode");
  SB_REQ(b, blocks_per_sm >= 0 && blocks_per_sm <= 64, SN_EINVAL, "blocks_per_sm must be 0..64");
  b->launch_mode = mode;
  b->blocks_per_sm = blocks_per_sm;
  free_graphs(b);
  return SN_OK;
}

sn_status sn_batch_si_begin(sn_batch* b, const double* const* phi0) {
  if (!b) return SN_EINVAL;
  SB_CUDA(b, cudaSetDevice(b->device));
  for (int k = 0; k < b->n; ++k) {
    sn_ctx* c = b->ctx[k];
    const size_t npsi = (size_t)c->M * c->E * c->N, nphi = (size_t)c->E * c->N;
    SB_CUDA(b, cudaMemsetAsync(c->d_psi[0], 0, npsi * 8, b->stream));
    SB_CUDA(b, cudaMemsetAsync(c->d_psih[0], 0, npsi * 4, b->stream));
    SB_CUDA(b, cudaMemsetAsync(c->d_psil[0], 0, npsi * 4, b->stream));
    if (phi0 && phi0[k])
      SB_CUDA(b, cudaMemcpyAsync(b->phiA[k], phi0[k], nphi * 8, cudaMemcpyDefault, b->stream));
    else
      SB_CUDA(b, cudaMemsetAsync(b->phiA[k], 0, nphi * 8, b->stream));
    DevProblem P = c->dev();
    SB_CUDA(b, launch_source(P, b->phiA[k], c->d_src, c->d_srch, c->d_srcl, b->stream));
    c->d_phi = b->phiA[k];
    c->d_phi2 = b->phiB[k];
    c->si_cur = 0;
    c->si_ready = true;
  }
  SB_CUDA(b, cudaStreamSynchronize(b->stream));
  b->parity = 0;
  b->ready = true;
  return SN_OK;
}

sn_status sn_batch_si_step(sn_batch* b, int precision, double* residuals, float* ms_sweep) {
  if (!b) return SN_EINVAL;
  SB_REQ(b, b->ready, SN_ESTATE, "sn_batch_si_begin first");
  SB_REQ(b, precision >= SN_PREC_FP64 && precision <= SN_PREC_DS_INV, SN_EINVAL, "unknown precision");
  SB_CUDA(b, cudaSetDevice(b->device));
  if (precision == SN_PREC_FP64_INV || precision == SN_PREC_DS_INV) {
    // every problem's stored inverses formed (once), and their addresses in the argument tables
    bool moved = !b->inv_linked;
    for (int k = 0; k < b->n; ++k) {
      sn_ctx* c = b->ctx[k];
      if (c->inv_form != precision) {
        sn_status st = sn_prepare_inverse(c, precision, nullptr);
        if (st != SN_OK) {
          b->err = std::string("problem ") + std::to_string(k) + ": " + c->err;
          return st;
        }
      }
      if (b->h_args[0][k].inv != c->d_inv || b->h_args[0][k].fblk != c->d_fblk) moved = true;
      for (int q = 0; q < 2; ++q) {
        b->h_args[q][k].inv = c->d_inv;
        b->h_args[q][k].fblk = c->d_fblk;
        b->h_args[q][k].fidx = c->d_fidx;
      }
    }
    if (moved) {
      SB_CUDA(b, cudaStreamSynchronize(b->stream));
      for (int q = 0; q < 2; ++q)
        SB_CUDA(b, cudaMemcpy(b->d_args[q], b->h_args[q].data(), b->h_args[q].size() * sizeof(SweepArgs),
                              cudaMemcpyHostToDevice));
      b->inv_linked = true;
    }
  }
  const int key = precision * 16 + b->launch_mode * 2 + b->parity;
  if (ms_sweep) SB_CUDA(b, cudaEventRecord(b->ev[0], b->stream));
  if (b->stream == nullptr) {
    SB_CUDA(b, enqueue_step(b, precision));
  } else {
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
      cudaGraph_t g;
      SB_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t le = enqueue_step(b, precision);
      cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
      SB_CUDA(b, le);
      SB_CUDA(b, ee);
      cudaGraphExec_t ge;
      cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      SB_CUDA(b, ie);
      it = b->graphs.emplace(key, ge).first;
    }
    SB_CUDA(b, cudaGraphLaunch(it->second, b->stream));
  }
  if (ms_sweep) SB_CUDA(b, cudaEventRecord(b->ev[1], b->stream));
  for (auto* c : b->ctx) c->launches += (b->launch_mode == SN_LAUNCH_DATAFLOW ? 1 : 0);
  SB_CUDA(b, cudaMemcpyAsync(b->h_red.data(), b->d_red, b->h_red.size() * 8, cudaMemcpyDeviceToHost, b->stream));
  SB_CUDA(b, cudaStreamSynchronize(b->stream));
  if (ms_sweep) SB_CUDA(b, cudaEventElapsedTime(ms_sweep, b->ev[0], b->ev[1]));
  const int p = b->parity;
  for (int k = 0; k < b->n; ++k) {
    sn_ctx* c = b->ctx[k];
    c->si_cur = p ^ 1;
    c->d_phi = (p == 0) ? b->phiB[k] : b->phiA[k];
    c->d_phi2 = (p == 0) ? b->phiA[k] : b->phiB[k];
    if (residuals) {
      double diff, mag;
      std::memcpy(&diff, &b->h_red[2 * k], 8);
      std::memcpy(&mag, &b->h_red[2 * k + 1], 8);
      residuals[k] = mag > 0.0 ? diff / mag : (diff > 0.0 ? INFINITY : 0.0);
    }
  }
  b->parity ^= 1;
  if (b->h_red[2 * b->n] & 0xffffffffull) {
    b->err = "batched dataflow sweep: a dependency wait exceeded its spin limit";
    return SN_ETIMEOUT;
  }
  return SN_OK;
}

sn_status sn_batch_source_iterate(sn_batch* b, double tol, int max_iter, int precision, int32_t* iters,
                                  double* residuals, double* ms_total) {
  if (!b) return SN_EINVAL;
  SB_REQ(b, tol > 0.0 && max_iter >= 1, SN_EINVAL, "tol > 0 and max_iter >= 1 required");
  auto t0 = std::chrono::steady_clock::now();
  sn_status st = sn_batch_si_begin(b, nullptr);
  if (st != SN_OK) return st;
  std::vector<double> res(b->n, INFINITY);
  std::vector<int32_t> it_conv(b->n, -1);
  int left = b->n;
  for (int it = 1; it <= max_iter && left > 0; ++it) {
    if ((st = sn_batch_si_step(b, precision, res.data(), nullptr)) != SN_OK) return st;
    for (int k = 0; k < b->n; ++k)
      if (it_conv[k] < 0 && res[k] < tol) {
        it_conv[k] = it;
        --left;
      }
  }
  if (iters) std::memcpy(iters, it_conv.data(), sizeof(int32_t) * b->n);
  if (residuals) std::memcpy(residuals, res.data(), sizeof(double) * b->n);
  if (ms_total) *ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (left > 0) {
    b->err = "batched source iteration: some problems did not reach tol within max_iter";
    return SN_ENOTCONVERGED;
  }
  return SN_OK;
}

// Autotuner: times the sweep of each schedule / CTAs-per-SM candidate over three steps and keeps
// the fastest (SI state is reset afterwards).
sn_status sn_batch_tune(sn_batch* b, int precision, int* mode_out, int* blocks_per_sm_out) {
  if (!b) return SN_EINVAL;
  const int cand[6][2] = {{SN_LAUNCH_LEVELS, 0}, {SN_LAUNCH_DATAFLOW, 1}, {SN_LAUNCH_DATAFLOW, 2},
                          {SN_LAUNCH_DATAFLOW, 3}, {SN_LAUNCH_DATAFLOW, 4}, {SN_LAUNCH_DATAFLOW, 0}};
  float best = 1e30f;
  int bm = SN_LAUNCH_DATAFLOW, bb = 0;
  for (auto& cd : cand) {
    sn_status st = sn_batch_set_launch(b, cd[0], cd[1]);
    if (st != SN_OK) return st;
    if ((st = sn_batch_si_begin(b, nullptr)) != SN_OK) return st;
    if ((st = sn_batch_si_step(b, precision, nullptr, nullptr)) != SN_OK) return st;
    if ((st = sn_batch_si_step(b, precision, nullptr, nullptr)) != SN_OK) return st;
    float tot = 1e30f;                   // fastest of 5 steps
    for (int r = 0; r < 5; ++r) {
      float ms = 0.0f;
      if ((st = sn_batch_si_step(b, precision, nullptr, &ms)) != SN_OK) return st;
      tot = std::min(tot, ms);
    }
    if (tot < best) {
      best = tot;
      bm = cd[0];
      bb = cd[1];
    }
  }
  sn_status st = sn_batch_set_launch(b, bm, bb);
  if (st != SN_OK) return st;
  if ((st = sn_batch_si_begin(b, nullptr)) != SN_OK) return st;
  if (mode_out) *mode_out = bm;
  if (blocks_per_sm_out) *blocks_per_sm_out = bb;
  return SN_OK;
}

}  // extern "C"
