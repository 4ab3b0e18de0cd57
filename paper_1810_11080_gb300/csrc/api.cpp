// C ABI of the snsweep library (declared in include/snsweep.h): context, problem upload,
// graph build (device weights -> host SCC/FAS -> device levels), sweeps and source iteration.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <cuda_runtime.h>
#include "common.h"

using namespace sn;

namespace {

struct Fail {
  sn_status st;
};

void set_err(sn_ctx* c, const std::string& m) {
  if (c) c->err = m;
}

#define SN_CUDA(ctx, call)                                                                      \
  do {                                                                                          \
    cudaError_t _e = (call);                                                                    \
    if (_e != cudaSuccess) {                                                                    \
      set_err(ctx, std::string(#call) + ": " + cudaGetErrorString(_e));                         \
      return SN_ECUDA;                                                                          \
    }                                                                                           \
  } while (0)

#define SN_REQ(ctx, cond, st, msg) \
  do {                             \
    if (!(cond)) {                 \
      set_err(ctx, msg);           \
      return st;                   \
    }                              \
  } while (0)

template <class T>
cudaError_t dalloc(T*& p, size_t n) {
  if (p) {
    cudaFree(p);
    p = nullptr;
  }
  if (n == 0) return cudaSuccess;
  return cudaMalloc((void**)&p, n * sizeof(T));
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void free_dsa(sn_ctx* c) {
  sn::DsaState& D = c->dsa;
  for (double** p : {&D.diag, &D.inv, &D.selfb, &D.offb, &D.vol, &D.b, &D.x, &D.r, &D.z, &D.p, &D.q, &D.sc}) dfree(*p);
  dfree(D.bad);
  D.ready = false;
}

// The captured sweep graphs hold the record addresses in their kernel arguments: every graph is
// dropped whenever the records are freed (and, in form_inverse, before they are allocated).
void drop_graphs(sn_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
}

void free_inverse(sn_ctx* c) {
  if (c->d_inv || c->d_fblk || c->d_fidx) drop_graphs(c);
  dfree(c->d_inv);
  dfree(c->d_fblk);
  dfree(c->d_fidx);
  c->inv_form = -1;
}

void free_graph_state(sn_ctx* c) {
  free_dsa(c);
  free_inverse(c);
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  dfree(c->d_facecode);
  dfree(c->d_mixed_off);
  dfree(c->d_mixedB);
  dfree(c->d_mixedB32);
  dfree(c->d_mixedB32lo);
  dfree(c->d_levels);
  dfree(c->d_pairs);
  dfree(c->d_elem);
  dfree(c->d_elem32);
  dfree(c->d_elem32lo);
  c->graph_ready = false;
  c->si_ready = false;
  for (auto& p : c->d_psi) dfree(p);
  dfree(c->d_phi);
  dfree(c->d_phi2);
  dfree(c->d_src);
  dfree(c->d_done);
  for (auto& p : c->d_stage) dfree(p);
  for (int k = 0; k < 2; ++k) {
    dfree(c->d_psih[k]);
    dfree(c->d_psil[k]);
    dfree(c->d_scr_h[k]);
    dfree(c->d_scr_l[k]);
  }
  dfree(c->d_srch);
  dfree(c->d_srcl);
  dfree(c->d_om32);
  dfree(c->d_st32);
  c->level_off.clear();
  c->h_removed.clear();
  c->n_removed = 0;
}

}  // namespace

sn::DevProblem sn_ctx::dev() const {
  DevProblem P{};
  P.dim = dim;
  P.r = r;
  P.p = p;
  P.N = N;
  P.Nf = Nf;
  P.nv = tab.nv;
  P.nf = tab.nf;
  P.K = (dim == 3 && !simplex) ? K : 1;
  P.Q = tab.Q;
  P.Nv = tab.Nv;
  P.nfc = nfc;
  P.simplex = simplex ? 1 : 0;
  P.M = M;
  P.E = E;
  P.n_bdr = n_bdr;
  P.ctrl = d_ctrl;
  P.nbr = d_nbr;
  P.nbr_face = d_nbr_face;
  P.orient = d_orient;
  P.bdr_index = d_bdr_index;
  P.omega = d_omega;
  P.w = d_w;
  P.sig_t = d_sig_t;
  P.sig_s = d_sig_s;
  P.q = d_q;
  P.q_dir = d_qdir;
  P.psi_inc = d_psi_inc;
  P.tab = d_tab;
  P.off_glv_t = tab_off[0];
  P.off_glv_w = tab_off[1];
  P.off_glf_t = tab_off[2];
  P.off_glf_w = tab_off[3];
  P.off_gll = tab_off[4];
  P.off_geo = tab_off[5];
  P.off_wq = tab_off[6];
  P.off_B = tab_off[7];
  P.off_dB = tab_off[8];
  P.off_dV = tab_off[9];
  P.off_V = tab_off[10];
  P.elem = d_elem;
  P.blk = blk;
  P.elem32 = d_elem32;
  P.elem32lo = d_elem32lo;
  P.om32 = d_om32;
  P.st32 = d_st32;
  return P;
}

extern "C" {

sn_status sn_create(sn_ctx** out, int device, void* cuda_stream) {
  if (!out) return SN_EINVAL;
  *out = nullptr;
  sn_ctx* c = new (std::nothrow) sn_ctx();
  if (!c) return SN_ENOMEM;
  c->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete c;
    return SN_ECUDA;
  }
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaMalloc((void**)&c->d_red, 4 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc((void**)&c->d_flag, 4 * sizeof(int)) != cudaSuccess) {
    cudaFree(c->d_red);
    delete c;
    return SN_ENOMEM;
  }
  *out = c;
  return SN_OK;
}

void sn_destroy(sn_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_graph_state(c);
  dfree(c->d_ctrl);
  dfree(c->d_omega);
  dfree(c->d_w);
  dfree(c->d_tab);
  dfree(c->d_nbr);
  dfree(c->d_bdr_index);
  dfree(c->d_nbr_face);
  dfree(c->d_orient);
  dfree(c->d_iface);
  dfree(c->d_bface);
  dfree(c->d_sig_t);
  dfree(c->d_sig_s);
  dfree(c->d_q);
  dfree(c->d_qdir);
  dfree(c->d_psi_inc);
  for (auto& p : c->d_psi) dfree(p);
  dfree(c->d_phi);
  dfree(c->d_phi2);
  dfree(c->d_src);
  dfree(c->d_done);
  for (auto& p : c->d_stage) dfree(p);
  dfree(c->d_red);
  dfree(c->d_flag);
  if (c->ev_a) cudaEventDestroy(c->ev_a);
  if (c->ev_b) cudaEventDestroy(c->ev_b);
  delete c;
}

const char* sn_last_error(const sn_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t sn_kernel_launches(const sn_ctx* c) { return c ? c->launches : 0; }

int64_t sn_num_boundary_faces(const sn_ctx* c) { return c ? c->n_bdr : 0; }

namespace {
sn_status set_mesh_impl(sn_ctx* c, int dim, int64_t n_elem, int r, const double* ctrl, const int64_t* face_nbr,
                        const int32_t* nbr_face, const int32_t* orient, bool simplex) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, dim == 2 || dim == 3, SN_EINVAL, "dim must be 2 or 3");
  SN_REQ(c, !simplex || dim == 2 || r == 1, SN_EINVAL, "tetrahedra: straight-sided (geometry order r = 1) only");
  SN_REQ(c, r >= 1 && r <= MAX_R, SN_EINVAL, "geometry order r must be 1..3");
  SN_REQ(c, n_elem >= 1 && n_elem < (1LL << 31) / 8, SN_EINVAL, "n_elem out of range");
  SN_REQ(c, ctrl && face_nbr && nbr_face && orient, SN_EINVAL, "null mesh array");
  cudaSetDevice(c->device);
  const int nfc = simplex ? dim + 1 : 2 * dim;
  int64_t nv = 1;
  if (simplex) nv = dim == 2 ? (int64_t)(r + 1) * (r + 2) / 2 : 4;
  else
    for (int k = 0; k < dim; ++k) nv *= (r + 1);
  std::vector<double> hc(n_elem * nv * dim);
  std::vector<int64_t> hn(n_elem * nfc);
  std::vector<int32_t> hf(n_elem * nfc), ho(n_elem * nfc);
  auto fetch = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (is_device_ptr(src)) return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
    std::memcpy(dst, src, bytes);
    return cudaSuccess;
  };
  SN_CUDA(c, fetch(hc.data(), ctrl, hc.size() * sizeof(double)));
  SN_CUDA(c, fetch(hn.data(), face_nbr, hn.size() * sizeof(int64_t)));
  SN_CUDA(c, fetch(hf.data(), nbr_face, hf.size() * sizeof(int32_t)));
  SN_CUDA(c, fetch(ho.data(), orient, ho.size() * sizeof(int32_t)));
  for (double v : hc) SN_REQ(c, std::isfinite(v), SN_EINVAL, "non-finite control point");
  // symmetric neighbour relation
  for (int64_t e = 0; e < n_elem; ++e)
    for (int f = 0; f < nfc; ++f) {
      int64_t nb = hn[e * nfc + f];
      if (nb < 0) continue;
      SN_REQ(c, nb < n_elem && nb != e, SN_EMESH, "face neighbour out of range");
      int fn = hf[e * nfc + f];
      SN_REQ(c, fn >= 0 && fn < nfc, SN_EMESH, "neighbour face out of range");
      SN_REQ(c, hn[nb * nfc + fn] == e && hf[nb * nfc + fn] == f, SN_EMESH, "neighbour relation not symmetric");
      int oc = ho[e * nfc + f];
      SN_REQ(c, oc >= 0 && oc < (dim == 2 ? 2 : (simplex ? 6 : 8)), SN_EINVAL, "orientation code out of range");
    }
  free_graph_state(c);
  c->dim = dim;
  c->r = r;
  c->simplex = simplex;
  c->nfc = nfc;
  c->E = n_elem;
  c->h_ctrl.swap(hc);
  c->h_nbr.swap(hn);
  c->h_nbr_face.swap(hf);
  c->h_orient.swap(ho);
  c->h_bdr_index.assign(n_elem * nfc, -1);
  c->h_iface.clear();
  c->h_bface.clear();
  c->n_bdr = 0;
  for (int64_t e = 0; e < n_elem; ++e)
    for (int f = 0; f < nfc; ++f) {
      int64_t nb = c->h_nbr[e * nfc + f];
      if (nb < 0) {
        c->h_bdr_index[e * nfc + f] = c->n_bdr++;
        c->h_bface.push_back((int32_t)e);
        c->h_bface.push_back(f);
      } else if (e < nb) {
        c->h_iface.insert(c->h_iface.end(),
                          {(int32_t)e, f, (int32_t)nb, c->h_nbr_face[e * nfc + f], c->h_orient[e * nfc + f]});
      }
    }
  SN_CUDA(c, dalloc(c->d_ctrl, c->h_ctrl.size()));
  SN_CUDA(c, dalloc(c->d_nbr, c->h_nbr.size()));
  SN_CUDA(c, dalloc(c->d_nbr_face, c->h_nbr_face.size()));
  SN_CUDA(c, dalloc(c->d_orient, c->h_orient.size()));
  SN_CUDA(c, dalloc(c->d_bdr_index, c->h_bdr_index.size()));
  SN_CUDA(c, dalloc(c->d_iface, std::max<size_t>(1, c->h_iface.size())));
  SN_CUDA(c, dalloc(c->d_bface, std::max<size_t>(1, c->h_bface.size())));
  SN_CUDA(c, cudaMemcpy(c->d_ctrl, c->h_ctrl.data(), c->h_ctrl.size() * 8, cudaMemcpyHostToDevice));
  SN_CUDA(c, cudaMemcpy(c->d_nbr, c->h_nbr.data(), c->h_nbr.size() * 8, cudaMemcpyHostToDevice));
  SN_CUDA(c, cudaMemcpy(c->d_nbr_face, c->h_nbr_face.data(), c->h_nbr_face.size() * 4, cudaMemcpyHostToDevice));
  SN_CUDA(c, cudaMemcpy(c->d_orient, c->h_orient.data(), c->h_orient.size() * 4, cudaMemcpyHostToDevice));
  SN_CUDA(c, cudaMemcpy(c->d_bdr_index, c->h_bdr_index.data(), c->h_bdr_index.size() * 8, cudaMemcpyHostToDevice));
  if (!c->h_iface.empty())
    SN_CUDA(c, cudaMemcpy(c->d_iface, c->h_iface.data(), c->h_iface.size() * 4, cudaMemcpyHostToDevice));
  if (!c->h_bface.empty())
    SN_CUDA(c, cudaMemcpy(c->d_bface, c->h_bface.data(), c->h_bface.size() * 4, cudaMemcpyHostToDevice));
  c->mesh_set = true;
  c->disc_set = false;
  c->mat_set = false;
  return SN_OK;
}
}  // namespace

sn_status sn_set_mesh(sn_ctx* c, int dim, int64_t n_elem, int r, const double* ctrl, const int64_t* face_nbr,
                      const int32_t* nbr_face, const int32_t* orient) {
  return set_mesh_impl(c, dim, n_elem, r, ctrl, face_nbr, nbr_face, orient, false);
}

sn_status sn_set_mesh_simplex(sn_ctx* c, int dim, int64_t n_elem, int r, const double* ctrl,
                              const int64_t* face_nbr, const int32_t* nbr_face, const int32_t* orient) {
  return set_mesh_impl(c, dim, n_elem, r, ctrl, face_nbr, nbr_face, orient, true);
}

sn_status sn_set_discretization(sn_ctx* c, int p, int face_subdiv) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->mesh_set, SN_ESTATE, "sn_set_mesh first");
  SN_REQ(c, p >= 1 && p <= MAX_P, SN_EINVAL, "DG order p must be 1..3");
  SN_REQ(c, c->dim == 2 || p <= 2, SN_EINVAL, "3D DG order p must be 1 or 2 ((p+1)^3 <= 32 unknowns per element)");
  SN_REQ(c, face_subdiv >= 1 && face_subdiv <= 4, SN_EINVAL, "face_subdiv must be 1..4");
  if (c->dim == 3 && !c->simplex) {
    const int nf = p + c->r;
    SN_REQ(c, face_subdiv * face_subdiv * nf * nf <= 256, SN_EINVAL, "3D face rule too large (K^2 n_f^2 > 256)");
  }
  cudaSetDevice(c->device);
  free_graph_state(c);
  c->p = p;
  c->K = face_subdiv;
  try {
    if (c->simplex && c->dim == 3) build_tables_tet(c->tab, p);
    else if (c->simplex) build_tables_tri(c->tab, p, c->r);
    else build_tables(c->tab, c->dim, p, c->r);
  } catch (const std::exception& ex) {
    set_err(c, ex.what());
    return SN_EINVAL;
  }
  c->N = c->tab.N;
  c->Nf = c->tab.Nf;
  c->blk = elem_block_doubles(c->dim, c->N, c->Nf, c->nfc);
  std::vector<double> packed;
  auto add = [&](int slot, const std::vector<double>& v) {
    c->tab_off[slot] = (int)packed.size();
    packed.insert(packed.end(), v.begin(), v.end());
    while (packed.size() % 2) packed.push_back(0.0);
  };
  add(0, c->tab.glv_t);
  add(1, c->tab.glv_w);
  add(2, c->tab.glf_t);
  add(3, c->tab.glf_w);
  add(4, c->tab.gll);
  add(5, c->tab.geo);
  add(6, c->tab.wq);
  add(7, c->tab.B);
  add(8, c->tab.dB);
  add(9, c->tab.dV);
  add(10, c->tab.V);
  SN_CUDA(c, dalloc(c->d_tab, packed.size()));
  SN_CUDA(c, cudaMemcpy(c->d_tab, packed.data(), packed.size() * 8, cudaMemcpyHostToDevice));
  c->disc_set = true;
  c->mat_set = false;
  return SN_OK;
}

sn_status sn_set_quadrature(sn_ctx* c, int n_dir, const double* omega, const double* w) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, n_dir >= 1 && n_dir <= 4096, SN_EINVAL, "n_dir must be 1..4096");
  SN_REQ(c, omega && w, SN_EINVAL, "null quadrature array");
  cudaSetDevice(c->device);
  std::vector<double> ho(n_dir * 3), hw(n_dir);
  if (is_device_ptr(omega)) SN_CUDA(c, cudaMemcpy(ho.data(), omega, ho.size() * 8, cudaMemcpyDeviceToHost));
  else std::memcpy(ho.data(), omega, ho.size() * 8);
  if (is_device_ptr(w)) SN_CUDA(c, cudaMemcpy(hw.data(), w, hw.size() * 8, cudaMemcpyDeviceToHost));
  else std::memcpy(hw.data(), w, hw.size() * 8);
  for (int d = 0; d < n_dir; ++d) {
    SN_REQ(c, std::isfinite(hw[d]) && hw[d] > 0.0, SN_EINVAL, "quadrature weights must be positive");
    for (int k = 0; k < 3; ++k) SN_REQ(c, std::isfinite(ho[d * 3 + k]), SN_EINVAL, "non-finite direction");
  }
  free_graph_state(c);
  c->M = n_dir;
  c->h_omega.swap(ho);
  c->h_w.swap(hw);
  SN_CUDA(c, dalloc(c->d_omega, c->h_omega.size()));
  SN_CUDA(c, dalloc(c->d_w, c->h_w.size()));
  SN_CUDA(c, cudaMemcpy(c->d_omega, c->h_omega.data(), c->h_omega.size() * 8, cudaMemcpyHostToDevice));
  SN_CUDA(c, cudaMemcpy(c->d_w, c->h_w.data(), c->h_w.size() * 8, cudaMemcpyHostToDevice));
  c->quad_set = true;
  c->mat_set = false;
  return SN_OK;
}

namespace {
// Host copy of a caller array (host or device pointer), checked: finite, and for cross sections
// > 0 (or >= 0 with allow_zero).
sn_status fetch_checked(sn_ctx* c, std::vector<double>& h, const double* src, size_t n, bool check_pos,
                        bool allow_zero) {
  h.resize(n);
  if (is_device_ptr(src)) SN_CUDA(c, cudaMemcpy(h.data(), src, n * 8, cudaMemcpyDeviceToHost));
  else std::memcpy(h.data(), src, n * 8);
  for (double v : h) {
    SN_REQ(c, std::isfinite(v), SN_EINVAL, "non-finite material or source value");
    if (check_pos) SN_REQ(c, allow_zero ? v >= 0.0 : v > 0.0, SN_EINVAL, "cross section out of range");
  }
  return SN_OK;
}
sn_status upload(sn_ctx* c, double*& dst, const std::vector<double>& h) {
  SN_CUDA(c, dalloc(dst, h.size()));
  SN_CUDA(c, cudaMemcpy(dst, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
  return SN_OK;
}
}  // namespace

sn_status sn_set_materials(sn_ctx* c, const double* sigma_t, const double* sigma_s, const double* q,
                           const double* q_dir, const double* psi_inc) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->mesh_set && c->disc_set && c->quad_set, SN_ESTATE, "mesh, discretization and quadrature first");
  SN_REQ(c, sigma_t && sigma_s, SN_EINVAL, "null cross sections");
  cudaSetDevice(c->device);
  // every array is checked before anything is replaced: a rejected call changes nothing
  std::vector<double> ht, hs, hq, hqd, hpi;
  sn_status st;
  if ((st = fetch_checked(c, ht, sigma_t, c->E, true, false)) != SN_OK) return st;
  if ((st = fetch_checked(c, hs, sigma_s, c->E, true, true)) != SN_OK) return st;
  if (q) {
    if ((st = fetch_checked(c, hq, q, (size_t)c->E * c->N, false, false)) != SN_OK) return st;
  } else {
    hq.assign((size_t)c->E * c->N, 0.0);
  }
  if (q_dir && (st = fetch_checked(c, hqd, q_dir, (size_t)c->M * c->E * c->N, false, false)) != SN_OK) return st;
  const bool has_inc = psi_inc && c->n_bdr > 0;
  if (has_inc && (st = fetch_checked(c, hpi, psi_inc, (size_t)c->M * c->n_bdr * c->Nf, false, false)) != SN_OK)
    return st;
  // sigma_t enters the graph (siginvface weights): rebuild it
  if (c->graph_ready) free_graph_state(c);
  c->mat_set = false;
  if ((st = upload(c, c->d_sig_t, ht)) != SN_OK) return st;
  if ((st = upload(c, c->d_sig_s, hs)) != SN_OK) return st;
  if ((st = upload(c, c->d_q, hq)) != SN_OK) return st;
  dfree(c->d_qdir);
  dfree(c->d_psi_inc);
  if (q_dir && (st = upload(c, c->d_qdir, hqd)) != SN_OK) return st;
  if (has_inc && (st = upload(c, c->d_psi_inc, hpi)) != SN_OK) return st;
  c->mat_set = true;
  return SN_OK;
}

namespace {

sn_status ensure_buffers(sn_ctx* c) {
  const size_t npsi = (size_t)c->M * c->E * c->N, nphi = (size_t)c->E * c->N;
  for (auto& p : c->d_psi)
    if (!p) SN_CUDA(c, dalloc(p, npsi));
  if (!c->d_phi) SN_CUDA(c, dalloc(c->d_phi, nphi));
  if (!c->d_phi2) SN_CUDA(c, dalloc(c->d_phi2, nphi));
  if (!c->d_src) SN_CUDA(c, dalloc(c->d_src, nphi));
  if (!c->d_done) SN_CUDA(c, dalloc(c->d_done, (size_t)c->M * c->E));
  for (int k = 0; k < 2; ++k) {
    if (!c->d_psih[k]) SN_CUDA(c, dalloc(c->d_psih[k], npsi));
    if (!c->d_psil[k]) SN_CUDA(c, dalloc(c->d_psil[k], npsi));
  }
  if (!c->d_srch) SN_CUDA(c, dalloc(c->d_srch, nphi));
  if (!c->d_srcl) SN_CUDA(c, dalloc(c->d_srcl, nphi));
  return SN_OK;
}

sn_status ensure_stage(sn_ctx* c, int slot) {
  if (!c->d_stage[slot]) SN_CUDA(c, dalloc(c->d_stage[slot], (size_t)c->M * c->E * c->N));
  return SN_OK;
}

}  // namespace

sn_status sn_build_graph(sn_ctx* c, int weighting, int exact_max, sn_graph_stats* stats) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->mat_set, SN_ESTATE, "sn_set_materials first");
  SN_REQ(c, weighting >= 0 && weighting <= 2, SN_EINVAL, "weighting must be 0, 1 or 2");
  SN_REQ(c, exact_max >= 1 && exact_max <= 16, SN_EINVAL, "exact_max must be 1..16");
  cudaSetDevice(c->device);
  free_graph_state(c);
  cudaStream_t s = c->stream;
  sn_graph_stats gs{};
  cudaEvent_t ev[5];
  for (auto& x : ev) SN_CUDA(c, cudaEventCreate(&x));
  const int64_t E = c->E, M = c->M;
  const int nfc = c->nfc;
  // geometric factors
  SN_CUDA(c, dalloc(c->d_elem, (size_t)E * c->blk));
  SN_CUDA(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
  SN_CUDA(c, cudaEventRecord(ev[0], s));
  DevProblem P = c->dev();
  SN_CUDA(c, launch_geometry(P, c->d_elem, c->d_flag, s));
  c->launches++;
  SN_CUDA(c, dalloc(c->d_elem32, (size_t)E * c->blk));
  SN_CUDA(c, dalloc(c->d_elem32lo, (size_t)E * c->blk));
  P = c->dev();
  SN_CUDA(c, launch_elem_to_fp32(P, c->d_elem32, c->d_elem32lo, s));
  c->launches++;
  SN_CUDA(c, cudaEventRecord(ev[1], s));
  int bad = 0;
  SN_CUDA(c, cudaMemcpyAsync(&bad, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  SN_CUDA(c, cudaStreamSynchronize(s));
  if (bad) {
    set_err(c, "invalid mesh: det J <= 0 at a volume quadrature point");
    free_graph_state(c);
    return SN_EMESH;
  }
  // edge weights and face modes
  const int64_t nI = (int64_t)c->h_iface.size() / 5, nB = (int64_t)c->h_bface.size() / 2;
  double *d_win = nullptr, *d_lu = nullptr;
  int32_t* d_perm = nullptr;
  SN_CUDA(c, dalloc(c->d_facecode, (size_t)M * E));
  SN_CUDA(c, cudaMemsetAsync(c->d_facecode, 0, (size_t)M * E * 4, s));
  SN_CUDA(c, dalloc(d_win, (size_t)M * E * nfc));
  if (weighting == SN_WEIGHT_SIGINVFACE) {
    SN_CUDA(c, dalloc(d_lu, (size_t)E * c->N * c->N));
    SN_CUDA(c, dalloc(d_perm, (size_t)E * c->N));
    SN_CUDA(c, launch_mass_lu(P, d_lu, d_perm, s));
    c->launches++;
  }
  SN_CUDA(c, launch_weights(P, c->d_iface, nI, weighting, d_lu, d_perm, d_win, c->d_facecode, s));
  SN_CUDA(c, launch_bdr_modes(P, c->d_bface, nB, c->d_facecode, s));
  c->launches += 2;
  SN_CUDA(c, cudaEventRecord(ev[2], s));
  // components and feedback arc sets of every direction's graph (device); lag bits into facecode
  SN_CUDA(c, cudaEventSynchronize(ev[2]));
  auto t0 = std::chrono::steady_clock::now();
  DeviceFasStats fs;
  {
    cudaError_t fe = device_fas(P, c->d_facecode, d_win, exact_max, &fs, s);
    dfree(d_win);
    dfree(d_lu);
    dfree(d_perm);
    if (fs.stuck) {
      set_err(c, "graph components: a fixed-point iteration did not settle");
      free_graph_state(c);
      return SN_ESTATE;
    }
    SN_CUDA(c, fe);
  }
  c->launches += fs.launches;
  gs.ms_fas = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  gs.n_scc = fs.n_scc;
  gs.max_scc = fs.max_scc;
  std::vector<uint32_t> fc((size_t)M * E);
  SN_CUDA(c, cudaMemcpyAsync(fc.data(), c->d_facecode, fc.size() * 4, cudaMemcpyDeviceToHost, s));
  SN_CUDA(c, cudaStreamSynchronize(s));
  // arcs and removed (lagged) arcs from the face codes: (d, e, e') rows sorted ascending
  c->h_removed.clear();
  for (int64_t d = 0; d < M; ++d)
    for (int64_t e = 0; e < E; ++e) {
      const uint32_t code = fc[d * E + e];
      std::pair<int32_t, int32_t> rr[6];
      int nr = 0;
      for (int f = 0; f < nfc; ++f) {
        const int64_t nb = c->h_nbr[e * nfc + f];
        if (nb < 0 || face_mode(code, f) == MODE_NONE) continue;
        gs.n_arcs++;
        if (face_lagged(code, f)) rr[nr++] = {(int32_t)e, (int32_t)nb};
      }
      std::sort(rr, rr + nr);
      for (int k = 0; k < nr; ++k) c->h_removed.insert(c->h_removed.end(), {(int32_t)d, rr[k].first, rr[k].second});
    }
  c->n_removed = (int64_t)c->h_removed.size() / 3;
  gs.n_removed = c->n_removed;
  if (c->n_removed != fs.n_removed) {
    set_err(c, "graph components: removed-arc count mismatch");
    free_graph_state(c);
    return SN_ESTATE;
  }
  // levels (device) and work lists
  SN_CUDA(c, cudaEventRecord(ev[3], s));
  SN_CUDA(c, dalloc(c->d_levels, (size_t)M * E));
  SN_CUDA(c, launch_levels_init(P, c->d_levels, s));
  c->launches++;
  int64_t rounds = 0;
  while (true) {
    SN_CUDA(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
    for (int k = 0; k < 8; ++k) {
      SN_CUDA(c, launch_levels_relax(P, c->d_facecode, c->d_levels, c->d_flag, s));
      c->launches++;
    }
    int changed = 0;
    SN_CUDA(c, cudaMemcpyAsync(&changed, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    SN_CUDA(c, cudaStreamSynchronize(s));
    rounds += 8;
    if (!changed) break;
    if (rounds > E + 16) {
      set_err(c, "level scheduling did not converge: kept graph is cyclic");
      free_graph_state(c);
      return SN_ESTATE;
    }
  }
  std::vector<int32_t> lv((size_t)M * E);
  SN_CUDA(c, cudaMemcpyAsync(lv.data(), c->d_levels, lv.size() * 4, cudaMemcpyDeviceToHost, s));
  SN_CUDA(c, cudaStreamSynchronize(s));
  int32_t Lmax = 0;
  for (int32_t v : lv) Lmax = std::max(Lmax, v);
  // Work list: pairs e*M+d sorted by (level, e, d); every level padded with -1 entries to a
  // multiple of the systems per warp, so that no warp ever holds pairs of two levels (a pair
  // may depend on the previous level; a warp must never wait on itself).
  const int W = c->N <= 4 ? 4 : c->N <= 8 ? 8 : c->N <= 16 ? 16 : 32;
  const int spw = 32 / W;
  std::vector<int64_t> cnt(Lmax + 1, 0);
  for (int32_t v : lv) cnt[v]++;
  c->level_off.assign(Lmax + 2, 0);
  for (int32_t L = 0; L <= Lmax; ++L) c->level_off[L + 1] = c->level_off[L] + (cnt[L] + spw - 1) / spw * spw;
  std::vector<int32_t> pairs((size_t)c->level_off.back(), -1);
  {
    std::vector<int64_t> pos(c->level_off.begin(), c->level_off.end() - 1);
    for (int64_t e = 0; e < E; ++e)
      for (int64_t d = 0; d < M; ++d) pairs[pos[lv[d * E + e]]++] = (int32_t)(e * M + d);
  }
  SN_CUDA(c, dalloc(c->d_pairs, pairs.size()));
  SN_CUDA(c, cudaMemcpyAsync(c->d_pairs, pairs.data(), pairs.size() * 4, cudaMemcpyHostToDevice, s));
  c->h_pairs = pairs;
  // partially-inflow blocks
  std::vector<int32_t> moff((size_t)M * E);
  int64_t nm = 0;
  for (size_t k = 0; k < fc.size(); ++k) {
    moff[k] = (int32_t)nm;
    for (int f = 0; f < nfc; ++f) nm += (face_mode(fc[k], f) == MODE_MIXED);
  }
  c->n_mixed = nm;
  SN_CUDA(c, dalloc(c->d_mixed_off, moff.size()));
  SN_CUDA(c, cudaMemcpyAsync(c->d_mixed_off, moff.data(), moff.size() * 4, cudaMemcpyHostToDevice, s));
  SN_CUDA(c, dalloc(c->d_mixedB, (size_t)std::max<int64_t>(1, nm) * c->Nf * c->Nf));
  SN_CUDA(c, dalloc(c->d_mixedB32, (size_t)std::max<int64_t>(1, nm) * c->Nf * c->Nf));
  SN_CUDA(c, dalloc(c->d_mixedB32lo, (size_t)std::max<int64_t>(1, nm) * c->Nf * c->Nf));
  if (nm > 0) {
    SN_CUDA(c, launch_mixed_blocks(P, c->d_iface, nI, c->d_bface, nB, c->d_facecode, c->d_mixed_off, c->d_mixedB,
                                   c->d_mixedB32, c->d_mixedB32lo, s));
    c->launches++;
  }
  SN_CUDA(c, cudaEventRecord(ev[4], s));
  SN_CUDA(c, cudaStreamSynchronize(s));
  float ms;
  cudaEventElapsedTime(&ms, ev[0], ev[1]);
  gs.ms_geometry = ms;
  cudaEventElapsedTime(&ms, ev[1], ev[2]);
  gs.ms_weights = ms;
  cudaEventElapsedTime(&ms, ev[3], ev[4]);
  gs.ms_levels = ms;
  for (auto& x : ev) cudaEventDestroy(x);
  gs.max_level = Lmax;
  gs.n_mixed_faces = nm;
  {
    // FP32 (hi, lo) splits of the directions and of sigma_t for the double-single form
    std::vector<float> om(6 * (size_t)M), stt(2 * (size_t)E), sig(E);
    std::vector<double> sigd(E);
    SN_CUDA(c, cudaMemcpy(sigd.data(), c->d_sig_t, E * 8, cudaMemcpyDeviceToHost));
    for (int64_t d = 0; d < M; ++d)
      for (int k = 0; k < 3; ++k) {
        const double x = c->h_omega[d * 3 + k];
        const float h = (float)x;
        om[d * 6 + 2 * k] = h;
        om[d * 6 + 2 * k + 1] = (float)(x - (double)h);
      }
    for (int64_t e = 0; e < E; ++e) {
      const float h = (float)sigd[e];
      stt[2 * e] = h;
      stt[2 * e + 1] = (float)(sigd[e] - (double)h);
    }
    SN_CUDA(c, dalloc(c->d_om32, om.size()));
    SN_CUDA(c, dalloc(c->d_st32, stt.size()));
    SN_CUDA(c, cudaMemcpy(c->d_om32, om.data(), om.size() * 4, cudaMemcpyHostToDevice));
    SN_CUDA(c, cudaMemcpy(c->d_st32, stt.data(), stt.size() * 4, cudaMemcpyHostToDevice));
  }
  sn_status st = ensure_buffers(c);
  if (st != SN_OK) return st;
  c->graph_ready = true;
  if (stats) *stats = gs;
  return SN_OK;
}

sn_status sn_set_launch(sn_ctx* c, int mode, int blocks_per_sm) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, mode == SN_LAUNCH_LEVELS || mode == SN_LAUNCH_DATAFLOW, SN_EINVAL, "unknown launch mode");
  SN_REQ(c, blocks_per_sm >= 0 && blocks_per_sm <= 64, SN_EINVAL, "blocks_per_sm must be 0..64");
  c->launch_mode = mode;
  c->blocks_per_sm = blocks_per_sm;
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  return SN_OK;
}

sn_status sn_set_spin_limit(sn_ctx* c, int64_t polls) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, polls >= 0, SN_EINVAL, "polls must be >= 0");
  c->spin_limit = (long long)polls;
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);   // captured launches hold the old limit
  c->graphs.clear();
  return SN_OK;
}

sn_status sn_autotune(sn_ctx* c, int precision, int* mode_out, int* blocks_per_sm_out) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->graph_ready, SN_ESTATE, "sn_build_graph first");
  const int cand[6][2] = {{SN_LAUNCH_LEVELS, 0}, {SN_LAUNCH_DATAFLOW, 1}, {SN_LAUNCH_DATAFLOW, 2},
                          {SN_LAUNCH_DATAFLOW, 3}, {SN_LAUNCH_DATAFLOW, 4}, {SN_LAUNCH_DATAFLOW, 0}};
  float best = 1e30f;
  int bm = SN_LAUNCH_LEVELS, bb = 0;
  for (auto& cd : cand) {
    sn_status st = sn_set_launch(c, cd[0], cd[1]);
    if (st != SN_OK) return st;
    if ((st = sn_si_begin(c, nullptr)) != SN_OK) return st;
    for (int w = 0; w < 2; ++w)                                                  // capture + warm
      if ((st = sn_si_step(c, precision, nullptr, nullptr)) != SN_OK) return st;
    float tot = 1e30f;                                                           // fastest of 5 sweeps
    for (int r = 0; r < 5; ++r) {
      float ms = 0.0f;
      if ((st = sn_si_step(c, precision, nullptr, &ms)) != SN_OK) return st;
      tot = std::min(tot, ms);
    }
    if (tot < best) {
      best = tot;
      bm = cd[0];
      bb = cd[1];
    }
  }
  sn_status st = sn_set_launch(c, bm, bb);
  if (st != SN_OK) return st;
  if ((st = sn_si_begin(c, nullptr)) != SN_OK) return st;
  if (mode_out) *mode_out = bm;
  if (blocks_per_sm_out) *blocks_per_sm_out = bb;
  return SN_OK;
}

sn_status sn_get_graph(sn_ctx* c, int64_t* n_removed, int32_t* removed, int64_t cap, int32_t* levels) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->graph_ready, SN_ESTATE, "sn_build_graph first");
  cudaSetDevice(c->device);
  if (n_removed) *n_removed = c->n_removed;
  if (removed) {
    SN_REQ(c, cap >= c->n_removed, SN_EINVAL, "removed buffer too small");
    std::memcpy(removed, c->h_removed.data(), c->h_removed.size() * 4);
  }
  if (levels) {
    SN_CUDA(c, cudaMemcpyAsync(levels, c->d_levels, (size_t)c->M * c->E * 4, cudaMemcpyDefault, c->stream));
    SN_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return SN_OK;
}

namespace {

// Stored inverses and inflow face blocks of the stored-inverse forms: the block index of every
// pair (its inflow faces counted in pair order) is set up on the host from the face codes, the
// buffers are allocated once per graph, and one launch forms every record in the layout of
// `prec` (doubles, or (hi, lo) FP32 pairs of the same values).
sn_status form_inverse(sn_ctx* c, int prec, float* ms) {
  const size_t npair = (size_t)c->M * c->E;
  const size_t nblk = (size_t)c->Nf * c->Nf;
  c->inv_form = -1;
  if (!c->d_fidx || !c->d_inv) drop_graphs(c);   // new record addresses: captured sweeps are stale
  if (!c->d_fidx) {
    std::vector<uint32_t> code(npair);
    SN_CUDA(c, cudaMemcpyAsync(code.data(), c->d_facecode, npair * 4, cudaMemcpyDeviceToHost, c->stream));
    SN_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<int32_t> fidx(npair);
    int64_t tot = 0;
    for (size_t q = 0; q < npair; ++q) {
      fidx[q] = (int32_t)tot;
      for (int f = 0; f < c->nfc; ++f) tot += face_mode(code[q], f) != MODE_NONE;
      if (tot > INT32_MAX) {
        set_err(c, "stored inverses: more than 2^31 inflow face blocks");
        return SN_EINVAL;
      }
    }
    // 2D: folded blocks C_f = Ainv B_f (N x Nf per inflow face); 3D: the blocks B_f (Nf x Nf)
    const size_t nfb = std::max<size_t>(1, (size_t)tot) * (c->dim == 2 ? (size_t)c->N * c->Nf : nblk);
    if (dalloc(c->d_fblk, nfb) != cudaSuccess || dalloc(c->d_fidx, npair) != cudaSuccess) {
      cudaGetLastError();
      dfree(c->d_fblk);
      dfree(c->d_fidx);
      set_err(c, "stored inverses: " + std::to_string(nfb * 8) + " bytes of face blocks do not fit in device memory");
      return SN_ENOMEM;
    }
    SN_CUDA(c, cudaMemcpyAsync(c->d_fidx, fidx.data(), npair * 4, cudaMemcpyHostToDevice, c->stream));
    SN_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  if (!c->d_inv) {
    const size_t n = npair * c->N * c->N;
    if (dalloc(c->d_inv, n) != cudaSuccess) {
      cudaGetLastError();
      c->d_inv = nullptr;
      set_err(c, "stored inverses: " + std::to_string(n * 8) + " bytes do not fit in device memory");
      return SN_ENOMEM;
    }
  }
  if (ms && !c->ev_a) {
    SN_CUDA(c, cudaEventCreate(&c->ev_a));
    SN_CUDA(c, cudaEventCreate(&c->ev_b));
  }
  DevProblem P = c->dev();
  SweepArgs sa{c->d_facecode, c->d_mixed_off, c->d_mixedB, c->d_mixedB32, c->d_mixedB32lo, c->d_src,
               nullptr, nullptr, nullptr, nullptr, nullptr,
               nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, c->d_inv, c->d_fblk, c->d_fidx};
  if (ms) SN_CUDA(c, cudaEventRecord(c->ev_a, c->stream));
  SN_CUDA(c, launch_invert(P, prec, sa, c->stream));
  c->launches++;
  if (ms) {
    SN_CUDA(c, cudaEventRecord(c->ev_b, c->stream));
    SN_CUDA(c, cudaEventSynchronize(c->ev_b));
    SN_CUDA(c, cudaEventElapsedTime(ms, c->ev_a, c->ev_b));
  } else {
    SN_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  c->inv_form = prec;
  return SN_OK;
}

// One sweep: either one launch per level, or one persistent dataflow launch (completion flags
// and queue head cleared first).  Replayed from a captured CUDA graph when the stream allows
// capture (not the legacy default stream).
sn_status run_levels(sn_ctx* c, int prec, const double* psi_old, double* psi_new) {
  DevProblem P = c->dev();
  const int64_t L = (int64_t)c->level_off.size() - 1;
  const int64_t total = c->level_off.back();
  int* err = reinterpret_cast<int*>(c->d_red + 2);
  unsigned long long* head = c->d_red + 3;
  const bool stored = prec == SN_PREC_FP64_INV || prec == SN_PREC_DS_INV;
  SN_REQ(c, stored || !c->simplex, SN_EINVAL,
         "triangle meshes: use a stored-inverse form (SN_PREC_FP64_INV or SN_PREC_DS_INV)");
  if (stored && c->inv_form != prec) {     // outside any capture: it synchronises
    sn_status st = form_inverse(c, prec, nullptr);
    if (st != SN_OK) return st;
  }
  SweepArgs sa{c->d_facecode, c->d_mixed_off, c->d_mixedB, c->d_mixedB32, c->d_mixedB32lo, c->d_src,
               psi_old, psi_new, c->d_done, err, c->d_pairs,
               c->d_srch, c->d_srcl, nullptr, nullptr, nullptr, nullptr, c->spin_limit,
               c->d_inv, c->d_fblk, c->d_fidx};
  // (hi, lo) splits of the two iterates: the context's own buffers, or scratch for caller buffers
  bool convert_old = false;
  const size_t npsi = (size_t)c->M * c->E * c->N;
  for (int k = 0; k < 2; ++k) {
    if (psi_old == c->d_psi[k]) {
      sa.psi_old_h = c->d_psih[k];
      sa.psi_old_l = c->d_psil[k];
    }
    if (psi_new == c->d_psi[k]) {
      sa.psi_new_h = c->d_psih[k];
      sa.psi_new_l = c->d_psil[k];
    }
  }
  if (prec == SN_PREC_MIXED_DS || prec == SN_PREC_DS_INV) {
    for (int k = 0; k < 2; ++k)
      if (!c->d_scr_h[k] && (k == 0 ? !sa.psi_old_h : !sa.psi_new_h)) {
        SN_CUDA(c, dalloc(c->d_scr_h[k], npsi));
        SN_CUDA(c, dalloc(c->d_scr_l[k], npsi));
      }
    if (!sa.psi_old_h) {
      sa.psi_old_h = c->d_scr_h[0];
      sa.psi_old_l = c->d_scr_l[0];
      convert_old = true;
    }
    if (!sa.psi_new_h) {
      sa.psi_new_h = c->d_scr_h[1];
      sa.psi_new_l = c->d_scr_l[1];
    }
  }
  const int mode = c->launch_mode;
  auto launch_all = [&]() -> cudaError_t {
    if (convert_old) {
      cudaError_t e = launch_split(psi_old, c->d_scr_h[0], c->d_scr_l[0], (int64_t)npsi, c->stream);
      if (e != cudaSuccess) return e;
    }
    if (mode == SN_LAUNCH_DATAFLOW) {
      cudaError_t e = cudaMemsetAsync(c->d_done, 0, (size_t)c->M * c->E * sizeof(int), c->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(c->d_red + 2, 0, 2 * sizeof(unsigned long long), c->stream);
      if (e == cudaSuccess)
        e = launch_sweep_flow(P, prec, c->d_pairs, total, sa, head, c->blocks_per_sm, c->stream);
      return e;
    }
    for (int64_t l = 0; l < L; ++l) {
      const int64_t off = c->level_off[l], cnt = c->level_off[l + 1] - off;
      cudaError_t e = launch_sweep_level(P, prec, c->d_pairs + off, cnt, sa, c->stream);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  c->launches += (mode == SN_LAUNCH_DATAFLOW) ? 1 : L;
  if (c->stream == nullptr) {
    SN_CUDA(c, launch_all());
    return SN_OK;
  }
  sn_ctx::GraphKey key{prec * 16 + mode, psi_old, psi_new};
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    if (c->graphs.size() >= 8) {
      for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
      c->graphs.clear();
    }
    cudaGraph_t g;
    SN_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = launch_all();
    cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    SN_CUDA(c, le);
    SN_CUDA(c, ee);
    cudaGraphExec_t ge;
    cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    SN_CUDA(c, ie);
    it = c->graphs.emplace(key, ge).first;
  }
  SN_CUDA(c, cudaGraphLaunch(it->second, c->stream));
  return SN_OK;
}

// After a synchronised sweep: SN_ETIMEOUT if a dataflow wait gave up.
sn_status check_err(sn_ctx* c) {
  if (c->launch_mode != SN_LAUNCH_DATAFLOW) return SN_OK;
  unsigned long long w = 0;
  SN_CUDA(c, cudaMemcpyAsync(&w, c->d_red + 2, sizeof(w), cudaMemcpyDeviceToHost, c->stream));
  SN_CUDA(c, cudaStreamSynchronize(c->stream));
  if (w & 0xffffffffull) {
    set_err(c, "dataflow sweep: a dependency wait exceeded its spin limit");
    return SN_ETIMEOUT;
  }
  return SN_OK;
}

const double* stage_in(sn_ctx* c, const double* p, size_t n, int slot, sn_status& st) {
  st = SN_OK;
  if (!p || is_device_ptr(p)) return p;
  if ((st = ensure_stage(c, slot)) != SN_OK) return nullptr;
  cudaError_t e = cudaMemcpyAsync(c->d_stage[slot], p, n * 8, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) {
    set_err(c, std::string("cudaMemcpyAsync H2D: ") + cudaGetErrorString(e));
    st = SN_ECUDA;
    return nullptr;
  }
  return c->d_stage[slot];
}

}  // namespace

sn_status sn_prepare_inverse(sn_ctx* c, int precision, float* ms) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->graph_ready, SN_ESTATE, "sn_build_graph first");
  SN_REQ(c, precision == SN_PREC_FP64_INV || precision == SN_PREC_DS_INV, SN_EINVAL,
         "precision must be SN_PREC_FP64_INV or SN_PREC_DS_INV");
  cudaSetDevice(c->device);
  return form_inverse(c, precision, ms);
}

sn_status sn_release_inverse(sn_ctx* c) {
  if (!c) return SN_EINVAL;
  cudaSetDevice(c->device);
  SN_CUDA(c, cudaStreamSynchronize(c->stream));
  free_inverse(c);
  return SN_OK;
}

sn_status sn_sweep(sn_ctx* c, const double* phi_in, const double* psi_old, double* psi_new, int precision) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->graph_ready, SN_ESTATE, "sn_build_graph first");
  SN_REQ(c, phi_in && psi_old && psi_new, SN_EINVAL, "null array");
  SN_REQ(c, (const void*)psi_old != (const void*)psi_new, SN_EINVAL, "psi_new must not alias psi_old");
  SN_REQ(c, precision >= SN_PREC_FP64 && precision <= SN_PREC_DS_INV, SN_EINVAL, "unknown precision");
  cudaSetDevice(c->device);
  const size_t npsi = (size_t)c->M * c->E * c->N, nphi = (size_t)c->E * c->N;
  sn_status st;
  const double* dphi = stage_in(c, phi_in, nphi, 0, st);
  if (st != SN_OK) return st;
  const double* dold = stage_in(c, psi_old, npsi, 1, st);
  if (st != SN_OK) return st;
  const bool host_out = !is_device_ptr(psi_new);
  double* dnew = psi_new;
  if (host_out) {
    if ((st = ensure_stage(c, 2)) != SN_OK) return st;
    dnew = c->d_stage[2];
  }
  DevProblem P = c->dev();
  SN_CUDA(c, launch_source(P, dphi, c->d_src, c->d_srch, c->d_srcl, c->stream));
  c->launches++;
  if ((st = run_levels(c, precision, dold, dnew)) != SN_OK) return st;
  if (host_out) {
    SN_CUDA(c, cudaMemcpyAsync(psi_new, dnew, npsi * 8, cudaMemcpyDeviceToHost, c->stream));
  }
  if (host_out || !is_device_ptr(phi_in) || !is_device_ptr(psi_old)) SN_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_err(c);
}

int32_t sn_num_volume_points(const sn_ctx* c) { return (c && c->disc_set) ? c->tab.Q : 0; }

sn_status sn_volume_points(sn_ctx* c, double* xq) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->mesh_set && c->disc_set, SN_ESTATE, "mesh and discretization first");
  SN_REQ(c, xq, SN_EINVAL, "null array");
  cudaSetDevice(c->device);
  const size_t n = (size_t)c->E * c->tab.Q * c->dim;
  const bool dev_out = is_device_ptr(xq);
  double* d = dev_out ? xq : nullptr;
  if (!dev_out) SN_CUDA(c, dalloc(d, n));
  DevProblem P = c->dev();
  cudaError_t e = launch_volume_points(P, nullptr, nullptr, d, nullptr, c->stream);
  if (e == cudaSuccess && !dev_out) e = cudaMemcpyAsync(xq, d, n * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (!dev_out) dfree(d);
  SN_CUDA(c, e);
  c->launches++;
  return SN_OK;
}

sn_status sn_l2_error(sn_ctx* c, const double* phi, const double* exact_q, double* err) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->mesh_set && c->disc_set, SN_ESTATE, "mesh and discretization first");
  SN_REQ(c, phi && exact_q && err, SN_EINVAL, "null array");
  cudaSetDevice(c->device);
  const size_t nphi = (size_t)c->E * c->N, nq = (size_t)c->E * c->tab.Q;
  double *dphi = nullptr, *dex = nullptr, *dacc = nullptr;
  cudaError_t e = dalloc(dphi, nphi);
  if (e == cudaSuccess) e = dalloc(dex, nq);
  if (e == cudaSuccess) e = dalloc(dacc, 1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dphi, phi, nphi * 8, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dex, exact_q, nq * 8, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dacc, 0, 8, c->stream);
  DevProblem P = c->dev();
  if (e == cudaSuccess) e = launch_volume_points(P, dphi, dex, nullptr, dacc, c->stream);
  double acc = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&acc, dacc, 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(dphi);
  dfree(dex);
  dfree(dacc);
  SN_CUDA(c, e);
  c->launches++;
  *err = std::sqrt(acc);
  return SN_OK;
}

sn_status sn_moment(sn_ctx* c, const double* psi, const double* phi_prev, double* phi_out, double* residual) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->graph_ready, SN_ESTATE, "sn_build_graph first");
  SN_REQ(c, psi && phi_out, SN_EINVAL, "null array");
  cudaSetDevice(c->device);
  const size_t npsi = (size_t)c->M * c->E * c->N, nphi = (size_t)c->E * c->N;
  sn_status st;
  const double* dpsi = stage_in(c, psi, npsi, 1, st);
  if (st != SN_OK) return st;
  const double* dprev = stage_in(c, phi_prev, nphi, 0, st);
  if (st != SN_OK) return st;
  const bool host_out = !is_device_ptr(phi_out);
  double* dout = host_out ? c->d_phi2 : phi_out;
  SN_CUDA(c, cudaMemsetAsync(c->d_red, 0, 2 * sizeof(unsigned long long), c->stream));
  DevProblem P = c->dev();
  SN_CUDA(c, launch_moment(P, dpsi, dprev, dout, c->d_src, c->d_srch, c->d_srcl, c->d_red, c->stream));
  c->launches++;
  unsigned long long red[2];
  SN_CUDA(c, cudaMemcpyAsync(red, c->d_red, sizeof(red), cudaMemcpyDeviceToHost, c->stream));
  if (host_out) SN_CUDA(c, cudaMemcpyAsync(phi_out, dout, nphi * 8, cudaMemcpyDeviceToHost, c->stream));
  SN_CUDA(c, cudaStreamSynchronize(c->stream));
  double diff, mag;
  std::memcpy(&diff, &red[0], 8);
  std::memcpy(&mag, &red[1], 8);
  if (residual) *residual = mag > 0.0 ? diff / mag : (diff > 0.0 ? INFINITY : 0.0);
  return SN_OK;
}

namespace {
// Allocates and assembles the DSA operator of the current graph and materials (once).
sn_status dsa_prepare(sn_ctx* c) {
  sn::DsaState& D = c->dsa;
  if (D.ready) return SN_OK;
  SN_REQ(c, !c->simplex, SN_EINVAL, "diffusion synthetic acceleration: quadrilateral and hexahedral meshes only");
  const size_t N = c->N, E = c->E, nfc = 2 * c->dim;
  SN_CUDA(c, dalloc(D.diag, E * N * N));
  SN_CUDA(c, dalloc(D.inv, E * N * N));
  SN_CUDA(c, dalloc(D.selfb, E * nfc * N * N));
  SN_CUDA(c, dalloc(D.offb, E * nfc * N * N));
  SN_CUDA(c, dalloc(D.vol, E));
  for (double** p : {&D.b, &D.x, &D.r, &D.z, &D.p, &D.q}) SN_CUDA(c, dalloc(*p, E * N));
  SN_CUDA(c, dalloc(D.sc, 10));
  SN_CUDA(c, dalloc(D.bad, 1));
  SN_CUDA(c, cudaMemsetAsync(D.bad, 0, sizeof(int), c->stream));
  DevProblem P = c->dev();
  SN_CUDA(c, dsa_assemble(P, D, c->stream));
  c->launches += 3;
  int bad = 0;
  SN_CUDA(c, cudaMemcpyAsync(&bad, D.bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SN_CUDA(c, cudaStreamSynchronize(c->stream));
  if (bad) {
    set_err(c, "DSA operator: a diagonal block is singular");
    free_dsa(c);
    return SN_EMESH;
  }
  D.ready = true;
  return SN_OK;
}
}  // namespace

sn_status sn_set_dsa(sn_ctx* c, int enable, double rtol, int max_iter) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, enable == 0 || enable == 1, SN_EINVAL, "enable must be 0 or 1");
  SN_REQ(c, std::isfinite(rtol) && rtol > 0.0 && rtol < 1.0, SN_EINVAL, "rtol must be in (0, 1)");
  SN_REQ(c, max_iter >= 1 && max_iter <= 100000, SN_EINVAL, "max_iter must be 1..100000");
  c->dsa_on = enable == 1;
  c->dsa_rtol = rtol;
  c->dsa_max_iter = max_iter;
  return SN_OK;
}

sn_status sn_dsa_correction(sn_ctx* c, const double* phi_half, const double* phi_prev, double* phi_out,
                            int* cg_iters) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->graph_ready, SN_ESTATE, "sn_build_graph first");
  SN_REQ(c, phi_half && phi_prev && phi_out, SN_EINVAL, "null array");
  cudaSetDevice(c->device);
  sn_status st = dsa_prepare(c);
  if (st != SN_OK) return st;
  const size_t nphi = (size_t)c->E * c->N;
  // host or device inputs: staged into the context's scalar-flux buffers
  SN_CUDA(c, cudaMemcpyAsync(c->d_phi2, phi_half, nphi * 8, cudaMemcpyDefault, c->stream));
  SN_CUDA(c, cudaMemcpyAsync(c->d_phi, phi_prev, nphi * 8, cudaMemcpyDefault, c->stream));
  SN_CUDA(c, cudaMemsetAsync(c->d_red, 0, 2 * sizeof(unsigned long long), c->stream));
  DevProblem P = c->dev();
  int it = 0;
  SN_CUDA(c, dsa_apply(P, c->dsa, c->d_phi2, c->d_phi, c->d_phi2, c->d_src, c->d_srch, c->d_srcl, c->d_red,
                       c->dsa_rtol, c->dsa_max_iter, &it, &c->launches, c->stream));
  SN_CUDA(c, cudaMemcpyAsync(phi_out, c->d_phi2, nphi * 8, cudaMemcpyDefault, c->stream));
  SN_CUDA(c, cudaStreamSynchronize(c->stream));
  c->dsa_last_iters = it;
  c->si_ready = false;                 // the iteration buffers were used as scratch
  if (cg_iters) *cg_iters = it;
  return SN_OK;
}

int32_t sn_dsa_last_iters(const sn_ctx* c) { return c ? c->dsa_last_iters : 0; }

sn_status sn_si_begin(sn_ctx* c, const double* phi0) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->graph_ready, SN_ESTATE, "sn_build_graph first");
  cudaSetDevice(c->device);
  const size_t npsi = (size_t)c->M * c->E * c->N, nphi = (size_t)c->E * c->N;
  cudaStream_t s = c->stream;
  if (phi0) SN_CUDA(c, cudaMemcpyAsync(c->d_phi, phi0, nphi * 8, cudaMemcpyDefault, s));
  else SN_CUDA(c, cudaMemsetAsync(c->d_phi, 0, nphi * 8, s));
  SN_CUDA(c, cudaMemsetAsync(c->d_psi[0], 0, npsi * 8, s));
  SN_CUDA(c, cudaMemsetAsync(c->d_psih[0], 0, npsi * 4, s));
  SN_CUDA(c, cudaMemsetAsync(c->d_psil[0], 0, npsi * 4, s));
  DevProblem P = c->dev();
  SN_CUDA(c, launch_source(P, c->d_phi, c->d_src, c->d_srch, c->d_srcl, s));
  c->launches++;
  SN_CUDA(c, cudaStreamSynchronize(s));
  c->si_cur = 0;
  c->si_ready = true;
  return SN_OK;
}

sn_status sn_si_step(sn_ctx* c, int precision, double* residual, float* ms_sweep) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->graph_ready && c->si_ready, SN_ESTATE, "sn_si_begin first");
  SN_REQ(c, precision >= SN_PREC_FP64 && precision <= SN_PREC_DS_INV, SN_EINVAL, "unknown precision");
  cudaSetDevice(c->device);
  cudaStream_t s = c->stream;
  if (ms_sweep && !c->ev_a) {
    SN_CUDA(c, cudaEventCreate(&c->ev_a));
    SN_CUDA(c, cudaEventCreate(&c->ev_b));
  }
  const int cur = c->si_cur;
  if (ms_sweep) SN_CUDA(c, cudaEventRecord(c->ev_a, s));
  sn_status st = run_levels(c, precision, c->d_psi[cur], c->d_psi[cur ^ 1]);
  if (st != SN_OK) return st;
  if (ms_sweep) SN_CUDA(c, cudaEventRecord(c->ev_b, s));
  SN_CUDA(c, cudaMemsetAsync(c->d_red, 0, 2 * sizeof(unsigned long long), s));
  DevProblem P = c->dev();
  if (c->dsa_on) {
    // phi_half = sum_d w_d psi_d, then phi = phi_half + dphi with the residual and the source
    if ((st = dsa_prepare(c)) != SN_OK) return st;
    SN_CUDA(c, launch_moment(P, c->d_psi[cur ^ 1], c->d_phi, c->d_phi2, nullptr, nullptr, nullptr, nullptr, s));
    c->launches++;
    int it = 0;
    SN_CUDA(c, dsa_apply(P, c->dsa, c->d_phi2, c->d_phi, c->d_phi2, c->d_src, c->d_srch, c->d_srcl, c->d_red,
                         c->dsa_rtol, c->dsa_max_iter, &it, &c->launches, s));
    c->dsa_last_iters = it;
  } else {
    SN_CUDA(c, launch_moment(P, c->d_psi[cur ^ 1], c->d_phi, c->d_phi2, c->d_src, c->d_srch, c->d_srcl, c->d_red,
                             s));
    c->launches++;
  }
  unsigned long long red[3];
  SN_CUDA(c, cudaMemcpyAsync(red, c->d_red, sizeof(red), cudaMemcpyDeviceToHost, s));
  SN_CUDA(c, cudaStreamSynchronize(s));
  if (c->launch_mode == SN_LAUNCH_DATAFLOW && (red[2] & 0xffffffffull)) {
    set_err(c, "dataflow sweep: a dependency wait exceeded its spin limit");
    return SN_ETIMEOUT;
  }
  double diff, mag;
  std::memcpy(&diff, &red[0], 8);
  std::memcpy(&mag, &red[1], 8);
  if (residual) *residual = mag > 0.0 ? diff / mag : (diff > 0.0 ? INFINITY : 0.0);
  if (ms_sweep) SN_CUDA(c, cudaEventElapsedTime(ms_sweep, c->ev_a, c->ev_b));
  std::swap(c->d_phi, c->d_phi2);
  c->si_cur = cur ^ 1;
  return SN_OK;
}

sn_status sn_si_result(sn_ctx* c, double* phi_out, double* psi_out) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->graph_ready && c->si_ready, SN_ESTATE, "sn_si_begin first");
  cudaSetDevice(c->device);
  const size_t npsi = (size_t)c->M * c->E * c->N, nphi = (size_t)c->E * c->N;
  if (phi_out) SN_CUDA(c, cudaMemcpyAsync(phi_out, c->d_phi, nphi * 8, cudaMemcpyDefault, c->stream));
  if (psi_out) SN_CUDA(c, cudaMemcpyAsync(psi_out, c->d_psi[c->si_cur], npsi * 8, cudaMemcpyDefault, c->stream));
  SN_CUDA(c, cudaStreamSynchronize(c->stream));
  return SN_OK;
}

sn_status sn_source_iterate(sn_ctx* c, double tol, int max_iter, int precision, const double* phi0, double* phi_out,
                            double* psi_out, sn_si_stats* stats, double* history, int history_cap) {
  if (!c) return SN_EINVAL;
  SN_REQ(c, c->graph_ready, SN_ESTATE, "sn_build_graph first");
  SN_REQ(c, max_iter >= 1 && tol > 0.0, SN_EINVAL, "max_iter >= 1 and tol > 0 required");
  SN_REQ(c, precision >= SN_PREC_FP64 && precision <= SN_PREC_DS_INV, SN_EINVAL, "unknown precision");
  auto t0 = std::chrono::steady_clock::now();
  sn_status st = sn_si_begin(c, phi0);
  if (st != SN_OK) return st;
  double res = INFINITY;
  int it = 0;
  bool conv = false;
  for (it = 1; it <= max_iter; ++it) {
    if ((st = sn_si_step(c, precision, &res, nullptr)) != SN_OK) return st;
    if (history && it <= history_cap) history[it - 1] = res;
    if (res < tol) {
      conv = true;
      break;
    }
  }
  if (it > max_iter) it = max_iter;
  if ((st = sn_si_result(c, phi_out, psi_out)) != SN_OK) return st;
  if (stats) {
    stats->iters = it;
    stats->converged = conv ? 1 : 0;
    stats->residual = res;
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (!conv) {
    set_err(c, "source iteration did not reach tol within max_iter");
    return SN_ENOTCONVERGED;
  }
  return SN_OK;
}

}  // extern "C"
