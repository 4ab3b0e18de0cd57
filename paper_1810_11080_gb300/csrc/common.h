// Internal declarations of the snsweep library: the context, host tables and the kernel
// launchers implemented in geom.cu (element factors), graph.cu (edge weights, levels) and
// sweep.cu (lagged sweep, scalar-flux moment and scattering source).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>
#include <map>
#include "../../include/snsweep.h"

namespace sn {

constexpr int MAX_DIM = 3;
constexpr int MAX_P = 3;
constexpr int MAX_R = 3;
constexpr int MAX_NF1 = 8;          // max 1D face GL points (p + r <= 6) ... headroom

// Face-code word per (direction, element): bits [2f, 2f+1] = inflow mode of local face f
// (0 none, 1 whole face inflow, 2 partial inflow), bit 16 + f = arc through face f lagged.
constexpr uint32_t MODE_NONE = 0, MODE_PURE = 1, MODE_MIXED = 2;
__host__ __device__ inline uint32_t face_mode(uint32_t code, int f) { return (code >> (2 * f)) & 3u; }
__host__ __device__ inline bool face_lagged(uint32_t code, int f) { return (code >> (16 + f)) & 1u; }

// 1D tables computed on the host (tables.cpp) and uploaded.
struct Tables {
  int nv = 0, nf = 0, p = 0, r = 0, dim = 0, N = 0, Nf = 0, Nv = 0, Q = 0;
  std::vector<double> glv_t, glv_w;     // volume GL nodes/weights on [0,1]
  std::vector<double> glf_t, glf_w;     // face GL nodes/weights on [0,1]
  std::vector<double> gll;              // DG nodes
  std::vector<double> geo;              // geometry nodes a/r
  std::vector<double> wq;               // [Q] tensor volume weights
  std::vector<double> B;                // [Q][N] DG basis at volume points
  std::vector<double> dB;               // [Q][N][dim] reference gradients
  std::vector<double> dV;               // [Q][Nv][dim] geometry basis reference gradients
  std::vector<double> V;                // [Q][Nv] geometry basis values
};

void gauss_legendre(int n, std::vector<double>& t, std::vector<double>& w);
void gll_nodes(int p, std::vector<double>& x);
double lagrange(const double* nodes, int n, int j, double x);
double lagrange_deriv(const double* nodes, int n, int j, double x);
void build_tables(Tables& T, int dim, int p, int r);
void build_tables_tri(Tables& T, int p, int r);
void build_tables_tet(Tables& T, int p);

// Components and feedback arc sets of every direction's graph on the device (scc.cu).
struct DeviceFasStats {
  int64_t n_scc = 0;        // components of at least two vertices, over all directions
  int32_t max_scc = 0;
  int64_t n_removed = 0;    // arcs marked lagged
  int64_t launches = 0;
  int stuck = 0;            // a fixed-point loop exceeded its bound
};
struct DevProblem;
cudaError_t device_fas(const DevProblem& P, uint32_t* fc, const double* win, int exact_max, DeviceFasStats* stats,
                       cudaStream_t s);

// Diffusion synthetic acceleration (dsa.cu): the operator's blocks and the CG vectors.
struct DsaState {
  double *diag = nullptr, *inv = nullptr, *selfb = nullptr, *offb = nullptr, *vol = nullptr;   // operator
  double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;   // CG
  double* sc = nullptr;    // [0] b.b, then a ring of three (p.q, r.z, r.r) slots
  int* bad = nullptr;      // a diagonal block was singular
  bool ready = false;
};
struct DevProblem;
cudaError_t dsa_assemble(const DevProblem& P, DsaState& D, cudaStream_t s);
cudaError_t dsa_apply(const DevProblem& P, DsaState& D, const double* half, const double* prev, double* phi_new,
                      double* src, float* src_h, float* src_l, unsigned long long* red, double rtol, int max_iter,
                      int* cg_iters, int64_t* launches, cudaStream_t s);

// Device-side view of a problem passed to kernels by value.
struct DevProblem {
  int dim, r, p, N, Nf, nv, nf, K, Q, Nv, M;
  int nfc;                   // faces per element: 2 dim (quadrilaterals, hexahedra) or dim + 1 (simplices)
  int simplex;               // 1: triangles (P_r geometry) or straight tetrahedra, P_p DG (see tables.cpp)
  int64_t E;
  int64_t n_bdr;
  const double* ctrl;        // [E][Nv][dim]
  const int64_t* nbr;        // [E][2dim]
  const int32_t* nbr_face;   // [E][2dim]
  const int32_t* orient;     // [E][2dim]
  const int64_t* bdr_index;  // [E][2dim] boundary-face number or -1
  const double* omega;       // [M][3]
  const double* w;           // [M]
  const double* sig_t;       // [E]
  const double* sig_s;       // [E]
  const double* q;           // [E][N]
  const double* q_dir;       // [M][E][N] or null
  const double* psi_inc;     // [M][n_bdr][Nf] or null
  const double* tab;         // packed tables (see TabOffsets)
  int off_glv_t, off_glv_w, off_glf_t, off_glf_w, off_gll, off_geo, off_wq, off_B, off_dB, off_dV, off_V;
  const double* elem;        // [E][blk] element factors
  int64_t blk;               // doubles per element block
  const float* elem32;       // [E][blk] FP32 rounding of elem (mixed forms) or null
  const float* elem32lo;     // [E][blk] FP32 rounding of elem - elem32 (double-single form) or null
  const float* om32;         // [M][6] (hi, lo) FP32 split of each direction's three components
  const float* st32;         // [E][2] (hi, lo) FP32 split of sigma_t
};

// Per-sweep buffers seen by the sweep kernels.
struct SweepArgs {
  const uint32_t* facecode;   // [M][E]
  const int32_t* mixed_off;   // [M][E]
  const double* mixedB;       // partially-inflow blocks, FP64
  const float* mixedBh;       // and their FP32 hi / lo split
  const float* mixedBl;
  const double* src;          // [E][N] M (q + sigma_s phi / 4 pi)
  const double* psi_old;      // previous iterate (lagged arcs)
  double* psi_new;            // this sweep's result
  int* done;                  // [M][E] completion flags (dataflow schedule) or null
  int* err;                   // device error word (dataflow wait gave up) or null
  const int32_t* pairs;       // level-ordered (e*M + d) work list (-1 = padding); batched kernels
  // double-single form: FP32 (hi, lo) splits of the source and of both angular-flux iterates
  const float* src_h;
  const float* src_l;
  const float* psi_old_h;
  const float* psi_old_l;
  float* psi_new_h;
  float* psi_new_l;
  long long spin_limit;       // dataflow schedule: polls of one upwind flag before giving up (<= 0: SPIN_LIMIT)
  // stored-inverse forms: per pair q = d E + e, inv + q N^2 holds the inverse column-major and
  // fblk + (fidx[q] + r) Nf^2 the block of its r-th inflow face (row-major); doubles for
  // SN_PREC_FP64_INV, (hi, lo) FP32 pairs for SN_PREC_DS_INV
  double* inv;
  double* fblk;
  const int32_t* fidx;
};

// Per-problem pointers of the fused moment / source kernel in a batch.
struct MomentArgs {
  const double* psi;          // [M][E][N] this sweep's angular flux
  const double* phi_prev;     // [E][N]
  double* phi_out;            // [E][N]
  double* src;                // [E][N] scattering + isotropic source for the next sweep
  float* src_h;               // its FP32 (hi, lo) split (double-single form)
  float* src_l;
};

// Batched sweep over problems of one dimension (batch.cu).  A task = up to 32/W consecutive
// entries of one problem's level-ordered pair list; int4 = (problem, p, offset, 0).
cudaError_t launch_batch_sweep(int dim, int precision, bool dataflow, const DevProblem* probs, const SweepArgs* args,
                               const int4* tasks, int64_t ntasks, unsigned long long* head, int* err,
                               int blocks_per_sm, cudaStream_t s);
cudaError_t launch_batch_moment(const DevProblem* probs, const MomentArgs* margs, const int64_t* block_off,
                                int nprob, int64_t nblocks, unsigned long long* red, cudaStream_t s);

// Element factor block layout: S^0..S^{dim-1} (N x N, S^k[m][n] = int du_m/dx_k u_n),
// mass M (N x N), then face matrices FN[f][k][i][j] = int_face w N_k phi_i phi_j with the
// element's own outward scaled normal (2 dim faces x dim components x Nf x Nf).
inline int64_t elem_block_doubles(int dim, int N, int Nf, int nfc) {
  return (int64_t)(dim + 1) * N * N + (int64_t)nfc * dim * Nf * Nf;
}

// Launchers (return cudaError_t of the launch).
cudaError_t launch_geometry(const DevProblem& P, double* elem, int* bad_flag, cudaStream_t s);
// Physical volume quadrature points (xq [E][Q][dim], may be null) and, if phi is not null,
// acc[0] += sum_e sum_q w_q |J_q| (sum_n B_qn phi_en - exact_q[e][q])^2 (geom.cu).
cudaError_t launch_volume_points(const DevProblem& P, const double* phi, const double* exact_q, double* xq,
                                 double* acc, cudaStream_t s);
cudaError_t launch_elem_to_fp32(const DevProblem& P, float* elem32, float* elem32lo, cudaStream_t s);
cudaError_t launch_mass_lu(const DevProblem& P, double* lu, int32_t* perm, cudaStream_t s);
cudaError_t launch_weights(const DevProblem& P, const int32_t* iface, int64_t n_iface, int weighting,
                           const double* mt_lu, const int32_t* mt_perm, double* win, uint32_t* facecode,
                           cudaStream_t s);
cudaError_t launch_bdr_modes(const DevProblem& P, const int32_t* bface, int64_t n_bface, uint32_t* facecode,
                             cudaStream_t s);
cudaError_t launch_mixed_blocks(const DevProblem& P, const int32_t* iface, int64_t n_iface,
                                const int32_t* bface, int64_t n_bface, const uint32_t* facecode,
                                const int32_t* mixed_off, double* mixedB, float* mixedB32, float* mixedB32lo,
                                cudaStream_t s);
cudaError_t launch_levels_init(const DevProblem& P, int32_t* levels, cudaStream_t s);
cudaError_t launch_levels_relax(const DevProblem& P, const uint32_t* facecode, int32_t* levels, int* changed,
                                cudaStream_t s);
cudaError_t launch_source(const DevProblem& P, const double* phi, double* src, float* src_h, float* src_l,
                          cudaStream_t s);
cudaError_t launch_moment(const DevProblem& P, const double* psi, const double* phi_prev, double* phi_out,
                          double* src, float* src_h, float* src_l, unsigned long long* red, cudaStream_t s);
cudaError_t launch_split(const double* x, float* h, float* l, int64_t n, cudaStream_t s);
cudaError_t launch_sweep_level(const DevProblem& P, int precision, const int32_t* pairs, int64_t count,
                               const SweepArgs& sa, cudaStream_t s);
cudaError_t launch_sweep_flow(const DevProblem& P, int precision, const int32_t* pairs, int64_t count,
                              const SweepArgs& sa, unsigned long long* head, int blocks_per_sm, cudaStream_t s);
// Forms sa.inv and sa.fblk for every (direction, element) pair in the layout of `precision`
// (SN_PREC_FP64_INV or SN_PREC_DS_INV) (sweep_inv.cu).
cudaError_t launch_invert(const DevProblem& P, int precision, const SweepArgs& sa, cudaStream_t s);

}  // namespace sn

struct sn_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int64_t launches = 0;
  // mesh (host copies)
  int dim = 0, r = 0;
  bool simplex = false;            // triangles or tetrahedra (sn_set_mesh_simplex)
  int nfc = 0;                     // faces per element
  int64_t E = 0;
  std::vector<double> h_ctrl;
  std::vector<int64_t> h_nbr;
  std::vector<int32_t> h_nbr_face, h_orient;
  std::vector<int64_t> h_bdr_index;
  std::vector<int32_t> h_iface;     // [n_iface][5]: owner, f, nbr, f_nbr, orient
  std::vector<int32_t> h_bface;     // [n_bface][2]: e, f
  int64_t n_bdr = 0;
  bool mesh_set = false;
  // discretization
  int p = 0, K = 2, N = 0, Nf = 0;
  bool disc_set = false;
  sn::Tables tab;
  // quadrature
  int M = 0;
  std::vector<double> h_omega, h_w;
  bool quad_set = false;
  bool mat_set = false;
  // device memory
  double *d_ctrl = nullptr, *d_omega = nullptr, *d_w = nullptr, *d_tab = nullptr;
  int64_t* d_nbr = nullptr;
  int64_t* d_bdr_index = nullptr;
  int32_t *d_nbr_face = nullptr, *d_orient = nullptr, *d_iface = nullptr, *d_bface = nullptr;
  double *d_sig_t = nullptr, *d_sig_s = nullptr, *d_q = nullptr, *d_qdir = nullptr, *d_psi_inc = nullptr;
  double* d_elem = nullptr;
  float* d_elem32 = nullptr;
  float* d_elem32lo = nullptr;
  int64_t blk = 0;
  int tab_off[11] = {0};
  // graph
  bool graph_ready = false;
  uint32_t* d_facecode = nullptr;
  int32_t* d_mixed_off = nullptr;
  double* d_mixedB = nullptr;
  float* d_mixedB32 = nullptr;
  float* d_mixedB32lo = nullptr;
  int64_t n_mixed = 0;
  int32_t* d_levels = nullptr;
  int32_t* d_pairs = nullptr;
  std::vector<int32_t> h_pairs;     // host copy of the padded, level-ordered work list
  std::vector<int64_t> level_off;
  std::vector<int32_t> h_removed;   // (d, e, e') triples
  int64_t n_removed = 0;
  // iteration state
  double* d_psi[2] = {nullptr, nullptr};
  double *d_phi = nullptr, *d_phi2 = nullptr, *d_src = nullptr;
  float* d_psih[2] = {nullptr, nullptr};   // FP32 (hi, lo) splits of d_psi (double-single form)
  float* d_psil[2] = {nullptr, nullptr};
  float *d_srch = nullptr, *d_srcl = nullptr;
  float *d_scr_h[2] = {nullptr, nullptr}, *d_scr_l[2] = {nullptr, nullptr};   // for caller psi buffers
  float *d_om32 = nullptr, *d_st32 = nullptr;
  double* d_stage[3] = {nullptr, nullptr, nullptr};   // host-pointer staging
  unsigned long long* d_red = nullptr;   // [0..1] residual maxima, [2] error word, [3] queue head
  int* d_flag = nullptr;
  int* d_done = nullptr;                 // [M][E] dataflow completion flags
  // diffusion synthetic acceleration (sn_set_dsa)
  sn::DsaState dsa;
  bool dsa_on = false;
  double dsa_rtol = 1e-4;
  int dsa_max_iter = 500;
  int dsa_last_iters = 0;
  // stored local inverses and inflow face blocks (SN_PREC_FP64_INV, SN_PREC_DS_INV)
  double* d_inv = nullptr;
  double* d_fblk = nullptr;
  int32_t* d_fidx = nullptr;
  int inv_form = -1;               // the form the stored records are written for (-1: none)
  int launch_mode = 0;                   // SN_LAUNCH_LEVELS / SN_LAUNCH_DATAFLOW
  long long spin_limit = 0;              // dataflow wait limit (0: the kernels' default)
  int blocks_per_sm = 0;                 // dataflow grid: 0 = occupancy limit
  int si_cur = 0;                 // which psi buffer holds the current iterate
  bool si_ready = false;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  // CUDA graphs of the per-level sweep launches, keyed by (precision, psi_old, psi_new)
  struct GraphKey {
    int prec; const void* a; const void* b;
    bool operator<(const GraphKey& o) const {
      if (prec != o.prec) return prec < o.prec;
      if (a != o.a) return a < o.a;
      return b < o.b;
    }
  };
  std::map<GraphKey, cudaGraphExec_t> graphs;
  sn::DevProblem dev() const;
};

