// Cycle breaking of every direction's dependency graph on the device (Sec. 3, last two
// paragraphs): strongly connected components, then per component a minimum-weight feedback arc
// set -- exact by dynamic programming over vertex subsets on components of at most exact_max
// vertices (the paper's integer program on components of "say 10" vertices), the weighted
// Eades-Lin-Smyth heuristic on larger ones.  The removed (lagged) arcs are marked in the face-code
// words; the sweep levels are computed from them afterwards.
//
// Graph of direction d: vertex e (an element); arc u -> e through face f of e when e's face f is
// an inflow face (mode != NONE) and u = nbr[e][f] >= 0; its weight is win[d][e][f] (unity, face or
// sigma-inverse-face, written by the edge-weight kernel).  An element shares at most one face with
// another element, so arcs are identified by their end points.
//
// Components (the partition is unique, so the parallel order of the steps does not matter):
// vertices without a live in-arc or without a live out-arc are trivial and are removed ("trim",
// repeated to a fixed point); on what is left every vertex takes the largest element id among its
// live ancestors ("colour"), a vertex whose colour is its own id is a root, and the vertices of
// that colour which reach the root within the colour form the root's component; those are
// removed, and trim / colour repeat until no vertex is left.
//
// The FAS of a component is deterministic and identical to the host restatement: members are
// ordered by element id; the subset DP takes cost(S + {v}) = cost(S) + sum over u outside S + {v}
// of z(u -> v) (u ascending from 0.0), subsets by increasing bitmask and v ascending with strict
// improvement only -- for a fixed set T the winning last vertex is therefore the largest v among
// the minimisers; Eades-Lin-Smyth removes the smallest-id sink (prepended to s2) while there is one,
// then the smallest-id source (appended to s1) while there is one, otherwise the vertex of largest
// delta = w_out - w_in (ties: smallest id, appended to s1), with w_out / w_in summed over live
// component neighbours in increasing id from 0.0.  Order = s1 s2; an arc is removed when its
// source comes after its destination.  Compiled with -fmad=false.
#include <algorithm>
#include <vector>
#include "common.h"

namespace sn {

namespace {

struct FasGraph {
  int M, nfc;
  int64_t E;
  const int64_t* nbr;
  const int32_t* nbr_face;
  const uint32_t* fc;
  const double* win;
};

// Arc u -> e through face f of e.
__device__ inline bool arc_in(const FasGraph& G, int64_t d, int64_t e, int f, int64_t& u) {
  u = G.nbr[e * G.nfc + f];
  return u >= 0 && face_mode(G.fc[d * G.E + e], f) != MODE_NONE;
}
// Arc e -> x through face f of e (x's face fx).
__device__ inline bool arc_out(const FasGraph& G, int64_t d, int64_t e, int f, int64_t& x, int& fx) {
  x = G.nbr[e * G.nfc + f];
  if (x < 0) return false;
  fx = G.nbr_face[e * G.nfc + f];
  return face_mode(G.fc[d * G.E + x], fx) != MODE_NONE;
}

__device__ inline int ld_vol(const int8_t* p) { return *(volatile const int8_t*)p; }
__device__ inline int ld_vol(const int32_t* p) { return *(volatile const int32_t*)p; }

// ---------------------------------------------------------------- components
__global__ void trim_kernel(FasGraph G, int8_t* alive, int* changed) {
  const int64_t n = (int64_t)G.M * G.E;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (!ld_vol(alive + v)) continue;
    const int64_t d = v / G.E, e = v % G.E;
    bool hin = false, hout = false;
    for (int f = 0; f < G.nfc; ++f) {
      int64_t u, x;
      int fx;
      if (arc_in(G, d, e, f, u) && ld_vol(alive + d * G.E + u)) hin = true;
      if (arc_out(G, d, e, f, x, fx) && ld_vol(alive + d * G.E + x)) hout = true;
    }
    if (!hin || !hout) {
      alive[v] = 0;
      *changed = 1;
    }
  }
}

__global__ void any_alive_kernel(const int8_t* alive, int64_t n, int* flag) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (alive[v]) {
      *flag = 1;
      return;
    }
}

__global__ void color_init_kernel(FasGraph G, const int8_t* alive, int32_t* color, int8_t* mark) {
  const int64_t n = (int64_t)G.M * G.E;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = (int32_t)(v % G.E);
    color[v] = e;
    mark[v] = 0;
    (void)alive;
  }
}

// colour = largest element id among live ancestors (values only grow: a unique fixed point)
__global__ void color_prop_kernel(FasGraph G, const int8_t* alive, int32_t* color, int* changed) {
  const int64_t n = (int64_t)G.M * G.E;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (!alive[v]) continue;
    const int64_t d = v / G.E, e = v % G.E;
    int32_t m = ld_vol(color + v);
    const int32_t m0 = m;
    for (int f = 0; f < G.nfc; ++f) {
      int64_t u;
      if (arc_in(G, d, e, f, u) && alive[d * G.E + u]) m = max(m, ld_vol(color + d * G.E + u));
    }
    if (m > m0) {
      color[v] = m;
      *changed = 1;
    }
  }
}

// roots mark themselves; then a live vertex is marked when a live successor of the same colour is
__global__ void mark_init_kernel(FasGraph G, const int8_t* alive, const int32_t* color, int8_t* mark) {
  const int64_t n = (int64_t)G.M * G.E;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    mark[v] = (alive[v] && color[v] == (int32_t)(v % G.E)) ? 1 : 0;
}

__global__ void mark_prop_kernel(FasGraph G, const int8_t* alive, const int32_t* color, int8_t* mark, int* changed) {
  const int64_t n = (int64_t)G.M * G.E;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (!alive[v] || ld_vol(mark + v)) continue;
    const int64_t d = v / G.E, e = v % G.E;
    for (int f = 0; f < G.nfc; ++f) {
      int64_t x;
      int fx;
      if (arc_out(G, d, e, f, x, fx)) {
        const int64_t w = d * G.E + x;
        if (alive[w] && ld_vol(mark + w) && color[w] == color[v]) {
          mark[v] = 1;
          *changed = 1;
          break;
        }
      }
    }
  }
}

// marked vertices form their root's component: record it and take them out of the live set
__global__ void assign_kernel(FasGraph G, int8_t* alive, const int32_t* color, const int8_t* mark, int32_t* scc,
                              int32_t* size) {
  const int64_t n = (int64_t)G.M * G.E;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (!alive[v] || !mark[v]) continue;
    const int64_t d = v / G.E;
    scc[v] = color[v];
    alive[v] = 0;
    atomicAdd(size + d * G.E + color[v], 1);
  }
}

__global__ void scc_init_kernel(int64_t E, int64_t n, int8_t* alive, int32_t* scc, int32_t* size) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    alive[v] = 1;
    scc[v] = (int32_t)(v % E);
    size[v] = 0;
  }
}

// ---------------------------------------------------------------- component lists
// cnt[0] = components of >= 2 vertices, cnt[1] = their total size, cnt[2] = largest size,
// cnt[3] = subset-DP entries (sum of 2^size over components of at most exact_max vertices)
__global__ void count_roots_kernel(FasGraph G, const int32_t* size, int exact_max, int32_t* sccid,
                                   int64_t* roots, unsigned long long* cnt) {
  const int64_t n = (int64_t)G.M * G.E;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = size[v];
    if (k < 2) continue;
    const unsigned long long slot = atomicAdd(cnt + 0, 1ull);
    roots[slot] = v;
    sccid[v] = (int32_t)slot;
    atomicAdd(cnt + 1, (unsigned long long)k);
    atomicMax(cnt + 2, (unsigned long long)k);
    if (k <= exact_max) atomicAdd(cnt + 3, 1ull << k);
  }
}

// offsets of the member lists and of the DP tables (one thread: the component count is small
// next to the vertex count)
__global__ void offsets_kernel(const int64_t* roots, int64_t nscc, const int32_t* size, int exact_max, int64_t* off,
                               int64_t* dpoff) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t a = 0, b = 0;
  for (int64_t i = 0; i < nscc; ++i) {
    const int32_t k = size[roots[i]];
    off[i] = a;
    dpoff[i] = b;
    a += k;
    if (k <= exact_max) b += (int64_t)1 << k;
  }
  off[nscc] = a;
  dpoff[nscc] = b;
}

__global__ void fill_members_kernel(FasGraph G, const int32_t* scc, const int32_t* size, const int32_t* sccid,
                                    const int64_t* off, int32_t* fill, int32_t* members) {
  const int64_t n = (int64_t)G.M * G.E;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = v / G.E;
    const int64_t r = d * G.E + scc[v];
    if (size[r] < 2) continue;
    const int32_t slot = sccid[r];
    const int32_t pos = atomicAdd(fill + slot, 1);
    members[off[slot] + pos] = (int32_t)(v % G.E);
  }
}

// members of each component in increasing element id (rank = number of smaller ids): one warp
// per component, through the scratch copy tmp
__global__ void sort_members_kernel(const int64_t* off, int64_t nscc, int32_t* members, int32_t* tmp) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= nscc) return;
  const int64_t o = off[c];
  const int n = (int)(off[c + 1] - o);
  for (int i = lane; i < n; i += 32) tmp[o + i] = members[o + i];
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    const int32_t x = tmp[o + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) rank += tmp[o + j] < x;
    members[o + rank] = x;
  }
}

__device__ inline int find_local(const int32_t* m, int n, int32_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (m[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return (lo < n && m[lo] == x) ? lo : -1;
}

// Component neighbours of element e of direction d (root r): one entry per face leading to a
// member, with the arc e -> x (out) and the arc x -> e (in) and their weights.
struct CompNbr {
  int32_t id;
  int32_t out, in;
  double wout, win;
};

__device__ inline int comp_nbrs(const FasGraph& G, int64_t d, int32_t e, int32_t r, const int32_t* scc,
                                CompNbr* nb) {
  int k = 0;
  for (int f = 0; f < G.nfc; ++f) {
    const int64_t x = G.nbr[(int64_t)e * G.nfc + f];
    if (x < 0 || scc[d * G.E + x] != r) continue;
    const int fx = G.nbr_face[(int64_t)e * G.nfc + f];
    CompNbr c;
    c.id = (int32_t)x;
    c.out = face_mode(G.fc[d * G.E + x], fx) != MODE_NONE;         // e -> x, weight at x's face
    c.wout = c.out ? G.win[(d * G.E + x) * G.nfc + fx] : 0.0;
    c.in = face_mode(G.fc[d * G.E + e], f) != MODE_NONE;           // x -> e, weight at e's face
    c.win = c.in ? G.win[(d * G.E + e) * G.nfc + f] : 0.0;
    nb[k++] = c;
  }
  return k;
}

// delta = w_out - w_in over the live neighbours, each sum in increasing neighbour id from 0.0
__device__ inline double live_delta(const CompNbr* nb, int k, const int32_t* m, int n, const int8_t* alive) {
  double wo = 0.0, wi = 0.0;
  int32_t prev = -1;
  for (int t = 0; t < k; ++t) {
    int best = -1;
    for (int s2 = 0; s2 < k; ++s2)
      if (nb[s2].id > prev && (best < 0 || nb[s2].id < nb[best].id)) best = s2;
    prev = nb[best].id;
    if (alive[find_local(m, n, prev)]) {
      if (nb[best].out) wo = wo + nb[best].wout;
      if (nb[best].in) wi = wi + nb[best].win;
    }
  }
  return wo - wi;
}

// ---------------------------------------------------------------- exact FAS (subset DP)
// One warp per component of 2..exact_max vertices; position of each member in the optimal order.
__global__ void fas_dp_kernel(FasGraph G, const int64_t* roots, int64_t nscc, const int32_t* size, int exact_max,
                              const int32_t* scc, const int64_t* off, const int64_t* dpoff, const int32_t* members,
                              double* dpf, int8_t* dppar, int32_t* pos) {
  __shared__ double zl_all[4][16 * 16];
  __shared__ uint8_t has_all[4][16 * 16];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (c >= nscc) return;
  const int64_t r = roots[c];
  const int k = size[r];
  if (k > exact_max) return;
  const int64_t d = r / G.E;
  const int32_t* m = members + off[c];
  double* zl = zl_all[wib];
  uint8_t* has = has_all[wib];
  for (int t = lane; t < k * k; t += 32) {
    zl[t] = 0.0;
    has[t] = 0;
  }
  __syncwarp();
  // arc m[a] -> m[b]: m[b]'s face towards m[a] is an inflow face
  for (int b = lane; b < k; b += 32) {
    const int32_t e = m[b];
    for (int f = 0; f < G.nfc; ++f) {
      int64_t u;
      if (!arc_in(G, d, e, f, u) || scc[d * G.E + u] != (int32_t)(r % G.E)) continue;
      const int a = find_local(m, k, (int32_t)u);
      zl[a * k + b] = G.win[(d * G.E + e) * G.nfc + f];
      has[a * k + b] = 1;
    }
  }
  __syncwarp();
  double* F = dpf + dpoff[c];
  int8_t* par = dppar + dpoff[c];
  const uint32_t full = (1u << k) - 1u;
  if (lane == 0) F[0] = 0.0;
  __syncwarp();
  for (int L = 1; L <= k; ++L) {
    for (uint32_t T = lane; T <= full; T += 32) {
      if (__popc(T) != L) continue;
      double best = 0.0;
      int bv = -1;
      for (int v = k - 1; v >= 0; --v) {       // largest v first: ties keep the largest v
        if (!(T >> v & 1u)) continue;
        double cc = 0.0;
        for (int u = 0; u < k; ++u)
          if (!(T >> u & 1u) && has[u * k + v]) cc = cc + zl[u * k + v];
        const double cand = F[T ^ (1u << v)] + cc;
        if (bv < 0 || cand < best) {
          best = cand;
          bv = v;
        }
      }
      F[T] = best;
      par[T] = (int8_t)bv;
    }
    __syncwarp();
  }
  if (lane == 0) {
    uint32_t T = full;
    int i = 0;
    int32_t* p = pos + off[c];
    while (T) {
      const int v = par[T];
      p[v] = k - 1 - i;          // the order is the reverse of the reconstruction
      ++i;
      T ^= 1u << v;
    }
  }
}

// ---------------------------------------------------------------- Eades-Lin-Smyth
// One warp per component of more than exact_max vertices; per-member state in global scratch.
__global__ void fas_els_kernel(FasGraph G, const int64_t* roots, int64_t nscc, const int32_t* size, int exact_max,
                               const int32_t* scc, const int64_t* off, const int32_t* members, int8_t* alive_g,
                               int32_t* ind_g, int32_t* outd_g, double* delta_g, int32_t* pos) {
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= nscc) return;
  const int64_t r = roots[c];
  const int n = size[r];
  if (n <= exact_max) return;
  const int64_t d = r / G.E;
  const int32_t rr = (int32_t)(r % G.E);
  const int64_t o = off[c];
  const int32_t* m = members + o;
  int8_t* alive = alive_g + o;
  int32_t* ind = ind_g + o;
  int32_t* outd = outd_g + o;
  double* delta = delta_g + o;
  int32_t* p = pos + o;
  constexpr int MAXF = 6;
  for (int i = lane; i < n; i += 32) alive[i] = 1;
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    CompNbr nb[MAXF];
    const int k = comp_nbrs(G, d, m[i], rr, scc, nb);
    int no = 0, ni = 0;
    for (int t = 0; t < k; ++t) {
      no += nb[t].out;
      ni += nb[t].in;
    }
    outd[i] = no;
    ind[i] = ni;
    delta[i] = live_delta(nb, k, m, n, alive);
  }
  __syncwarp();
  int n1 = 0, n2 = 0, left = n;
  // remove member a (lane 0 updates the neighbours; the others wait)
  auto remove = [&](int a, bool as_sink) {
    if (lane == 0) {
      alive[a] = 0;
      p[a] = as_sink ? n - 1 - n2 : n1;
      CompNbr nb[MAXF];
      const int k = comp_nbrs(G, d, m[a], rr, scc, nb);
      for (int t = 0; t < k; ++t) {
        const int j = find_local(m, n, nb[t].id);
        if (!alive[j]) continue;
        if (nb[t].out) --ind[j];               // a -> j: j loses an in-arc
        if (nb[t].in) --outd[j];               // j -> a: j loses an out-arc
        CompNbr nj[MAXF];
        const int kj = comp_nbrs(G, d, m[j], rr, scc, nj);
        delta[j] = live_delta(nj, kj, m, n, alive);
      }
    }
    if (as_sink) ++n2;
    else ++n1;
    --left;
    __syncwarp();
  };
  // smallest live index with outd == 0 (sinks) or ind == 0 (sources), -1 if none
  auto first_with = [&](bool sinks) {
    int best = 0x7fffffff;
    for (int i = lane; i < n; i += 32)
      if (alive[i] && (sinks ? outd[i] : ind[i]) == 0) {
        best = i;
        break;
      }
    best = __reduce_min_sync(0xffffffffu, (unsigned)best);
    return best == 0x7fffffff ? -1 : best;
  };
  while (left > 0) {
    for (int a = first_with(true); a >= 0; a = first_with(true)) remove(a, true);
    for (int a = first_with(false); a >= 0; a = first_with(false)) remove(a, false);
    if (left > 0) {
      // largest delta, ties smallest index
      double bd = 0.0;
      int bi = -1;
      for (int i = lane; i < n; i += 32)
        if (alive[i] && (bi < 0 || delta[i] > bd)) {
          bd = delta[i];
          bi = i;
        }
      for (int sh = 16; sh > 0; sh >>= 1) {
        const double od = __shfl_xor_sync(0xffffffffu, bd, sh);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, sh);
        if (oi >= 0 && (bi < 0 || od > bd || (od == bd && oi < bi))) {
          bd = od;
          bi = oi;
        }
      }
      remove(bi, false);
    }
  }
}

// lag bit of every arc whose source comes after its destination in its component's order
__global__ void set_lags_kernel(FasGraph G, uint32_t* fc, const int64_t* roots, int64_t nscc, const int32_t* size,
                                const int32_t* scc, const int64_t* off, const int32_t* members, const int32_t* pos,
                                unsigned long long* nremoved) {
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= nscc) return;
  const int64_t r = roots[c];
  const int n = size[r];
  const int64_t d = r / G.E;
  const int32_t rr = (int32_t)(r % G.E);
  const int32_t* m = members + off[c];
  const int32_t* p = pos + off[c];
  for (int b = lane; b < n; b += 32) {           // destination m[b]
    const int32_t e = m[b];
    uint32_t bits = 0;
    for (int f = 0; f < G.nfc; ++f) {
      int64_t u;
      if (!arc_in(G, d, e, f, u) || scc[d * G.E + u] != rr) continue;
      const int a = find_local(m, n, (int32_t)u);
      if (p[a] > p[b]) bits |= 1u << (16 + f);
    }
    if (bits) {
      atomicOr(fc + d * G.E + e, bits);
      atomicAdd(nremoved, (unsigned long long)__popc(bits));
    }
  }
}

template <class T>
cudaError_t alloc_n(T*& p, size_t n) {
  p = nullptr;
  return cudaMalloc((void**)&p, std::max<size_t>(1, n) * sizeof(T));
}

}  // namespace

// Runs the component search and the per-component FAS for all directions; sets the lag bits of
// the removed arcs in fc.  Iterated steps run in rounds of 8 launches between checks of a
// device flag.  Returns cudaErrorUnknown (with stats->stuck = 1) if a fixed point is not reached
// within the bound the graph size implies.
cudaError_t device_fas(const DevProblem& P, uint32_t* fc, const double* win, int exact_max, DeviceFasStats* stats,
                       cudaStream_t s) {
  FasGraph G{P.M, P.nfc, P.E, P.nbr, P.nbr_face, fc, win};
  const int64_t n = (int64_t)P.M * P.E;
  const unsigned grid = 1216, block = 256;
  int8_t *alive = nullptr, *mark = nullptr;
  int32_t *color = nullptr, *scc = nullptr, *size = nullptr, *sccid = nullptr;
  int* flag = nullptr;
  unsigned long long* cnt = nullptr;
  int64_t* roots = nullptr;
  cudaError_t e = cudaSuccess;
  *stats = DeviceFasStats{};
#define FAS_TRY(x)                \
  do {                            \
    e = (x);                      \
    if (e != cudaSuccess) goto done; \
  } while (0)
  FAS_TRY(alloc_n(alive, n));
  FAS_TRY(alloc_n(mark, n));
  FAS_TRY(alloc_n(color, n));
  FAS_TRY(alloc_n(scc, n));
  FAS_TRY(alloc_n(size, n));
  FAS_TRY(alloc_n(sccid, n));
  FAS_TRY(alloc_n(flag, 1));
  FAS_TRY(alloc_n(cnt, 5));
  FAS_TRY(alloc_n(roots, n / 2 + 1));
  {
    scc_init_kernel<<<grid, block, 0, s>>>(P.E, n, alive, scc, size);
    const int64_t bound = 4 * P.E + 64;            // rounds of any fixed-point loop
    int64_t total = 0;
    // launches `step` until a round of 8 leaves the flag clear
    auto until_stable = [&](auto step) -> cudaError_t {
      for (int64_t it = 0;; it += 8) {
        cudaError_t ee = cudaMemsetAsync(flag, 0, sizeof(int), s);
        if (ee != cudaSuccess) return ee;
        for (int k = 0; k < 8; ++k) step();
        int h = 0;
        ee = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (ee == cudaSuccess) ee = cudaStreamSynchronize(s);
        if (ee != cudaSuccess) return ee;
        total += 8;
        if (!h) return cudaSuccess;
        if (it > bound) {
          stats->stuck = 1;
          return cudaErrorUnknown;
        }
      }
    };
    auto trim = [&]() { trim_kernel<<<grid, block, 0, s>>>(G, alive, flag); };
    FAS_TRY(until_stable(trim));
    for (int64_t round = 0;; ++round) {
      int h = 0;
      FAS_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
      any_alive_kernel<<<grid, block, 0, s>>>(alive, n, flag);
      FAS_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      FAS_TRY(cudaStreamSynchronize(s));
      if (!h) break;
      if (round > bound) {
        stats->stuck = 1;
        e = cudaErrorUnknown;
        goto done;
      }
      color_init_kernel<<<grid, block, 0, s>>>(G, alive, color, mark);
      FAS_TRY(until_stable([&]() { color_prop_kernel<<<grid, block, 0, s>>>(G, alive, color, flag); }));
      mark_init_kernel<<<grid, block, 0, s>>>(G, alive, color, mark);
      FAS_TRY(until_stable([&]() { mark_prop_kernel<<<grid, block, 0, s>>>(G, alive, color, mark, flag); }));
      assign_kernel<<<grid, block, 0, s>>>(G, alive, color, mark, scc, size);
      FAS_TRY(until_stable(trim));
    }
    stats->launches += total;
    // component lists
    FAS_TRY(cudaMemsetAsync(cnt, 0, 5 * sizeof(unsigned long long), s));
    count_roots_kernel<<<grid, block, 0, s>>>(G, size, exact_max, sccid, roots, cnt);
    unsigned long long hc[4];
    FAS_TRY(cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s));
    FAS_TRY(cudaStreamSynchronize(s));
    const int64_t nscc = (int64_t)hc[0], nmem = (int64_t)hc[1], ndp = (int64_t)hc[3];
    stats->n_scc = nscc;
    stats->max_scc = (int32_t)hc[2];
    if (nscc > 0) {
      int64_t *off = nullptr, *dpoff = nullptr;
      int32_t *members = nullptr, *tmp = nullptr, *fill = nullptr, *pos = nullptr, *ind = nullptr, *outd = nullptr;
      int8_t *dppar = nullptr, *alive2 = nullptr;
      double *dpf = nullptr, *delta = nullptr;
      cudaError_t e2 = cudaSuccess;
      const unsigned warps_grid = (unsigned)((nscc + 3) / 4);
      if ((e2 = alloc_n(off, nscc + 1)) == cudaSuccess && (e2 = alloc_n(dpoff, nscc + 1)) == cudaSuccess &&
          (e2 = alloc_n(members, nmem)) == cudaSuccess && (e2 = alloc_n(tmp, nmem)) == cudaSuccess &&
          (e2 = alloc_n(fill, nscc)) == cudaSuccess && (e2 = alloc_n(pos, nmem)) == cudaSuccess &&
          (e2 = alloc_n(ind, nmem)) == cudaSuccess && (e2 = alloc_n(outd, nmem)) == cudaSuccess &&
          (e2 = alloc_n(alive2, nmem)) == cudaSuccess && (e2 = alloc_n(delta, nmem)) == cudaSuccess &&
          (e2 = alloc_n(dpf, ndp)) == cudaSuccess && (e2 = alloc_n(dppar, ndp)) == cudaSuccess &&
          (e2 = cudaMemsetAsync(fill, 0, nscc * sizeof(int32_t), s)) == cudaSuccess) {
        offsets_kernel<<<1, 1, 0, s>>>(roots, nscc, size, exact_max, off, dpoff);
        fill_members_kernel<<<grid, block, 0, s>>>(G, scc, size, sccid, off, fill, members);
        sort_members_kernel<<<warps_grid, 128, 0, s>>>(off, nscc, members, tmp);
        fas_dp_kernel<<<warps_grid, 128, 0, s>>>(G, roots, nscc, size, exact_max, scc, off, dpoff, members, dpf, dppar,
                                                  pos);
        fas_els_kernel<<<warps_grid, 128, 0, s>>>(G, roots, nscc, size, exact_max, scc, off, members, alive2, ind, outd,
                                                   delta, pos);
        set_lags_kernel<<<warps_grid, 128, 0, s>>>(G, fc, roots, nscc, size, scc, off, members, pos, cnt + 4);
        e2 = cudaGetLastError();
        unsigned long long nr = 0;
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(&nr, cnt + 4, sizeof(nr), cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
        stats->n_removed = (int64_t)nr;
        stats->launches += 6;
      }
      cudaFree(off);
      cudaFree(dpoff);
      cudaFree(members);
      cudaFree(tmp);
      cudaFree(fill);
      cudaFree(pos);
      cudaFree(ind);
      cudaFree(outd);
      cudaFree(alive2);
      cudaFree(delta);
      cudaFree(dpf);
      cudaFree(dppar);
      e = e2;
    }
  }
done:
#undef FAS_TRY
  cudaFree(alive);
  cudaFree(mark);
  cudaFree(color);
  cudaFree(scc);
  cudaFree(size);
  cudaFree(sccid);
  cudaFree(flag);
  cudaFree(cnt);
  cudaFree(roots);
  return e;
}

}  // namespace sn
