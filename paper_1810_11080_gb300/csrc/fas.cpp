// Cycle breaking of one direction's dependency graph (Sec. 3, last two paragraphs):
// Tarjan SCCs; per SCC a minimum-weight feedback arc set -- exact by dynamic programming
// over vertex subsets on SCCs of at most exact_max vertices (the paper's integer program on
// SCCs of 'say 10' vertices), the weighted Eades-Lin-Smyth heuristic on larger ones.
// Compiled with -ffp-contract=off: weight sums follow the stated order so that the removed
// set is a deterministic function of the weights.
#include <algorithm>
#include <limits>
#include <set>
#include <utility>
#include "common.h"

namespace sn {

namespace {

struct Csr {
  std::vector<int64_t> off;
  std::vector<int32_t> nb;
  std::vector<double> w;
  std::vector<int64_t> arc;   // index into the caller's arc list
};

// CSR of successors (by_src = true) or predecessors, neighbours ascending.
Csr make_csr(int64_t n, const std::vector<int32_t>& a, const std::vector<int32_t>& b,
             const std::vector<double>& z, const std::vector<int64_t>& arcs) {
  Csr c;
  c.off.assign(n + 1, 0);
  for (int64_t i : arcs) c.off[a[i] + 1]++;
  for (int64_t v = 0; v < n; ++v) c.off[v + 1] += c.off[v];
  c.nb.resize(arcs.size());
  c.w.resize(arcs.size());
  c.arc.resize(arcs.size());
  std::vector<int64_t> pos(c.off.begin(), c.off.end() - 1);
  for (int64_t i : arcs) {
    int64_t k = pos[a[i]]++;
    c.nb[k] = b[i];
    c.w[k] = z[i];
    c.arc[k] = i;
  }
  for (int64_t v = 0; v < n; ++v) {
    std::vector<std::pair<int32_t, int64_t>> tmp;
    for (int64_t k = c.off[v]; k < c.off[v + 1]; ++k) tmp.push_back({c.nb[k], k});
    std::sort(tmp.begin(), tmp.end());
    std::vector<int32_t> nb2;
    std::vector<double> w2;
    std::vector<int64_t> a2;
    for (auto& t : tmp) {
      nb2.push_back(c.nb[t.second]);
      w2.push_back(c.w[t.second]);
      a2.push_back(c.arc[t.second]);
    }
    std::copy(nb2.begin(), nb2.end(), c.nb.begin() + c.off[v]);
    std::copy(w2.begin(), w2.end(), c.w.begin() + c.off[v]);
    std::copy(a2.begin(), a2.end(), c.arc.begin() + c.off[v]);
  }
  return c;
}

// Iterative Tarjan; comp[v] = component id.  Returns the number of components.
int64_t tarjan(int64_t n, const Csr& succ, std::vector<int64_t>& comp) {
  std::vector<int64_t> index(n, -1), low(n, 0);
  std::vector<char> onstack(n, 0);
  std::vector<int32_t> stack;
  std::vector<std::pair<int32_t, int64_t>> work;
  comp.assign(n, -1);
  int64_t counter = 0, ncomp = 0;
  for (int64_t root = 0; root < n; ++root) {
    if (index[root] != -1) continue;
    index[root] = low[root] = counter++;
    stack.push_back((int32_t)root);
    onstack[root] = 1;
    work.push_back({(int32_t)root, succ.off[root]});
    while (!work.empty()) {
      int32_t v = work.back().first;
      int64_t& it = work.back().second;
      if (it < succ.off[v + 1]) {
        int32_t w = succ.nb[it++];
        if (index[w] == -1) {
          index[w] = low[w] = counter++;
          stack.push_back(w);
          onstack[w] = 1;
          work.push_back({w, succ.off[w]});
        } else if (onstack[w]) {
          low[v] = std::min(low[v], index[w]);
        }
      } else {
        work.pop_back();
        if (!work.empty()) {
          int32_t u = work.back().first;
          low[u] = std::min(low[u], low[v]);
        }
        if (low[v] == index[v]) {
          while (true) {
            int32_t w = stack.back();
            stack.pop_back();
            onstack[w] = 0;
            comp[w] = ncomp;
            if (w == v) break;
          }
          ++ncomp;
        }
      }
    }
  }
  return ncomp;
}

// Exact minimum FAS by DP over subsets: cost(S + {v}) = cost(S) + sum_{u not in S+{v}} z(u->v),
// u increasing from 0.0; S by increasing bitmask, v by increasing local index, strict <.
void fas_exact(const std::vector<int32_t>& verts, const std::vector<std::vector<double>>& zl,
               const std::vector<std::vector<char>>& has, std::vector<int>& order) {
  const int n = (int)verts.size();
  const uint32_t full = (1u << n) - 1u;
  std::vector<double> f(1u << n, std::numeric_limits<double>::infinity());
  std::vector<int8_t> par(1u << n, -1);
  f[0] = 0.0;
  for (uint32_t S = 0; S <= full; ++S) {
    if (f[S] == std::numeric_limits<double>::infinity()) continue;
    for (int v = 0; v < n; ++v) {
      if (S >> v & 1u) continue;
      uint32_t T = S | (1u << v);
      double c = 0.0;
      for (int u = 0; u < n; ++u)
        if (!(T >> u & 1u) && has[u][v]) c = c + zl[u][v];
      double cand = f[S] + c;
      if (cand < f[T]) {
        f[T] = cand;
        par[T] = (int8_t)v;
      }
    }
  }
  order.clear();
  uint32_t T = full;
  while (T) {
    int v = par[T];
    order.push_back(v);
    T ^= 1u << v;
  }
  std::reverse(order.begin(), order.end());
}

// Weighted Eades-Lin-Smyth on one SCC (global ids, adjacency restricted to the SCC):
// smallest-id sinks are prepended to s2, smallest-id sources appended to s1, otherwise the
// vertex of largest delta = w_out - w_in (ties: smallest id) is appended to s1.  w_out/w_in sum
// over remaining neighbours in increasing id from 0.0.
void fas_els(const std::vector<int32_t>& verts, const Csr& succ, const Csr& pred,
             const std::vector<int64_t>& comp, int64_t cid, std::vector<int32_t>& order) {
  std::set<int32_t> sinks, sources;
  std::set<std::pair<double, int32_t>> byd;   // (-delta, id)
  std::vector<char> rem_flag;                 // indexed by position in verts via map
  // local maps
  std::vector<int32_t> sorted = verts;
  std::sort(sorted.begin(), sorted.end());
  auto loc = [&](int32_t v) { return (int64_t)(std::lower_bound(sorted.begin(), sorted.end(), v) - sorted.begin()); };
  const int64_t n = (int64_t)sorted.size();
  std::vector<char> alive(n, 1);
  std::vector<int64_t> outd(n, 0), ind(n, 0);
  std::vector<double> delta(n, 0.0);
  auto in_scc = [&](int32_t v) { return comp[v] == cid; };
  auto compute_delta = [&](int32_t v) {
    double wo = 0.0, wi = 0.0;
    for (int64_t k = succ.off[v]; k < succ.off[v + 1]; ++k) {
      int32_t t = succ.nb[k];
      if (in_scc(t) && alive[loc(t)]) wo = wo + succ.w[k];
    }
    for (int64_t k = pred.off[v]; k < pred.off[v + 1]; ++k) {
      int32_t s = pred.nb[k];
      if (in_scc(s) && alive[loc(s)]) wi = wi + pred.w[k];
    }
    return wo - wi;
  };
  for (int64_t i = 0; i < n; ++i) {
    int32_t v = sorted[i];
    for (int64_t k = succ.off[v]; k < succ.off[v + 1]; ++k)
      if (in_scc(succ.nb[k])) outd[i]++;
    for (int64_t k = pred.off[v]; k < pred.off[v + 1]; ++k)
      if (in_scc(pred.nb[k])) ind[i]++;
    if (outd[i] == 0) sinks.insert(v);
    if (ind[i] == 0) sources.insert(v);
    delta[i] = compute_delta(v);
    byd.insert({-delta[i], v});
  }
  std::vector<int32_t> s1, s2rev;
  auto remove_vertex = [&](int32_t v) {
    int64_t i = loc(v);
    alive[i] = 0;
    sinks.erase(v);
    sources.erase(v);
    byd.erase({-delta[i], v});
    for (int64_t k = succ.off[v]; k < succ.off[v + 1]; ++k) {
      int32_t t = succ.nb[k];
      if (!in_scc(t)) continue;
      int64_t j = loc(t);
      if (!alive[j]) continue;
      if (--ind[j] == 0) sources.insert(t);
      byd.erase({-delta[j], t});
      delta[j] = compute_delta(t);
      byd.insert({-delta[j], t});
    }
    for (int64_t k = pred.off[v]; k < pred.off[v + 1]; ++k) {
      int32_t s = pred.nb[k];
      if (!in_scc(s)) continue;
      int64_t j = loc(s);
      if (!alive[j]) continue;
      if (--outd[j] == 0) sinks.insert(s);
      byd.erase({-delta[j], s});
      delta[j] = compute_delta(s);
      byd.insert({-delta[j], s});
    }
  };
  int64_t left = n;
  while (left > 0) {
    while (!sinks.empty()) {
      int32_t v = *sinks.begin();
      remove_vertex(v);
      s2rev.push_back(v);
      --left;
    }
    while (!sources.empty()) {
      int32_t v = *sources.begin();
      remove_vertex(v);
      s1.push_back(v);
      --left;
    }
    if (left > 0) {
      int32_t u = byd.begin()->second;
      remove_vertex(u);
      s1.push_back(u);
      --left;
    }
  }
  order = s1;
  for (auto it = s2rev.rbegin(); it != s2rev.rend(); ++it) order.push_back(*it);
}

}  // namespace

FasStats break_cycles(int64_t n, const std::vector<int32_t>& src, const std::vector<int32_t>& dst,
                      const std::vector<double>& z, int exact_max, std::vector<uint8_t>& removed) {
  FasStats st;
  const int64_t m = (int64_t)src.size();
  removed.assign(m, 0);
  std::vector<int64_t> all(m);
  for (int64_t i = 0; i < m; ++i) all[i] = i;
  Csr succ = make_csr(n, src, dst, z, all);
  Csr pred = make_csr(n, dst, src, z, all);
  std::vector<int64_t> comp;
  int64_t ncomp = tarjan(n, succ, comp);
  std::vector<int64_t> csize(ncomp, 0);
  for (int64_t v = 0; v < n; ++v) csize[comp[v]]++;
  std::vector<std::vector<int32_t>> members(ncomp);
  for (int64_t v = 0; v < n; ++v)
    if (csize[comp[v]] > 1) members[comp[v]].push_back((int32_t)v);
  for (int64_t c = 0; c < ncomp; ++c) {
    const auto& verts = members[c];
    if (verts.size() < 2) continue;
    st.n_scc++;
    st.max_scc = std::max<int32_t>(st.max_scc, (int32_t)verts.size());
    std::vector<int32_t> gorder;
    if ((int)verts.size() <= exact_max) {
      const int k = (int)verts.size();
      std::vector<std::vector<double>> zl(k, std::vector<double>(k, 0.0));
      std::vector<std::vector<char>> has(k, std::vector<char>(k, 0));
      for (int a = 0; a < k; ++a) {
        int32_t u = verts[a];
        for (int64_t e = succ.off[u]; e < succ.off[u + 1]; ++e) {
          int32_t v = succ.nb[e];
          if (comp[v] != c) continue;
          int b = (int)(std::lower_bound(verts.begin(), verts.end(), v) - verts.begin());
          zl[a][b] = succ.w[e];
          has[a][b] = 1;
        }
      }
      std::vector<int> lorder;
      fas_exact(verts, zl, has, lorder);
      for (int v : lorder) gorder.push_back(verts[v]);
    } else {
      fas_els(verts, succ, pred, comp, c, gorder);
    }
    // position in order; removed = arcs whose source comes after their destination
    std::vector<int64_t> posv(verts.size());
    for (size_t i = 0; i < gorder.size(); ++i) {
      int64_t l = std::lower_bound(verts.begin(), verts.end(), gorder[i]) - verts.begin();
      posv[l] = (int64_t)i;
    }
    for (int32_t u : verts) {
      int64_t pu = posv[std::lower_bound(verts.begin(), verts.end(), u) - verts.begin()];
      for (int64_t e = succ.off[u]; e < succ.off[u + 1]; ++e) {
        int32_t v = succ.nb[e];
        if (comp[v] != c) continue;
        int64_t pv = posv[std::lower_bound(verts.begin(), verts.end(), v) - verts.begin()];
        if (pu > pv) removed[succ.arc[e]] = 1;
      }
    }
  }
  return st;
}

}  // namespace sn
