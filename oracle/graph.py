"""Upwind dependency graph, cycle breaking and sweep levels (paper Sec. 3).

Per direction d: one vertex per element; an arc e' -> e ("e depends on e'") whenever
Fbar^{(d)}_{e,e'} != 0, i.e. max_ij |Fbar_ij| > 0 (Sec. 3, graph definition).
Weights z (Sec. 3, enumerated list and eq. 22): unity; face = max_ij |Fbar_{e,e'}|;
siginvface = max_ij |(M_{t,e})^{-1} Fbar_{e,e'}| (max-entry norm).

Cycle breaking (Sec. 3, last paragraphs): Tarjan SCCs; on each SCC independently a minimum
feedback arc set -- exact on SCCs of at most `exact_max` vertices (the paper's 'say 10'),
the Eades-Lin-Smyth heuristic above that.  The arcs are removed from the sweep graph and
their dependencies lagged (eq. 21).

Reading of the FAS objective (Sec. 3 prints 'forward edges e' > e' but sums over e' < e):
for a linear order of the vertices, a removed (lagged) arc is one whose upwind vertex e'
comes after its dependent e, i.e. the block upper part F_> of eq. 20; the order minimises
the summed weight of those arcs.

Levels (not in the paper; the sweep order it leaves free): longest-path layering of the
kept acyclic graph, level(e) = 0 without kept in-arcs, else 1 + max level of kept upwind
neighbours.
"""
import numpy as np
from .basis import lu_factor, lu_solve
from .dg import Discretization

WEIGHTINGS = {"unity": 0, "face": 1, "siginvface": 2}


def lu_factor_batch(A):
    """lu_factor applied to each matrix of A [B, n, n]: the same pivot rule (first row of
    largest |A[i][k]|) and the same elementwise operation order, vectorised over B."""
    A = np.array(A, dtype=np.float64, copy=True)
    B, n, _ = A.shape
    perm = np.tile(np.arange(n), (B, 1))
    ar = np.arange(B)
    for k in range(n):
        p = k + np.argmax(np.abs(A[:, k:, k]), axis=1)
        if np.any(A[ar, p, k] == 0.0):
            raise np.linalg.LinAlgError("singular matrix in lu_factor_batch")
        rk = A[ar, k, :].copy()
        A[ar, k, :] = A[ar, p, :]
        A[ar, p, :] = rk
        pk = perm[ar, k].copy()
        perm[ar, k] = perm[ar, p]
        perm[ar, p] = pk
        for i in range(k + 1, n):
            l = A[:, i, k] / A[:, k, k]
            A[:, i, k] = l
            for j in range(k + 1, n):
                A[:, i, j] = A[:, i, j] - l * A[:, k, j]
    return A, perm


def lu_solve_batch(LU, perm, b):
    """lu_solve for each item of a batch: LU [B, n, n], perm [B, n], b [B, n]."""
    B, n, _ = LU.shape
    y = np.take_along_axis(b, perm, axis=1).copy()
    for i in range(n):
        for j in range(i):
            y[:, i] = y[:, i] - LU[:, i, j] * y[:, j]
    for i in range(n - 1, -1, -1):
        for j in range(i + 1, n):
            y[:, i] = y[:, i] - LU[:, i, j] * y[:, j]
        y[:, i] = y[:, i] / LU[:, i, i]
    return y


def max_abs(x, axes):
    return np.max(np.abs(x), axis=axes) if x.size else np.zeros(x.shape[:-len(axes)])


def edge_weights(disc, dirs, weighting):
    """Arcs and weights for the directions in `dirs`.

    Returns a list (one entry per direction) of (src, dst, z) int64/int64/float64 arrays:
    src = upwind element e', dst = dependent element e, sorted by (dst, src).
    """
    fb = disc.face_blocks(dirs)
    iface = np.array(disc.iface, dtype=np.int64).reshape(-1, 5)
    N = disc.N
    wcode = WEIGHTINGS[weighting]
    zo_face = max_abs(fb["bar_o"], (2, 3))       # [F, D]: owner <- neighbour
    zn_face = max_abs(fb["bar_n"], (2, 3))       # neighbour <- owner
    if wcode == 2:
        zo = _siginv(disc, iface[:, 0], iface[:, 1], iface[:, 3], fb["bar_o"])
        zn = _siginv(disc, iface[:, 2], iface[:, 3], iface[:, 1], fb["bar_n"])
    out = []
    for j in range(len(dirs)):
        eo = zo_face[:, j] > 0.0
        en = zn_face[:, j] > 0.0
        if wcode == 0:
            wo, wn = np.ones(len(iface)), np.ones(len(iface))
        elif wcode == 1:
            wo, wn = zo_face[:, j], zn_face[:, j]
        else:
            wo, wn = zo[:, j], zn[:, j]
        src = np.concatenate([iface[eo, 2], iface[en, 0]])
        dst = np.concatenate([iface[eo, 0], iface[en, 2]])
        z = np.concatenate([wo[eo], wn[en]])
        order = np.lexsort((src, dst))
        out.append((src[order], dst[order], z[order]))
    return out


def _siginv(disc, recv, recv_face, up_face, bar):
    """max |M_{t,recv}^{-1} Fbar_full| for each face and direction slot (eq. 22).

    M_t = sigma_t * M with M in the fixed order of Discretization.mass_exact_order;
    each of the N_f nonzero columns of the full N x N Fbar (rows at the receiving
    element's face nodes) is solved by the plain pivoted LU."""
    N, Nf = disc.N, disc.Nf
    F, D = bar.shape[:2]
    uniq, inv = np.unique(recv, return_inverse=True)
    M = disc.mass_exact_order(uniq)
    Mt = disc.prob.sigma_t[uniq][:, None, None] * M
    LU, perm = lu_factor_batch(Mt)
    out = np.zeros((F, D))
    for f in range(disc.n_faces):
        sel = np.nonzero(recv_face == f)[0]
        if len(sel) == 0:
            continue
        rows = disc.fnode[f]
        for j in range(D):
            for c in range(Nf):
                b = np.zeros((len(sel), N))
                b[:, rows] = bar[sel, j, :, c]
                x = lu_solve_batch(LU[inv[sel]], perm[inv[sel]], b)
                out[sel, j] = np.maximum(out[sel, j], np.max(np.abs(x), axis=1))
    return out


# ---------------------------------------------------------------- SCC / FAS

def tarjan_scc(n, succ):
    """Strongly connected components (Tarjan 1972), iterative.  succ[v] = successors of v.
    Returns a list of SCCs, each a sorted list of vertices."""
    index = [-1] * n
    low = [0] * n
    onstack = [False] * n
    stack, comps = [], []
    counter = 0
    for root in range(n):
        if index[root] != -1:
            continue
        work = [(root, 0)]
        index[root] = low[root] = counter
        counter += 1
        stack.append(root)
        onstack[root] = True
        while work:
            v, i = work[-1]
            if i < len(succ[v]):
                work[-1] = (v, i + 1)
                w = succ[v][i]
                if index[w] == -1:
                    index[w] = low[w] = counter
                    counter += 1
                    stack.append(w)
                    onstack[w] = True
                    work.append((w, 0))
                elif onstack[w]:
                    low[v] = min(low[v], index[w])
            else:
                work.pop()
                if work:
                    u = work[-1][0]
                    low[u] = min(low[u], low[v])
                if low[v] == index[v]:
                    comp = []
                    while True:
                        w = stack.pop()
                        onstack[w] = False
                        comp.append(w)
                        if w == v:
                            break
                    comps.append(sorted(comp))
    return comps


def fas_exact(verts, z):
    """Exact minimum-weight feedback arc set on a small vertex set by dynamic programming
    over subsets (replaces the paper's integer program, same optimum).

    verts: sorted global ids (local index = position).  z: dict (u, v) -> weight of arc u -> v.
    cost(S + {v}) = cost(S) + sum_{u not in S + {v}} z(u -> v)   (u increasing, from 0.0):
    v is placed right after the set S, so its in-arcs from vertices placed later are lagged.
    S runs over increasing bitmasks, v over increasing local index; a strictly smaller
    cost replaces the stored one.  The order is rebuilt backwards from the full set.
    Returns (order as global ids, removed arcs as (u, v) global pairs).
    """
    n = len(verts)
    zl = [[0.0] * n for _ in range(n)]
    has = [[False] * n for _ in range(n)]
    for a in range(n):
        for b in range(n):
            if (verts[a], verts[b]) in z:
                zl[a][b] = z[(verts[a], verts[b])]
                has[a][b] = True
    full = (1 << n) - 1
    INF = float("inf")
    f = [INF] * (1 << n)
    par = [-1] * (1 << n)
    f[0] = 0.0
    for S in range(1 << n):
        if f[S] == INF:
            continue
        for v in range(n):
            if S >> v & 1:
                continue
            T = S | (1 << v)
            c = 0.0
            for u in range(n):
                if not (T >> u & 1) and has[u][v]:
                    c = c + zl[u][v]
            cand = f[S] + c
            if cand < f[T]:
                f[T] = cand
                par[T] = v
    order = []
    T = full
    while T:
        v = par[T]
        order.append(v)
        T ^= 1 << v
    order.reverse()
    pos = {v: i for i, v in enumerate(order)}
    removed = [(verts[u], verts[v]) for u in range(n) for v in range(n)
               if has[u][v] and pos[u] > pos[v]]
    return [verts[v] for v in order], removed


def fas_els(verts, z):
    """Weighted Eades-Lin-Smyth (1993) heuristic on one SCC.

    Arc u -> v (v depends on u).  Repeat until no vertex is left: (1) while a sink exists,
    remove the smallest-id sink and prepend it to s2; (2) while a source exists, remove the
    smallest-id source and append it to s1; (3) if vertices remain, remove the vertex with
    the largest delta(u) = w_out(u) - w_in(u) (ties: smallest id) and append it to s1.
    w_out / w_in sum the weights of arcs to / from remaining vertices, in increasing
    neighbour id from 0.0.  Order = s1 + s2; arcs pointing backwards in it are removed.
    """
    vs = set(verts)
    outs = {v: [] for v in verts}
    ins = {v: [] for v in verts}
    for (u, v), w in z.items():
        if u in vs and v in vs:
            outs[u].append((v, w))
            ins[v].append((u, w))
    for v in verts:
        outs[v].sort()
        ins[v].sort()
    rem = set(verts)
    s1, s2 = [], []
    while rem:
        while True:
            sink = None
            for v in sorted(rem):
                if not any(t in rem for t, _ in outs[v]):
                    sink = v
                    break
            if sink is None:
                break
            rem.discard(sink)
            s2.insert(0, sink)
        while True:
            src = None
            for v in sorted(rem):
                if not any(s in rem for s, _ in ins[v]):
                    src = v
                    break
            if src is None:
                break
            rem.discard(src)
            s1.append(src)
        if rem:
            best, bu = None, None
            for u in sorted(rem):
                wo = 0.0
                for t, w in outs[u]:
                    if t in rem:
                        wo = wo + w
                wi = 0.0
                for s, w in ins[u]:
                    if s in rem:
                        wi = wi + w
                dl = wo - wi
                if best is None or dl > best:
                    best, bu = dl, u
            rem.discard(bu)
            s1.append(bu)
    order = s1 + s2
    pos = {v: i for i, v in enumerate(order)}
    removed = [(u, v) for (u, v) in z if u in vs and v in vs and pos[u] > pos[v]]
    return order, sorted(removed, key=lambda a: (a[1], a[0]))


def levels_from_kept(n, src, dst, keep):
    """Longest-path layering of the kept arcs (Kahn order).  Returns int array [n]."""
    preds = [[] for _ in range(n)]
    succs = [[] for _ in range(n)]
    indeg = [0] * n
    for u, v, k in zip(src.tolist(), dst.tolist(), keep.tolist()):
        if k:
            preds[v].append(u)
            succs[u].append(v)
            indeg[v] += 1
    level = [0] * n
    frontier = [v for v in range(n) if indeg[v] == 0]
    seen = 0
    while frontier:
        nxt = []
        for v in frontier:
            seen += 1
            for w in succs[v]:
                level[w] = max(level[w], level[v] + 1)
                indeg[w] -= 1
                if indeg[w] == 0:
                    nxt.append(w)
        frontier = nxt
    if seen != n:
        raise RuntimeError("kept graph is not acyclic")
    return np.array(level, dtype=np.int32)


def break_cycles(n, src, dst, z, exact_max=10):
    """Removed arcs (as a boolean mask over the arc list) and SCC sizes (> 1) of one direction."""
    succ = [[] for _ in range(n)]
    for u, v in zip(src.tolist(), dst.tolist()):
        succ[u].append(v)
    for v in range(n):
        succ[v].sort()
    comps = tarjan_scc(n, succ)
    comp_of = np.zeros(n, dtype=np.int64)
    for ci, c in enumerate(comps):
        comp_of[c] = ci
    removed = set()
    sizes = []
    arcs = {}
    same = comp_of[src] == comp_of[dst]
    for u, v, w, s in zip(src.tolist(), dst.tolist(), z.tolist(), same.tolist()):
        if s:
            arcs.setdefault(int(comp_of[u]), {})[(u, v)] = w
    for ci, c in enumerate(comps):
        if len(c) < 2:
            continue
        sizes.append(len(c))
        zc = arcs.get(ci, {})
        if len(c) <= exact_max:
            _o, rm = fas_exact(c, zc)
        else:
            _o, rm = fas_els(c, zc)
        removed.update(rm)
    mask = np.array([(u, v) in removed for u, v in zip(src.tolist(), dst.tolist())], dtype=bool)
    return mask, sorted(sizes)


def build_graph(disc, weighting="face", exact_max=10, chunk=4):
    """The full graph stage for every direction of `disc`.

    Returns dict with
      arcs[d]    = (src, dst, z) sorted by (dst, src)
      removed    = int64 [k, 3] rows (d, e, e') sorted: e depends on e', lagged
      levels     = int32 [M, E]
      scc_sizes  = list per direction of the sizes of non-trivial SCCs
    """
    M, E = disc.M_dirs, disc.E
    arcs = []
    for d0 in range(0, M, chunk):
        arcs += edge_weights(disc, list(range(d0, min(M, d0 + chunk))), weighting)
    removed = []
    levels = np.zeros((M, E), dtype=np.int32)
    sccs = []
    for d in range(M):
        src, dst, z = arcs[d]
        mask, sizes = break_cycles(E, src, dst, z, exact_max)
        sccs.append(sizes)
        for u, v in zip(src[mask].tolist(), dst[mask].tolist()):
            removed.append((d, v, u))
        levels[d] = levels_from_kept(E, src, dst, ~mask)
    removed = np.array(sorted(removed), dtype=np.int64).reshape(-1, 3)
    return dict(arcs=arcs, removed=removed, levels=levels, scc_sizes=sccs, weighting=weighting)


def build_graph_dirs(disc, dirs, weighting="face", exact_max=10, chunk=4):
    """build_graph restricted to the directions in `dirs` (levels of other directions are 0,
    their arc lists empty)."""
    M, E = disc.M_dirs, disc.E
    arcs = [None] * M
    dirs = list(dirs)
    for c0 in range(0, len(dirs), chunk):
        ds = dirs[c0:c0 + chunk]
        for d, a in zip(ds, edge_weights(disc, ds, weighting)):
            arcs[d] = a
    removed = []
    levels = np.zeros((M, E), dtype=np.int32)
    sccs = [[] for _ in range(M)]
    for d in dirs:
        src, dst, z = arcs[d]
        mask, sizes = break_cycles(E, src, dst, z, exact_max)
        sccs[d] = sizes
        for u, v in zip(src[mask].tolist(), dst[mask].tolist()):
            removed.append((d, v, u))
        levels[d] = levels_from_kept(E, src, dst, ~mask)
    removed = np.array(sorted(removed), dtype=np.int64).reshape(-1, 3)
    return dict(arcs=arcs, removed=removed, levels=levels, scc_sizes=sccs, weighting=weighting)
