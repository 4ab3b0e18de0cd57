"""Pins of the oracle's graph stage: SCCs against networkx, the exact FAS against brute force
over all orders, ELS invariants, level validity, and the paper's qualitative claims."""
import itertools
import numpy as np
import pytest

import sn_inputs as si
from oracle.dg import Discretization
from oracle.graph import tarjan_scc, fas_exact, fas_els, levels_from_kept, build_graph, break_cycles

nx = pytest.importorskip("networkx")


def random_digraph(n, p, rng, unity=False):
    z = {}
    for u in range(n):
        for v in range(n):
            if u != v and rng.uniform() < p:
                z[(u, v)] = 1.0 if unity else float(rng.uniform(0.1, 2.0))
    return z


def cost_of_order(order, z):
    pos = {v: i for i, v in enumerate(order)}
    return sum(w for (u, v), w in z.items() if pos[u] > pos[v])


@pytest.mark.parametrize("seed", range(12))
def test_tarjan_matches_networkx(seed):
    rng = np.random.default_rng(seed)
    n = 30
    z = random_digraph(n, 0.08, rng)
    succ = [sorted(v for (u, v) in z if u == a) for a in range(n)]
    mine = sorted(tuple(c) for c in tarjan_scc(n, succ))
    g = nx.DiGraph(); g.add_nodes_from(range(n)); g.add_edges_from(z)
    ref = sorted(tuple(sorted(c)) for c in nx.strongly_connected_components(g))
    assert mine == ref


@pytest.mark.parametrize("seed,unity", [(s, u) for s in range(10) for u in (False, True)])
def test_exact_fas_equals_brute_force(seed, unity):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 8))
    z = random_digraph(n, 0.5, rng, unity)
    verts = list(range(n))
    order, removed = fas_exact(verts, z)
    best = min(cost_of_order(o, z) for o in itertools.permutations(verts))
    assert abs(cost_of_order(order, z) - best) < 1e-12
    assert abs(sum(z[a] for a in removed) - best) < 1e-12
    # removing the arcs leaves an acyclic graph
    g = nx.DiGraph(); g.add_nodes_from(verts); g.add_edges_from(a for a in z if a not in set(removed))
    assert nx.is_directed_acyclic_graph(g)


@pytest.mark.parametrize("seed", range(10))
def test_els_gives_acyclic_graph_and_upper_bound(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(4, 8))
    z = random_digraph(n, 0.45, rng)
    verts = list(range(n))
    order, removed = fas_els(verts, z)
    assert sorted(order) == verts
    g = nx.DiGraph(); g.add_nodes_from(verts); g.add_edges_from(a for a in z if a not in set(removed))
    assert nx.is_directed_acyclic_graph(g)
    best = min(cost_of_order(o, z) for o in itertools.permutations(verts))
    assert cost_of_order(order, z) >= best - 1e-12
    # Eades-Lin-Smyth guarantee: at most m/2 - n/6 arcs removed on an unweighted, connected
    # graph without 2-cycles
    uz = {a: 1.0 for a in z if (a[1], a[0]) not in z or a[0] < a[1]}
    gu = nx.DiGraph(); gu.add_nodes_from(verts); gu.add_edges_from(uz)
    if nx.is_weakly_connected(gu):
        _o, urem = fas_els(verts, uz)
        assert len(urem) <= len(uz) / 2 - n / 6 + 1e-9


def test_els_on_known_cases():
    # a directed cycle: one arc must go; delta ties -> smallest id starts, arc (2 -> 0) removed
    z = {(0, 1): 1.0, (1, 2): 1.0, (2, 0): 1.0}
    order, removed = fas_els([0, 1, 2], z)
    assert order == [0, 1, 2] and removed == [(2, 0)]
    # the heavier arc of a 2-cycle is kept (the lighter one is lagged)
    z = {(0, 1): 3.0, (1, 0): 1.0}
    assert fas_els([0, 1], z)[1] == [(1, 0)]
    assert fas_exact([0, 1], z)[1] == [(1, 0)]
    # a DAG loses nothing
    z = {(0, 1): 1.0, (1, 2): 2.0, (0, 2): 1.0}
    assert fas_els([0, 1, 2], z)[1] == []


def test_levels_are_a_valid_layering():
    rng = np.random.default_rng(5)
    n = 40
    z = random_digraph(n, 0.05, rng)
    src = np.array([u for (u, v) in z]); dst = np.array([v for (u, v) in z]); w = np.array(list(z.values()))
    mask, _ = break_cycles(n, src, dst, w, exact_max=10)
    lv = levels_from_kept(n, src, dst, ~mask)
    kept = [(u, v) for u, v, m in zip(src, dst, mask) if not m]
    for u, v in kept:
        assert lv[v] > lv[u]
    has_in = set(v for _, v in kept)
    for v in range(n):
        assert (lv[v] == 0) == (v not in has_in)
        if v in has_in:
            assert lv[v] == 1 + max(lv[u] for u, vv in kept if vv == v)


def test_cartesian_mesh_has_no_cycles_and_diagonal_levels():
    prob = si.make_config("2d_sine_q2_p1_s4", n=5, p=1)
    prob.mesh = si.structured_mesh((5, 5), 2, None)
    D = Discretization(prob)
    G = build_graph(D, "face")
    assert len(G["removed"]) == 0
    for d in range(D.M_dirs):
        sx, sy = np.sign(D.omega[d, 0]), np.sign(D.omega[d, 1])
        for e in range(D.E):
            i, j = e % 5, e // 5
            ii = i if sx > 0 else 4 - i
            jj = j if sy > 0 else 4 - j
            assert G["levels"][d, e] == ii + jj


def test_scc_membership_is_weighting_independent():
    """Sec. 4.2: the elements in each SCC do not depend on the weighting; removed edges may."""
    prob = si.make_config("2d_sine_q2_p1_s4", n=8, p=1)
    prob.mesh = si.structured_mesh((8, 8), 2, si.disp_sine_2d(0.08))
    D = Discretization(prob)
    res = {w: build_graph(D, w) for w in ("unity", "face", "siginvface")}
    for w in res:
        assert res[w]["scc_sizes"] == res["unity"]["scc_sizes"]
    assert sum(len(s) for s in res["unity"]["scc_sizes"]) > 0
    arcs_u = [(a[0].tolist(), a[1].tolist()) for a in res["unity"]["arcs"]]
    arcs_f = [(a[0].tolist(), a[1].tolist()) for a in res["face"]["arcs"]]
    assert arcs_u == arcs_f                                      # same graph, different weights
