"""CPU FP64 oracle of the graph-based S_N sweep (Haut et al., arXiv 1810.11080).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this package.  It shares no code with
the CUDA library (paper_1810_11080_gb300) and imports nothing from it.

Layout (each function cites the passage of the paper it restates):
  basis.py    1D Gauss-Legendre / GLL / Lagrange tables, plain partial-pivot LU.
  geometry.py curved-element map, Jacobian, face normals (Sec. 2, eqs. 1 and 14).
  dg.py       local DG blocks G, F_e, F_{e,e'}, M_t, M_s, q (Sec. 2, eqs. 6-13, 15-16).
  graph.py    upwind dependency graph, edge weights, Tarjan SCC, exact FAS on small
              SCCs, Eades-Lin-Smyth on large ones, wavefront levels (Sec. 3).
  sweep.py    lagged sweep, source iteration, dense global solve (Sec. 3, eqs. 17-21).
  mlp.py      reference per-element MLP (forward, backward, finite differences).

Floating point: everything is IEEE binary64.  The quantities that decide the graph
(face normals at face quadrature points, upwind coupling blocks, edge weights,
the sigma_t mass matrix and its LU) are evaluated in the fixed operation order
written in each function, with no fused multiply-add, so that an independent
implementation following the same order reproduces them bit for bit.
"""
