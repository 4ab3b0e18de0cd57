"""Pins of the oracle's tetrahedra (straight-sided, P_1 geometry, P_p DG with p = 1, 2; Sec. 2
simplicial elements) against closed forms, surface identities, pure-absorber convergence at
order p + 1, the dense coupled solve and renumbering invariance."""
import math

import numpy as np
import pytest

from sn_inputs.configs import tet_problem
from sn_inputs.mms import attenuation
from oracle.graph import build_graph
from oracle.simplex3 import (FACES, TetDiscretization, basis_values, basis_grads, face_normal_tet,
                             face_rule_points, volume_rule, face_basis_values, orient_face, PERMS)
from oracle.sweep import Sweeper, global_solve


@pytest.mark.parametrize("p", [1, 2])
def test_tet_basis_is_nodal_and_reproduces_polynomials(p):
    nodes = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    if p == 2:
        edges = ((0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3))
        nodes += [tuple(0.5 * (np.array(nodes[a]) + np.array(nodes[b]))) for a, b in edges]
    X = np.array(nodes, dtype=float)
    V = np.stack(basis_values(p, X[:, 0], X[:, 1], X[:, 2]), axis=1)
    assert np.allclose(V, np.eye(len(nodes)), atol=1e-15)
    rng = np.random.default_rng(p)
    P = rng.dirichlet([1, 1, 1, 1], size=15)[:, 1:]
    f = lambda Y: 1.0 - Y[:, 0] + 2 * Y[:, 1] + 0.5 * Y[:, 2] + (Y[:, 0] * Y[:, 2] - Y[:, 1] ** 2 if p == 2 else 0.0)
    B = np.stack(basis_values(p, P[:, 0], P[:, 1], P[:, 2]), axis=1)
    assert np.allclose(B @ f(X), f(P), atol=1e-13)
    G = np.stack([np.stack(g, axis=-1) for g in basis_grads(p, P[:, 0], P[:, 1], P[:, 2])], axis=1)
    h = 1e-6
    for k in range(3):
        dP = P.copy()
        dP[:, k] += h
        Bp = np.stack(basis_values(p, dP[:, 0], dP[:, 1], dP[:, 2]), axis=1)
        assert np.allclose((Bp - B) / h, G[:, :, k], atol=1e-5)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_collapsed_rules_integrate_monomials(n):
    pts, w = volume_rule(n)
    for a in range(2 * n - 2):
        for b in range(2 * n - 2 - a):
            for c in range(2 * n - 2 - a - b):
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                assert abs(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c) - exact) < 1e-15
    s, t, wf = face_rule_points(n)
    for a in range(2 * n - 1):
        for b in range(2 * n - 1 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.sum(wf * s ** a * t ** b) - exact) < 1e-15


def test_affine_p1_mass_and_stiffness_closed_forms():
    prob = tet_problem(1, 1)
    A = np.array([[1.2, 0.1, -0.2], [0.3, 0.9, 0.1], [0.0, -0.2, 1.1]])
    prob.mesh.ctrl = np.einsum("ij,emj->emi", A, prob.mesh.ctrl)
    D = TetDiscretization(prob)
    for e in range(prob.mesh.n_elem):
        v = prob.mesh.ctrl[e]
        J = np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]], axis=1)
        vol = np.linalg.det(J) / 6.0
        assert np.allclose(D.M[e], vol / 20.0 * (np.ones((4, 4)) + np.eye(4)), rtol=1e-13)
        grads = np.linalg.solve(J.T, np.array([[-1.0, -1.0, -1.0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]).T).T
        for i in range(4):
            for k in range(3):
                assert np.allclose(D.S[e, k, i, :], grads[i, k] * vol / 4.0, rtol=1e-12, atol=1e-15)


def test_face_normals_close_the_surface_and_point_outwards():
    prob = tet_problem(2, 1, rotate_seed=3)
    ctrl = prob.mesh.ctrl
    tot = np.zeros((ctrl.shape[0], 3))
    for f in range(4):
        n = face_normal_tet(ctrl, f)
        a, b, c = FACES[f]
        cf = (ctrl[:, a] + ctrl[:, b] + ctrl[:, c]) / 3.0
        assert np.all(np.einsum("ed,ed->e", n, cf - ctrl.mean(axis=1)) > 0.0)
        tot += n
    assert np.allclose(tot, 0.0, atol=1e-15)


def test_orientation_maps_the_shared_face_points():
    """Our face point and the neighbour's point at the mapped coordinates are the same physical
    point, for every interior face of a renumbered mesh."""
    prob = tet_problem(2, 2, rotate_seed=7)
    m = prob.mesh
    s = np.array([0.1, 0.3, 0.6])
    t = np.array([0.2, 0.5, 0.1])
    for e in range(m.n_elem):
        for f in range(4):
            nb = m.face_nbr[e, f]
            if nb < 0:
                continue
            a, b, c = FACES[f]
            X = m.ctrl[e, a] + s[:, None] * (m.ctrl[e, b] - m.ctrl[e, a]) + t[:, None] * (m.ctrl[e, c] - m.ctrl[e, a])
            s2, t2 = orient_face(int(m.orient[e, f]), s, t)
            a2, b2, c2 = FACES[m.nbr_face[e, f]]
            Y = m.ctrl[nb, a2] + s2[:, None] * (m.ctrl[nb, b2] - m.ctrl[nb, a2]) + t2[:, None] * (m.ctrl[nb, c2] - m.ctrl[nb, a2])
            assert np.allclose(X, Y, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2])
def test_divergence_identity_on_tets(p):
    prob = tet_problem(2, p, rotate_seed=2)
    D = TetDiscretization(prob)
    lhs = D.S.sum(axis=-1)                                                # [E, 3, N]
    rhs = np.zeros_like(lhs)
    s, t, w = face_rule_points(p + 2)
    for f in range(4):
        n = face_normal_tet(prob.mesh.ctrl, f)
        vals = face_basis_values(p, s, t)
        for j, m in enumerate(D.fnode[f]):
            rhs[:, :, m] += np.sum(w * vals[j]) * n
    assert np.allclose(lhs, rhs, atol=1e-13)


@pytest.mark.parametrize("weighting", ["unity", "face", "siginvface"])
@pytest.mark.parametrize("p", [1, 2])
def test_source_iteration_equals_the_dense_solve_on_tets(p, weighting):
    prob = tet_problem(2, p, rotate_seed=1)
    D = TetDiscretization(prob)
    R = Sweeper(D, build_graph(D, weighting)).source_iterate(tol=1e-14, max_iter=300)
    _psi, phi = global_solve(D)
    assert np.allclose(R["phi"], phi, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2])
def test_lagged_source_iteration_equals_the_dense_solve_on_twisted_tets(p):
    """A twisted column of straight tetrahedra has sweep cycles; the lagged iteration still
    converges to the coupled solution."""
    prob = tet_problem(2, p, twist=2.5, rotate_seed=3)
    D = TetDiscretization(prob)
    G = build_graph(D, "face")
    assert len(G["removed"]) > 0
    R = Sweeper(D, G).source_iterate(tol=1e-14, max_iter=400)
    _psi, phi = global_solve(D)
    assert np.allclose(R["phi"], phi, rtol=1e-11, atol=1e-13)


def test_renumbered_tets_give_the_same_solution():
    out = []
    for seed in (None, 6):
        prob = tet_problem(2, 2, rotate_seed=seed)
        D = TetDiscretization(prob)
        R = Sweeper(D, build_graph(D, "face")).source_iterate(tol=1e-13)
        out.append(np.einsum("emn,en->e", D.M, R["phi"]))
    assert np.allclose(out[0], out[1], rtol=1e-12, atol=0)


@pytest.mark.parametrize("p", [1, 2])
def test_pure_absorber_on_tets_converges_at_order_p_plus_1(p):
    errs = []
    for n in (2, 4, 8):
        prob, exact = attenuation(tet_problem(n, p), sigma_t=2.0)
        D = TetDiscretization(prob)
        R = Sweeper(D, build_graph(D, "face")).source_iterate(tol=1e-13)
        e2 = 0.0
        for d in range(D.M_dirs):
            v = np.einsum("qm,em->eq", D.B, R["psi"][d]) - exact(D.xq, d)
            e2 += D.w[d] * float(np.einsum("q,eq,eq->", D.wq, D.detJ, v * v))
        errs.append(math.sqrt(e2))
    assert math.log2(errs[-2] / errs[-1]) >= p + 1 - 0.25, errs


def test_half_the_faces_are_inflow_on_average():
    """The four scaled face normals of a tetrahedron sum to zero and the level-symmetric set holds
    -Omega with every Omega, so over the directions exactly half the faces (2 of 4) are inflow
    faces: the F = 2 of the stored-inverse byte count."""
    prob = tet_problem(3, 1, sn=8, twist=1.0)
    n = np.stack([face_normal_tet(prob.mesh.ctrl, f) for f in range(4)], axis=1)     # [E, 4, 3]
    g = np.einsum("dk,efk->def", prob.omega, n)
    assert np.all(g != 0.0)
    inflow = (g < 0.0).sum(axis=2)                                                  # [M, E]
    assert inflow.min() >= 1 and inflow.max() <= 3
    assert inflow.mean() == 2.0


# ---------------------------------------------------------------- P_2 geometry (curved tetrahedra)
from oracle.simplex3 import face_nodes, face_normal_tet_p2


def _volume(D):
    return float(np.einsum("q,eq->", D.wq, D.detJ))


def test_p2_geometry_volume_of_a_twisted_column_converges_at_fourth_order():
    """The twisted column's volume is 1 (every z-slice is a rotated unit square).  Straight
    tetrahedra approximate it at order 2 in h, P_2 tetrahedra at order 4 (the interpolation
    error of the twist's map integrates to the next even order)."""
    for r, order in ((1, 2.0), (2, 4.0)):
        errs = [abs(_volume(TetDiscretization(tet_problem(n, 1, r=r, twist=1.5))) - 1.0) for n in (2, 4, 8)]
        rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert all(abs(x - order) < 0.1 for x in rates), (r, errs, rates)


def test_p2_tets_of_an_affine_mesh_equal_the_straight_ones():
    """An affine mesh written with P_2 geometry (edge nodes at the straight midpoints): the same
    M, S, volume points and face blocks as the straight tetrahedra, to rounding."""
    for p in (1, 2):
        D1 = TetDiscretization(tet_problem(2, p, rotate_seed=4))
        D2 = TetDiscretization(tet_problem(2, p, rotate_seed=4, r=2))
        assert np.allclose(D1.M, D2.M, rtol=0, atol=1e-16) and np.allclose(D1.S, D2.S, rtol=0, atol=1e-15)
        assert np.allclose(D1.xnodes, D2.xnodes, rtol=0, atol=1e-15)
        dirs = list(range(0, D1.M_dirs, 5))
        f1, f2 = D1.face_blocks(dirs), D2.face_blocks(dirs)
        for k in ("out_o", "out_n", "bar_o", "bar_n", "bout", "bin"):
            assert np.allclose(f1[k], f2[k], rtol=0, atol=1e-15), k


def _face_map(ctrl, f, s, t):
    vals = face_basis_values(2, s, t)
    return sum(ctrl[:, m, None, :] * vals[j][None, :, None] for j, m in enumerate(face_nodes(2, f)))


def test_p2_face_normals_close_the_surface_and_orientation_maps_shared_points():
    prob = tet_problem(2, 1, r=2, twist=2.0, rotate_seed=5)
    m = prob.mesh
    s, t, w = face_rule_points(3)                      # exact for the quadratic normal
    tot = np.zeros((m.n_elem, 3))
    for f in range(4):
        tot += np.einsum("q,eqk->ek", w, face_normal_tet_p2(m.ctrl, f, s, t))
    assert np.allclose(tot, 0.0, atol=1e-15)
    # the collapsed-square normal at u = 0 and the P_2 normal agree with a finite difference of the
    # face map
    h = 1e-6
    x0 = _face_map(m.ctrl, 1, np.array([0.3]), np.array([0.2]))
    xs = (_face_map(m.ctrl, 1, np.array([0.3 + h]), np.array([0.2])) - x0) / h
    xt = (_face_map(m.ctrl, 1, np.array([0.3]), np.array([0.2 + h])) - x0) / h
    assert np.allclose(np.cross(xs, xt)[:, 0], face_normal_tet_p2(m.ctrl, 1, np.array([0.3]), np.array([0.2]))[:, 0],
                       atol=1e-5)
    ss = np.array([0.1, 0.3, 0.6])
    tt = np.array([0.2, 0.5, 0.1])
    for e in range(m.n_elem):
        for f in range(4):
            nb = m.face_nbr[e, f]
            if nb < 0:
                continue
            X = _face_map(m.ctrl[e:e + 1], f, ss, tt)[0]
            s2, t2 = orient_face(int(m.orient[e, f]), ss, tt)
            Y = _face_map(m.ctrl[nb:nb + 1], int(m.nbr_face[e, f]), s2, t2)[0]
            assert np.allclose(X, Y, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2])
def test_divergence_identity_on_p2_tets(p):
    """sum_n S^k_mn = oint u_m n_k over the four curved faces (exact rules on both sides): pins
    S, the P_2 Jacobian, the curved normals and the face-node maps together."""
    prob = tet_problem(2, p, r=2, twist=2.0, rotate_seed=2)
    D = TetDiscretization(prob)
    lhs = D.S.sum(axis=-1)
    rhs = np.zeros_like(lhs)
    s, t, w = face_rule_points(p + 3)
    for f in range(4):
        n = face_normal_tet_p2(prob.mesh.ctrl, f, s, t)                 # [E, P, 3]
        vals = face_basis_values(p, s, t)
        for j, mm in enumerate(D.fnode[f]):
            rhs[:, :, mm] += np.einsum("q,eqk->ek", w * vals[j], n)
    assert np.allclose(lhs, rhs, atol=1e-13)


@pytest.mark.parametrize("kw", [dict(bubble=0.05), dict(twist=2.5)])
@pytest.mark.parametrize("weighting", ["unity", "face", "siginvface"])
def test_lagged_source_iteration_equals_the_dense_solve_on_p2_tets(kw, weighting):
    """Curved faces carry partially-inflow couplings (two-way arcs), so even the interior-curved
    cube has cycles to lag; the lagged iteration converges to the coupled solution."""
    prob = tet_problem(2, 1, r=2, **kw)
    D = TetDiscretization(prob)
    G = build_graph(D, weighting)
    assert len(G["removed"]) > 0
    R = Sweeper(D, G).source_iterate(tol=1e-14, max_iter=400)
    _psi, phi = global_solve(D)
    assert np.allclose(R["phi"], phi, rtol=1e-11, atol=1e-13)


def test_face_rule_of_curved_faces_converges_with_k():
    """The kink-aligned rule's blocks on curved faces converge as the composite pieces are
    refined (K = 1, 2, 4 against K = 16), and a K = 1 rule is already within 1e-3."""
    prob = tet_problem(2, 2, r=2, twist=2.5)
    dirs = list(range(0, len(prob.w), 3))
    ref = TetDiscretization(prob, face_subdiv=16).face_blocks(dirs)["bar_o"]
    errs = [float(np.max(np.abs(TetDiscretization(prob, face_subdiv=K).face_blocks(dirs)["bar_o"] - ref)))
            for K in (1, 2, 4)]
    scale = float(np.max(np.abs(ref)))
    assert errs[0] < 1e-3 * scale and errs[1] < errs[0] / 4 and errs[2] < errs[1] / 4, (errs, scale)


@pytest.mark.parametrize("p", [1, 2])
def test_pure_absorber_on_p2_tets_converges_at_order_p_plus_1(p):
    """The interior-curved cube (P_2 geometry; its boundary stays the cube's), S2."""
    errs = []
    for n in (2, 4, 8):
        prob, exact = attenuation(tet_problem(n, p, sn=2, r=2, bubble=0.05), sigma_t=2.0)
        D = TetDiscretization(prob)
        R = Sweeper(D, build_graph(D, "face")).source_iterate(tol=1e-13)
        e2 = 0.0
        for d in range(D.M_dirs):
            v = np.einsum("qm,em->eq", D.B, R["psi"][d]) - exact(D.xq, d)
            e2 += D.w[d] * float(np.einsum("q,eq,eq->", D.wq, D.detJ, v * v))
        errs.append(math.sqrt(e2))
    assert math.log2(errs[-2] / errs[-1]) >= p + 1 - 0.25, errs


def test_renumbered_p2_tets_agree_to_the_face_rule_accuracy():
    """Renumbering a curved tetrahedron moves the apex of its faces' collapsed squares, so the
    kinked face integrals are approximated on other pieces: the solutions differ by the face
    rule's error, and that difference shrinks as the composite pieces are refined."""
    diffs = []
    for K in (2, 8):
        out = []
        for seed in (None, 6):
            prob = tet_problem(2, 2, r=2, twist=2.0, rotate_seed=seed)
            D = TetDiscretization(prob, face_subdiv=K)
            R = Sweeper(D, build_graph(D, "face")).source_iterate(tol=1e-13)
            out.append(np.einsum("emn,en->e", D.M, R["phi"]))
        diffs.append(float(np.max(np.abs(out[0] - out[1]) / np.abs(out[0]))))
    assert diffs[0] < 1e-5 and diffs[1] < diffs[0] / 3, diffs
