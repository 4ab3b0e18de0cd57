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
