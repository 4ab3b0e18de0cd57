"""Pins of the oracle's triangle discretisation (P_r geometry, P_p DG; Sec. 2) against closed
forms, identities that a wrong face map or sign breaks, manufactured-solution convergence at
order p + 1 on curved triangles, and the dense coupled solve."""
import math

import numpy as np
import pytest

from sn_inputs.configs import triangle_problem
from sn_inputs.mesh import triangle_mesh
from sn_inputs.mms import annulus_mms, attenuation
from oracle.basis import gll_nodes, equispaced_nodes
from oracle.graph import build_graph
from oracle.simplex import (LagrangeTri, SimplexDiscretization, edge_nodes, face_normal_tri, node_coords,
                            volume_rule)
from oracle.sweep import Sweeper, global_solve


@pytest.mark.parametrize("k", [1, 2, 3])
def test_lagrange_basis_is_nodal_and_reproduces_polynomials(k):
    nodes = node_coords(k, gll_nodes(k))
    L = LagrangeTri(k, nodes)
    assert np.allclose(L.values(nodes), np.eye(len(nodes)), atol=1e-12)
    rng = np.random.default_rng(k)
    pts = rng.dirichlet([1, 1, 1], size=20)[:, :2]
    f = lambda P: 1.0 + 2.0 * P[:, 0] - P[:, 1] + (0.5 * P[:, 0] * P[:, 1] if k >= 2 else 0.0) + \
        (P[:, 1] ** 3 if k >= 3 else 0.0)
    assert np.allclose(L.values(pts) @ f(nodes), f(pts), atol=1e-12)
    g = L.grads(pts)
    assert np.allclose(g.sum(axis=1), 0.0, atol=1e-11)                   # partition of unity


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_collapsed_rule_integrates_monomials(n):
    pts, w = volume_rule(n)
    for a in range(2 * n - 1):
        for b in range(2 * n - 1 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b) - exact) < 1e-14


def _affine_problem(p):
    prob = triangle_problem(2, 1, p, amp=0.0)
    A = np.array([[1.4, 0.3], [-0.2, 0.9]])
    prob.mesh.ctrl = np.einsum("ij,emj->emi", A, prob.mesh.ctrl)
    return prob, A


def test_affine_p1_mass_and_stiffness_closed_forms():
    prob, A = _affine_problem(1)
    D = SimplexDiscretization(prob)
    for e in range(prob.mesh.n_elem):
        v = prob.mesh.ctrl[e, :3]
        area = 0.5 * ((v[1, 0] - v[0, 0]) * (v[2, 1] - v[0, 1]) - (v[2, 0] - v[0, 0]) * (v[1, 1] - v[0, 1]))
        assert np.allclose(D.M[e], area / 12.0 * (np.ones((3, 3)) + np.eye(3)), rtol=1e-13)
        # barycentric gradients: grad lambda_i = (-d_y, d_x) / (2 area), d = v_{i+2} - v_{i+1}
        # (the inward normal of the opposite edge over the height)
        for i in range(3):
            d = v[(i + 2) % 3] - v[(i + 1) % 3]
            grad = np.array([-d[1], d[0]]) / (2.0 * area)
            for k in range(2):
                assert np.allclose(D.S[e, k, i, :], grad[k] * area / 3.0, rtol=1e-12, atol=1e-15)


def test_straight_face_normals_are_outward_with_edge_length():
    prob, _ = _affine_problem(1)
    ctrl = prob.mesh.ctrl
    for f in range(3):
        n = face_normal_tri(ctrl, 1, f, np.array([0.3]))[:, 0, :]      # [E, 2]
        a, b = [edge_nodes(1, f)[0], edge_nodes(1, f)[-1]]
        t = ctrl[:, b] - ctrl[:, a]
        assert np.allclose(np.linalg.norm(n, axis=1), np.linalg.norm(t, axis=1), rtol=1e-14)
        c = ctrl[:, :3].mean(axis=1)
        mid = 0.5 * (ctrl[:, a] + ctrl[:, b])
        assert np.all(np.einsum("ed,ed->e", n, mid - c) > 0.0)            # points away from the centroid


@pytest.mark.parametrize("p,r", [(1, 2), (2, 3), (3, 3)])
def test_divergence_identity_on_curved_triangles(p, r):
    """sum_n S^k[m][n] = int du_m/dx_k = oint u_m n_k ds: pins S, the face normals and the face
    node maps together (a wrong edge node order or normal sign breaks it)."""
    prob = triangle_problem(3, r, p, amp=0.06)
    D = SimplexDiscretization(prob)
    from oracle.basis import gauss_legendre
    t, wt = gauss_legendre(p + r + 1)
    lhs = D.S.sum(axis=-1)                                                # [E, 2, N]
    rhs = np.zeros_like(lhs)
    from oracle.basis import lagrange
    for f in range(3):
        n = face_normal_tri(prob.mesh.ctrl, r, f, t)                      # [E, P, 2]
        ids = edge_nodes(p, f)
        for j, m in enumerate(ids):
            uj = np.array([lagrange(D.gll, j, x) for x in t])
            rhs[:, :, m] += np.einsum("q,q,eqk->ek", wt, uj, n)
    assert np.allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_mms_on_curved_triangles_converges_at_order_p_plus_1(p):
    errs = []
    for n in (4, 8, 16):
        prob, fex, fac = annulus_mms(triangle_problem(n, 3, p))
        D = SimplexDiscretization(prob)
        R = Sweeper(D, build_graph(D, "face")).source_iterate(tol=1e-12)
        v = np.einsum("qm,em->eq", D.B, R["phi"]) - fac * fex(D.xq)
        errs.append(float(np.sqrt(np.einsum("q,eq,eq->", D.wq, D.detJ, v * v))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] >= p + 1 - 0.2, (errs, orders)


@pytest.mark.parametrize("weighting", ["unity", "face", "siginvface"])
def test_lagged_source_iteration_equals_the_dense_solve_on_triangles(weighting):
    prob = triangle_problem(3, 2, 2, amp=0.08)
    D = SimplexDiscretization(prob)
    G = build_graph(D, weighting)
    assert len(G["removed"]) > 0                      # the curved mesh has cycles to lag
    R = Sweeper(D, G).source_iterate(tol=1e-14, max_iter=400)
    _psi, phi = global_solve(D)
    assert np.allclose(R["phi"], phi, rtol=1e-10, atol=1e-12)


def test_rotated_local_numbering_gives_the_same_solution():
    out = []
    for seed in (None, 5):
        prob = triangle_problem(4, 2, 2, amp=0.06, rotate_seed=seed)
        D = SimplexDiscretization(prob)
        R = Sweeper(D, build_graph(D, "face")).source_iterate(tol=1e-13)
        out.append(np.einsum("emn,en->e", D.M, R["phi"]))                # int_e phi, numbering-free
    assert np.allclose(out[0], out[1], rtol=1e-10, atol=0)


def test_pure_absorber_on_triangles_converges():
    errs = []
    for n in (4, 8, 16):
        prob, exact = attenuation(triangle_problem(n, 2, 2), sigma_t=2.0)
        D = SimplexDiscretization(prob)
        R = Sweeper(D, build_graph(D, "face")).source_iterate(tol=1e-13)
        e2 = 0.0
        for d in range(D.M_dirs):
            v = np.einsum("qm,em->eq", D.B, R["psi"][d]) - exact(D.xq, d)
            e2 += D.w[d] * float(np.einsum("q,eq,eq->", D.wq, D.detJ, v * v))
        errs.append(math.sqrt(e2))
    assert math.log2(errs[-2] / errs[-1]) >= 3 - 0.2, errs
