"""Pins of the oracle's diffusion synthetic acceleration (DSA): the symmetric interior-penalty
diffusion operator on curved elements and the accelerated source iteration.

- the operator is symmetric and positive definite on curved 2D/3D meshes;
- it is consistent: with the boundary functional of a manufactured smooth solution, its discrete
  solution converges at order p + 1 in L2 on curved quads (a wrong sign or a dropped face term
  breaks the order);
- DSA leaves the fixed point unchanged (dense coupled solve of the transport system) and cuts the
  iteration count of a scattering-dominated problem by an order of magnitude."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import sn_inputs as si
from oracle.dg import Discretization
from oracle.dsa import DiffusionOperator, dsa_source_iterate, _base_face_points, _basis_and_grad
from oracle.geometry import face_normal, face_reference_coords, physical_points
from oracle.graph import build_graph
from oracle.sweep import Sweeper, global_solve


def _curved(p, n=4, amp=0.08):
    prob = si.make_config("2d_sine_q2_p1_s4", n=n, p=p)
    prob.mesh = si.structured_mesh((n, n), 2, si.disp_sine_2d(amp))
    return prob


@pytest.mark.parametrize("case", ["2d_p1", "2d_p2", "2d_p3", "2d_smooth_p3", "3d_p1", "3d_p2"])
def test_operator_is_symmetric_positive_definite(case):
    if case.startswith("2d_p"):
        prob = _curved(int(case[-1]))
    elif case == "2d_smooth_p3":
        prob = si.make_config("2d_smooth_q3_p3_s8", n=4)
    else:
        prob = si.make_config("3d_twist_q2_p2_s8", n=2, p=int(case[-1]), sn=2)
    prob.sigma_s = 0.999 * prob.sigma_t                 # nearly no absorption: the hardest case
    A = DiffusionOperator(Discretization(prob)).A.toarray()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0.0


def _u(X):
    x, y = X[..., 0], X[..., 1]
    return np.sin(2 * x + 1) * np.cos(1.5 * y) + 0.5 * x * y


def _grad_u(X):
    x, y = X[..., 0], X[..., 1]
    return np.stack([2 * np.cos(2 * x + 1) * np.cos(1.5 * y) + 0.5 * y,
                     -1.5 * np.sin(2 * x + 1) * np.sin(1.5 * y) + 0.5 * x], -1)


def _lap_u(X):
    x, y = X[..., 0], X[..., 1]
    return -6.25 * np.sin(2 * x + 1) * np.cos(1.5 * y)


@pytest.mark.parametrize("p", [1, 2])
def test_manufactured_diffusion_solution_converges_at_order_p_plus_1(p):
    errs = []
    for n in (4, 8, 16):
        prob = si.make_config("2d_sine_q2_p1_s4", n=n, p=p)
        prob.sigma_t = np.ones(prob.mesh.n_elem)
        prob.sigma_s = 0.5 * prob.sigma_t
        disc = Discretization(prob)
        op = DiffusionOperator(disc)
        D, sa = 1.0 / 3.0, 0.5
        # l(v) = int f v + sum_bdr int ((D/2) du/dn + kappa u) v - (D/2) u dv/dn
        f = -D * _lap_u(disc.xq) + sa * _u(disc.xq)
        rhs = np.einsum("q,eq,eq,qm->em", disc.wq, disc.detJ, f, disc.B)
        s0, s1, wf = _base_face_points(2, disc.nf, 1)
        for (e, fc), kap in op.kappa_bdr.items():
            ctrl = prob.mesh.ctrl[e:e + 1]
            co = [np.broadcast_to(np.asarray(x, dtype=float), s0.shape) for x in face_reference_coords(2, fc, s0)]
            v, gv = _basis_and_grad(disc, ctrl, co)
            nt = face_normal(ctrl, disc.r, fc, s0)[0]                       # scaled normal n |J|
            X = physical_points(ctrl, disc.r, co)[0]
            dudn = np.einsum("pk,pk->p", _grad_u(X), nt)
            dvdn = np.einsum("pmk,pk->pm", gv[0], nt)
            ds = wf * np.linalg.norm(nt, axis=-1)
            rhs[e] += np.einsum("p,p,pm->m", wf, 0.5 * D * dudn, v[0]) + kap * np.einsum("p,p,pm->m", ds, _u(X), v[0])
            rhs[e] -= 0.5 * D * np.einsum("p,p,pm->m", wf, _u(X), dvdn)
        uh = op.solve(rhs)
        err = np.einsum("qm,em->eq", disc.B, uh) - _u(disc.xq)
        errs.append(np.sqrt(np.einsum("q,eq,eq->", disc.wq, disc.detJ, err ** 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] >= p + 1 - 0.25, (errs, orders)


def test_dsa_keeps_the_fixed_point():
    prob = _curved(2, n=4)
    prob.sigma_t = np.linspace(0.5, 3.0, prob.mesh.n_elem)
    prob.sigma_s = 0.9 * prob.sigma_t
    disc = Discretization(prob)
    G = build_graph(disc, "face")
    assert len(G["removed"]) > 0
    R = dsa_source_iterate(Sweeper(disc, G), DiffusionOperator(disc), tol=1e-13)
    _, phi_ref = global_solve(disc)
    assert R["converged"]
    assert np.abs(R["phi"] - phi_ref).max() <= 1e-10 * np.abs(phi_ref).max()


def test_dsa_cuts_the_iterations_of_a_scattering_dominated_problem():
    prob = si.make_config("2d_sine_q2_p1_s4", n=8, p=1)
    prob.sigma_t = 10.0 * np.ones(prob.mesh.n_elem)
    prob.sigma_s = 0.99 * prob.sigma_t
    disc = Discretization(prob)
    S = Sweeper(disc, build_graph(disc, "face"))
    plain = S.source_iterate(tol=1e-8, max_iter=3000)
    acc = dsa_source_iterate(S, DiffusionOperator(disc), tol=1e-8, max_iter=3000)
    assert plain["converged"] and acc["converged"]
    assert acc["iters"] * 8 <= plain["iters"], (plain["iters"], acc["iters"])
    assert np.abs(acc["phi"] - plain["phi"]).max() <= 1e-6 * np.abs(plain["phi"]).max()
