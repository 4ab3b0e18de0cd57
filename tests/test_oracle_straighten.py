"""The straightened low-order comparison (Sec. 4.1: a curved mesh divided N_ref times per
direction, its sub-cell vertices taken as the nodes of a linear mesh, solved with low-order
elements) on a quarter annulus with curved boundaries.

Pins of the straightening itself (areas against closed forms, topology), then the paper's
comparison with the oracle: the manufactured solution of its annulus problem is reproduced far
more accurately by the high-order discretisation on the curved mesh than by the low-order one on
the straightened mesh, with fewer unknowns; each converges at its own order."""
import math

import numpy as np
import pytest

import sn_inputs as si
from sn_inputs.configs import annulus_problem, straightened_problem
from sn_inputs.mesh import annulus_mesh, straighten, structured_mesh
from sn_inputs.mms import annulus_mms
from oracle.dg import Discretization
from oracle.graph import build_graph
from oracle.sweep import Sweeper


def _area(mesh):
    """Sum over elements of the shoelace area of the straight-sided cell through the Q_1
    control points (valid for straightened meshes only: Q_1 quads with straight edges)."""
    c = mesh.ctrl                          # [E][4][2], local order (0,0), (1,0), (0,1), (1,1)
    x = c[:, [0, 1, 3, 2], 0]
    y = c[:, [0, 1, 3, 2], 1]
    return float(np.sum(0.5 * (x * np.roll(y, -1, axis=1) - np.roll(x, -1, axis=1) * y).sum(axis=1)))


def test_straightening_an_affine_mesh_keeps_its_area():
    A = np.array([[1.3, 0.2], [-0.1, 0.8]])
    m = structured_mesh((3, 2), 2, lambda X: X @ (A - np.eye(2)).T)
    s = straighten(m, 4)
    assert s.r == 1 and s.n_elem == 6 * 16
    assert np.isclose(_area(s), abs(np.linalg.det(A)), rtol=1e-13)


def test_straightened_annulus_area_converges_at_second_order():
    exact = 0.25 * math.pi * (1.0 - 0.25)        # quarter annulus, radii 0.5 and 1
    errs = []
    for n_ref in (1, 2, 4):
        s = straighten(annulus_mesh(2, 3, 3), n_ref)
        a = _area(s)
        assert a < exact                          # chords lie inside the outer arc ...
        errs.append(exact - a)
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 4.0) < 0.3), (errs, ratios)


def test_straightened_topology():
    m = annulus_mesh(2, 3, 3)
    s = straighten(m, 3)
    nb = s.face_nbr
    # (2*3) x (3*3) grid of cells: 2 * 6 * 9 - 6 - 9 interior faces, each seen from both sides
    assert int((nb >= 0).sum()) == 2 * (2 * 6 * 9 - 6 - 9)
    assert int((nb < 0).sum()) == 2 * (6 + 9)
    for e in range(s.n_elem):
        for f in range(4):
            if nb[e, f] >= 0:
                assert nb[nb[e, f], s.nbr_face[e, f]] == e


def _mms_error(prob):
    prob, fex, fac = annulus_mms(prob)
    D = Discretization(prob)
    G = build_graph(D, "face")
    R = Sweeper(D, G).source_iterate(tol=1e-12)
    phi_q = np.einsum("qm,em->eq", D.B, R["phi"])
    v = phi_q - fac * fex(D.xq)
    return float(np.sqrt(np.einsum("q,eq,eq->", D.wq, D.detJ, v * v))), prob.mesh.n_elem * D.N, len(G["removed"])


def test_high_order_on_curved_mesh_beats_straightened_low_order():
    ho = [_mms_error(annulus_problem(n, 2 * n, 3, 3)) for n in (3, 6)]
    lo = [_mms_error(straightened_problem(annulus_problem(n, 2 * n, 3, 3), 3, 1)) for n in (3, 6)]
    for (eh, nh, _), (el, nl, _) in zip(ho, lo):
        assert nh < nl and eh < el / 20.0, (ho, lo)
    # orders: p + 1 = 4 for cubic elements on the cubic mesh, 2 for linear elements
    assert abs(math.log2(ho[0][0] / ho[1][0]) - 4.0) < 0.5, ho
    assert abs(math.log2(lo[0][0] / lo[1][0]) - 2.0) < 0.3, lo
    # the curved mesh has graph cycles (lagged arcs), the straightened one of the same problem none
    assert ho[0][2] > 0 and lo[0][2] == 0
