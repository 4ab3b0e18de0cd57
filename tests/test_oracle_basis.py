"""Pins of the oracle's 1D tables, quadrature sets and LU against closed forms and
library routines (not against the oracle itself)."""
import math
import numpy as np
import pytest

from oracle.basis import (gauss_legendre, gll_nodes, equispaced_nodes, lagrange, lagrange_deriv,
                          lu_factor, lu_solve, lu_solve_dense)
from oracle.graph import lu_factor_batch, lu_solve_batch
import sn_inputs as si


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_legendre_matches_numpy_and_is_exact(n):
    t, w = gauss_legendre(n)
    x, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(t, np.sort(0.5 * (1 - x))[::1][np.argsort(np.argsort(t))], atol=2e-16)
    assert np.allclose(np.sort(w), np.sort(wr / 2), atol=5e-16)
    for k in range(2 * n):          # exact for degree <= 2n-1 on [0,1]
        assert abs(np.dot(w, t ** k) - 1.0 / (k + 1)) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3])
def test_gll_nodes_are_lobatto_points(p):
    g = gll_nodes(p)
    # interior GLL nodes are the roots of P_p'(x) on [-1,1]
    dP = np.polynomial.legendre.Legendre.basis(p).deriv()
    roots = np.sort(0.5 * (1 + dP.roots())) if p > 1 else np.array([])
    assert np.allclose(g[1:-1], roots, atol=1e-15)
    assert g[0] == 0.0 and g[-1] == 1.0
    assert np.allclose(g + g[::-1], 1.0, atol=1e-16)


@pytest.mark.parametrize("nodes", [gll_nodes(1), gll_nodes(2), gll_nodes(3), equispaced_nodes(2), equispaced_nodes(3)])
def test_lagrange_partition_of_unity_and_cardinal(nodes):
    x = np.linspace(-0.2, 1.2, 37)
    s = sum(lagrange(nodes, j, x) for j in range(len(nodes)))
    ds = sum(lagrange_deriv(nodes, j, x) for j in range(len(nodes)))
    assert np.allclose(s, 1.0, atol=1e-13)
    assert np.allclose(ds, 0.0, atol=1e-11)
    for j in range(len(nodes)):
        for k in range(len(nodes)):
            assert lagrange(nodes, j, nodes[k]) == (1.0 if j == k else 0.0)
    # derivative against numpy's polynomial fit of the cardinal function
    for j in range(len(nodes)):
        y = np.zeros(len(nodes)); y[j] = 1
        c = np.polyfit(nodes, y, len(nodes) - 1)
        assert np.allclose(lagrange_deriv(nodes, j, x), np.polyval(np.polyder(c), x), atol=1e-9)


def test_lu_matches_numpy_and_batch_is_bitwise_plain():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(6, 9, 9))
    b = rng.normal(size=(6, 9))
    LUb, pb = lu_factor_batch(A)
    xb = lu_solve_batch(LUb, pb, b)
    for i in range(6):
        LU, perm = lu_factor(A[i])
        assert np.array_equal(np.array(LU), LUb[i]) and list(pb[i]) == perm
        x = lu_solve(LU, perm, b[i])
        assert np.array_equal(x, xb[i])
        assert np.allclose(x, np.linalg.solve(A[i], b[i]), rtol=1e-12, atol=1e-12)
    # partial pivoting: a zero leading entry must be pivoted away
    A = np.array([[0.0, 1.0], [2.0, 3.0]])
    assert np.allclose(lu_solve_dense(A, np.array([1.0, 5.0])), [1.0, 1.0])


@pytest.mark.parametrize("N,dim,count", [(2, 2, 4), (4, 2, 12), (8, 2, 40), (4, 3, 24), (8, 3, 80), (12, 3, 168), (6, 3, 48)])
def test_level_symmetric_moments(N, dim, count):
    om, w = si.level_symmetric(N, dim)
    assert om.shape == (count, 3) and np.all(w > 0)
    assert abs(w.sum() - 4 * np.pi) < 1e-13                         # sum omega = 4 pi
    assert np.allclose(np.linalg.norm(om, axis=1), 1.0, atol=1e-7)   # unit directions (7-digit table)
    c = om[:, :dim]                  # 2D sets stand for both hemispheres: in-plane moments only
    assert np.allclose(c.T @ w, 0.0, atol=1e-13)                     # first moments vanish
    sec = np.einsum("d,di,dj->ij", w, c, c)                          # second moments 4pi/3 delta
    assert np.allclose(sec, 4 * np.pi / 3 * np.eye(dim), atol=2e-6)
    if N > 2:                        # S2 integrates only up to second moments
        assert abs(np.sum(w * om[:, 0] ** 4) - 4 * np.pi / 5) < 2e-6  # fourth moment 4pi/5


def test_s2_directions_are_the_papers_a():
    """Sec. 4.2/4.3 quote the S2 ordinates as <+-a, +-a> with a = sqrt(3)/3."""
    with open(__file__.replace("test_oracle_basis.py", "golden/s2_level_symmetric.txt")) as fh:
        a = float([l for l in fh if not l.startswith("#")][0])
    om, w = si.level_symmetric(2, 3)
    assert np.allclose(np.abs(om), a, atol=1e-15)
    assert abs(a - math.sqrt(3) / 3) < 1e-15
