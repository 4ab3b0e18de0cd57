"""sn_quadrature_level_symmetric through the C ABI (no GPU needed: the call touches no device).

The sets must equal the seeded input generator's bit for bit, and meet the moment conditions of
an S_N set (Sec. 2, after eq. 2: positive weights summing to 4 pi; level-symmetric sets integrate
the first moments to 0, the second to 4 pi / 3 delta_ij and the fourth to 4 pi / 5)."""
import ctypes
import os

import numpy as np
import pytest

import sn_inputs as si


@pytest.fixture(scope="module")
def q():
    from paper_1810_11080_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1810_11080_gb300 as g
    return g


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("N", [2, 4, 6, 8, 12])
def test_library_sets_equal_the_input_generator_bitwise(q, N, dim):
    om, w = q.sn_quadrature_level_symmetric(N, dim)
    om_ref, w_ref = si.level_symmetric(N, dim)
    assert om.shape == om_ref.shape and w.shape == w_ref.shape
    assert np.array_equal(om, om_ref) and np.array_equal(w, w_ref)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("N", [2, 4, 6, 8, 12])
def test_library_sets_meet_the_moment_conditions(q, N, dim):
    om, w = q.sn_quadrature_level_symmetric(N, dim)
    M = N * (N + 2) // (2 if dim == 2 else 1)
    assert len(w) == M and np.all(w > 0)
    assert np.allclose(np.linalg.norm(om, axis=1), 1.0, atol=1e-6)     # 7-digit table mu_1
    four_pi = 4 * np.pi
    assert abs(w.sum() - four_pi) <= 1e-13 * four_pi
    if dim == 3:
        assert np.allclose(om.T @ w, 0.0, atol=1e-13)
        np.testing.assert_allclose(np.einsum("d,di,dj->ij", w, om, om), four_pi / 3 * np.eye(3), atol=2e-6)
        if N >= 4:
            np.testing.assert_allclose(np.einsum("d,d->", w, om[:, 0] ** 4), four_pi / 5, rtol=2e-6)
    else:
        # 2D sets keep the upper hemisphere with doubled weights: x/y moments as in 3D
        assert np.allclose(om[:, :2].T @ w, 0.0, atol=1e-13)
        np.testing.assert_allclose(np.einsum("d,di,dj->ij", w, om[:, :2], om[:, :2]), four_pi / 3 * np.eye(2),
                                   atol=2e-6)


def test_size_query_and_bad_arguments(q):
    lib = q.lib()
    n = ctypes.c_int(-1)
    assert lib.sn_quadrature_level_symmetric(8, 3, ctypes.byref(n), None, None) == 0 and n.value == 80
    assert lib.sn_quadrature_level_symmetric(8, 2, ctypes.byref(n), None, None) == 0 and n.value == 40
    assert lib.sn_quadrature_level_symmetric(12, 3, ctypes.byref(n), None, None) == 0 and n.value == 168
    assert lib.sn_quadrature_level_symmetric(10, 3, ctypes.byref(n), None, None) == q.SN_EINVAL
    assert lib.sn_quadrature_level_symmetric(8, 4, ctypes.byref(n), None, None) == q.SN_EINVAL
    assert lib.sn_quadrature_level_symmetric(8, 3, None, None, None) == q.SN_EINVAL
    w = np.zeros(80)
    assert lib.sn_quadrature_level_symmetric(8, 3, ctypes.byref(n), None, w.ctypes.data) == q.SN_EINVAL
