"""GPU side of the straightened low-order comparison (Sec. 4.1): volume quadrature points and
L2 errors through the C ABI against the oracle, and the manufactured-solution errors of the
curved high-order and straightened low-order annulus problems solved on the GPU against the
oracle's."""
import numpy as np
import pytest

from sn_inputs.configs import annulus_problem, straightened_problem
from sn_inputs.mms import annulus_mms
from gpu_util import gpu_ctx
from oracle.dg import Discretization
from oracle.graph import build_graph
from oracle.sweep import Sweeper

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _oracle_l2(D, v):
    return float(np.sqrt(np.einsum("q,eq,eq->", D.wq, D.detJ, v * v)))


@pytest.mark.parametrize("straight", [False, True])
def test_volume_points_and_l2_error_match_the_oracle(straight):
    prob = annulus_problem(3, 5, 3, 2)
    if straight:
        prob = straightened_problem(prob, 2, 1)
    D = Discretization(prob)
    ctx, _ = gpu_ctx(prob, "face")
    xq = ctx.sn_volume_points()
    assert xq.shape == D.xq.shape
    assert np.allclose(xq, D.xq, rtol=0, atol=1e-14)
    rng = np.random.default_rng(5)
    phi = rng.uniform(-1.0, 1.0, size=(prob.mesh.n_elem, D.N))
    exact = np.sin(3 * D.xq[..., 0]) * np.cos(2 * D.xq[..., 1])
    ref = _oracle_l2(D, np.einsum("qm,em->eq", D.B, phi) - exact)
    got = ctx.sn_l2_error(phi, exact)
    assert abs(got - ref) <= 1e-12 * ref, (got, ref)


@pytest.mark.parametrize("prec", [0, 4])
def test_mms_errors_high_order_and_straightened_match_the_oracle(prec):
    for prob in (annulus_problem(3, 6, 3, 3), straightened_problem(annulus_problem(3, 6, 3, 3), 3, 1)):
        prob, fex, fac = annulus_mms(prob)
        D = Discretization(prob)
        R = Sweeper(D, build_graph(D, "face")).source_iterate(tol=1e-12)
        ref = _oracle_l2(D, np.einsum("qm,em->eq", D.B, R["phi"]) - fac * fex(D.xq))
        ctx, _ = gpu_ctx(prob, "face")
        phi = np.zeros((prob.mesh.n_elem, D.N))
        res = ctx.sn_source_iterate(1e-12, 500, prec, phi_out=phi)
        assert res["converged"]
        got = ctx.sn_l2_error(phi, fac * fex(ctx.sn_volume_points()))
        print(f"{prob.name} prec={prec}: L2 error GPU {got:.6e}, oracle {ref:.6e}")
        assert abs(got - ref) <= 1e-6 * ref, (got, ref)
