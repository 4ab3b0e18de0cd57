"""Triangles (P_r geometry, P_p DG; Sec. 2 simplicial elements) on the GPU against the oracle:
graph bit-exact, one lagged sweep of both stored-inverse forms, source iteration, the
manufactured-solution error, schedules bitwise equal, and the refused forms."""
import numpy as np
import pytest

from sn_inputs.configs import triangle_problem
from sn_inputs.mms import annulus_mms
from gpu_util import oracle_graph, gpu_ctx, rel_l2, random_state
from oracle.sweep import Sweeper

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

FP64_TOL = 1e-11
DS_TOL = 1e-11

CASES = {
    "tri_6_r2_p1": lambda: triangle_problem(6, 2, 1, amp=0.06),
    "tri_6_r2_p2": lambda: triangle_problem(6, 2, 2, amp=0.06),
    "tri_5_r3_p3": lambda: triangle_problem(5, 3, 3, amp=0.07),
    "tri_8_r3_p2_s8": lambda: triangle_problem(8, 3, 2, sn=8, amp=0.05),
    "tri_5_r2_p3_rotated": lambda: triangle_problem(5, 2, 3, amp=0.06, rotate_seed=4),
}


def _random_state(prob, seed):
    rng = np.random.default_rng(seed)
    N = (prob.p + 1) * (prob.p + 2) // 2
    M, E = len(prob.w), prob.mesh.n_elem
    return rng.uniform(0.5, 2.0, size=(E, N)), rng.uniform(0.0, 1.0, size=(M, E, N))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("weighting", ["unity", "face", "siginvface"])
def test_triangle_graph_bit_exact(case, weighting):
    prob = CASES[case]()
    disc, G = oracle_graph(prob, weighting)
    ctx, stats = gpu_ctx(prob, weighting)
    removed, levels = ctx.sn_get_graph(len(prob.w), prob.mesh.n_elem)
    assert np.array_equal(removed, G["removed"]), (len(removed), len(G["removed"]))
    assert np.array_equal(levels, G["levels"])


@pytest.mark.parametrize("prec", [3, 4])
@pytest.mark.parametrize("case", list(CASES))
def test_triangle_sweep_parity(case, prec):
    prob = CASES[case]()
    disc, G = oracle_graph(prob, "face")
    ctx, _ = gpu_ctx(prob, "face")
    phi, psi_old = _random_state(prob, 7)
    ref = Sweeper(disc, G).sweep(phi, psi_old)
    out = np.zeros_like(psi_old)
    ctx.sn_sweep(phi, psi_old, out, prec)
    err = rel_l2(out, ref)
    print(f"{case} prec={prec}: rel L2 {err:.3e}")
    assert err <= (FP64_TOL if prec == 3 else DS_TOL), err


@pytest.mark.parametrize("prec", [3, 4])
def test_triangle_schedules_bitwise_equal(prec):
    import paper_1810_11080_gb300 as g
    prob = CASES["tri_8_r3_p2_s8"]()
    ctx, _ = gpu_ctx(prob, "face")
    phi, psi_old = _random_state(prob, 8)
    ref = np.zeros_like(psi_old)
    ctx.sn_set_launch(g.SN_LAUNCH_LEVELS)
    ctx.sn_sweep(phi, psi_old, ref, prec)
    for bps in (0, 1):
        out = np.full_like(psi_old, np.nan)
        ctx.sn_set_launch(g.SN_LAUNCH_DATAFLOW, bps)
        ctx.sn_sweep(phi, psi_old, out, prec)
        assert np.array_equal(out, ref)


@pytest.mark.parametrize("prec", [3, 4])
def test_triangle_mms_error_matches_the_oracle(prec):
    prob, fex, fac = annulus_mms(triangle_problem(6, 3, 3))
    disc, G = oracle_graph(prob, "face")
    R = Sweeper(disc, G).source_iterate(tol=1e-12)
    v = np.einsum("qm,em->eq", disc.B, R["phi"]) - fac * fex(disc.xq)
    ref = float(np.sqrt(np.einsum("q,eq,eq->", disc.wq, disc.detJ, v * v)))
    ctx, _ = gpu_ctx(prob, "face")
    xq = ctx.sn_volume_points()
    assert np.allclose(xq, disc.xq, rtol=0, atol=1e-14)
    phi = np.zeros((prob.mesh.n_elem, 10))
    res = ctx.sn_source_iterate(1e-12, 500, prec, phi_out=phi)
    assert res["converged"] and res["iters"] == R["iters"]
    assert rel_l2(phi, R["phi"]) <= 1e-10
    got = ctx.sn_l2_error(phi, fac * fex(xq))
    print(f"triangle MMS prec={prec}: GPU {got:.6e}, oracle {ref:.6e}")
    assert abs(got - ref) <= 1e-6 * ref


def test_triangles_refuse_the_other_forms():
    import paper_1810_11080_gb300 as g
    prob = CASES["tri_6_r2_p1"]()
    ctx, _ = gpu_ctx(prob, "face")
    phi, psi_old = _random_state(prob, 9)
    for prec in (0, 1, 2):
        with pytest.raises(g.SnError) as ex:
            ctx.sn_sweep(phi, psi_old, np.zeros_like(psi_old), prec)
        assert ex.value.status == g.SN_EINVAL
