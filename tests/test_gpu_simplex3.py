"""Straight-sided tetrahedra (P_1 geometry, P_1 / P_2 DG; Sec. 2 simplicial elements) on the GPU
against the oracle: graph bit-exact (including the lagged arcs of a twisted column), one lagged
sweep of both stored-inverse forms, the schedules bitwise equal, source iteration, volume
points and the pure-absorber error, and the refused forms."""
import math

import numpy as np
import pytest

from sn_inputs.configs import tet_problem
from sn_inputs.mms import attenuation
from gpu_util import oracle_graph, gpu_ctx, rel_l2
from oracle.sweep import Sweeper

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

FP64_TOL = 1e-11
DS_TOL = 1e-11

CASES = {
    "tet_3_p1": lambda: tet_problem(3, 1),
    "tet_3_p2_rotated": lambda: tet_problem(3, 2, rotate_seed=5),
    "tet_4_p1_twist2_s8": lambda: tet_problem(4, 1, sn=8, twist=2.0),
    "tet_4_p2_twist2_s8_rotated": lambda: tet_problem(4, 2, sn=8, twist=2.0, rotate_seed=2),
    "tet_3_p2_twist2.5": lambda: tet_problem(3, 2, twist=2.5),
}


def _random_state(prob, seed):
    rng = np.random.default_rng(seed)
    N = (prob.p + 1) * (prob.p + 2) * (prob.p + 3) // 6
    M, E = len(prob.w), prob.mesh.n_elem
    return rng.uniform(0.5, 2.0, size=(E, N)), rng.uniform(0.0, 1.0, size=(M, E, N))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("weighting", ["unity", "face", "siginvface"])
def test_tet_graph_bit_exact(case, weighting):
    prob = CASES[case]()
    disc, G = oracle_graph(prob, weighting)
    if "twist" in case:
        assert len(G["removed"]) > 0                   # the twisted columns have cycles to lag
    ctx, stats = gpu_ctx(prob, weighting)
    removed, levels = ctx.sn_get_graph(len(prob.w), prob.mesh.n_elem)
    assert np.array_equal(removed, G["removed"]), (len(removed), len(G["removed"]))
    assert np.array_equal(levels, G["levels"])


@pytest.mark.parametrize("prec", [3, 4])
@pytest.mark.parametrize("case", list(CASES))
def test_tet_sweep_parity(case, prec):
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
def test_tet_schedules_bitwise_equal(prec):
    import paper_1810_11080_gb300 as g
    prob = CASES["tet_4_p2_twist2_s8_rotated"]()
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
def test_tet_source_iteration_matches_the_oracle(prec):
    prob = CASES["tet_3_p2_twist2.5"]()
    disc, G = oracle_graph(prob, "face")
    R = Sweeper(disc, G).source_iterate(tol=1e-12)
    ctx, _ = gpu_ctx(prob, "face")
    phi = np.zeros((prob.mesh.n_elem, 10))
    res = ctx.sn_source_iterate(1e-12, 500, prec, phi_out=phi)
    assert res["converged"] and res["iters"] == R["iters"]
    assert rel_l2(phi, R["phi"]) <= 1e-10


@pytest.mark.parametrize("prec", [3, 4])
def test_tet_pure_absorber_error_matches_the_oracle(prec):
    """Volume points and the L2 error of the scalar flux of the attenuation problem against the
    oracle's (sigma_s = 0: one sweep is the solution)."""
    prob, exact = attenuation(tet_problem(4, 2, rotate_seed=1), sigma_t=2.0)
    disc, G = oracle_graph(prob, "face")
    R = Sweeper(disc, G).source_iterate(tol=1e-13)
    ctx, _ = gpu_ctx(prob, "face")
    xq = ctx.sn_volume_points()
    assert xq.shape == disc.xq.shape
    assert np.allclose(xq, disc.xq, rtol=0, atol=1e-14)
    phi = np.zeros((prob.mesh.n_elem, 10))
    res = ctx.sn_source_iterate(1e-13, 50, prec, phi_out=phi)
    assert res["converged"]
    assert rel_l2(phi, R["phi"]) <= 1e-10
    phi_ex = sum(disc.w[d] * exact(disc.xq, d) for d in range(disc.M_dirs))
    v = np.einsum("qm,em->eq", disc.B, R["phi"]) - phi_ex
    ref = math.sqrt(float(np.einsum("q,eq,eq->", disc.wq, disc.detJ, v * v)))
    got = ctx.sn_l2_error(phi, phi_ex)
    print(f"tet absorber prec={prec}: GPU {got:.6e}, oracle {ref:.6e}")
    assert abs(got - ref) <= 1e-6 * ref


def test_tets_refuse_the_other_forms():
    import paper_1810_11080_gb300 as g
    prob = CASES["tet_3_p1"]()
    ctx, _ = gpu_ctx(prob, "face")
    phi, psi_old = _random_state(prob, 9)
    for prec in (0, 1, 2):
        with pytest.raises(g.SnError) as ex:
            ctx.sn_sweep(phi, psi_old, np.zeros_like(psi_old), prec)
        assert ex.value.status == g.SN_EINVAL
