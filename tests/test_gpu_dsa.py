"""Diffusion synthetic acceleration through the C ABI against the oracle (oracle/dsa.py): one
correction from the same (phi_half, phi_prev), the accelerated source iteration's fixed point and
its iteration count on a scattering-dominated problem."""
import numpy as np
import pytest

import sn_inputs as si
from gpu_util import oracle_graph, gpu_ctx, rel_l2
from oracle.dsa import DiffusionOperator, dsa_source_iterate
from oracle.sweep import Sweeper

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1810_11080_gb300 as g   # noqa: E402


def _curved2d(n=8, p=2):
    prob = si.make_config("2d_sine_q2_p1_s4", n=n, p=p)
    prob.mesh = si.structured_mesh((n, n), 2, si.disp_sine_2d(0.08))
    prob.sigma_t = np.linspace(0.5, 4.0, prob.mesh.n_elem)
    prob.sigma_s = 0.95 * prob.sigma_t
    return prob


CASES = {
    "2d_curved_8_p2": lambda: _curved2d(8, 2),
    "2d_smooth_6_p3": lambda: si.make_config("2d_smooth_q3_p3_s8", n=6),
    "3d_twist_3_p2": lambda: si.make_config("3d_twist_q2_p2_s8", n=3, sn=4),
    "3d_twist_3_p1_reoriented": lambda: si.make_config("3d_twist_q2_p2_s8", n=3, p=1, sn=4, reorient_seed=5),
}


@pytest.mark.parametrize("case", list(CASES))
def test_dsa_correction_matches_oracle(case):
    prob = CASES[case]()
    disc, _G = oracle_graph(prob, "face")
    ctx, _ = gpu_ctx(prob, "face")
    rng = np.random.default_rng(4)
    half = rng.uniform(0.5, 2.0, size=(disc.E, disc.N))
    prev = half + rng.uniform(-0.2, 0.2, size=half.shape)
    ref = half + DiffusionOperator(disc).correction(half, prev)
    ctx.sn_set_dsa(True, 1e-13, 5000)
    out = np.zeros_like(half)
    it = ctx.sn_dsa_correction(half, prev, out)
    err = rel_l2(out - half, ref - half)
    print(f"DSA correction {case}: CG iterations {it}, rel L2 of dphi vs oracle {err:.3e}")
    assert 0 < it < 5000
    assert err <= 1e-9


def test_dsa_source_iteration_keeps_the_fixed_point_and_matches_the_oracle_iterations():
    prob = _curved2d(8, 2)
    disc, G = oracle_graph(prob, "face")
    S = Sweeper(disc, G)
    ref = dsa_source_iterate(S, DiffusionOperator(disc), tol=1e-10)
    plain = S.source_iterate(tol=1e-12)
    ctx, _ = gpu_ctx(prob, "face")
    ctx.sn_set_dsa(True, 1e-12, 5000)
    phi = np.zeros((disc.E, disc.N))
    res = ctx.sn_source_iterate(1e-10, 500, g.SN_PREC_FP64, phi_out=phi, history_cap=500)
    assert res["converged"] and ref["converged"]
    assert abs(res["iters"] - ref["iters"]) <= 1
    np.testing.assert_allclose(res["history"][:6], ref["history"][:6], rtol=1e-6)
    assert rel_l2(phi, plain["phi"]) <= 1e-9


@pytest.mark.parametrize("prec", [0, 2])
def test_dsa_cuts_the_iterations_of_a_scattering_dominated_problem(prec):
    prob = si.make_config("2d_sine_q2_p1_s4", n=16, p=2)
    prob.sigma_t = 20.0 * np.ones(prob.mesh.n_elem)
    prob.sigma_s = 0.995 * prob.sigma_t
    ctx, _ = gpu_ctx(prob, "face")
    E, N = prob.mesh.n_elem, 9
    phi0, phi1 = np.zeros((E, N)), np.zeros((E, N))
    plain = ctx.sn_source_iterate(1e-8, 5000, prec, phi_out=phi0)
    ctx.sn_set_dsa(True, 1e-4, 500)
    acc = ctx.sn_source_iterate(1e-8, 5000, prec, phi_out=phi1)
    print(f"prec {prec}: plain {plain['iters']} iterations, DSA {acc['iters']} (last CG {ctx.sn_dsa_last_iters()})")
    assert plain["converged"] and acc["converged"]
    assert acc["iters"] * 8 <= plain["iters"]
    assert rel_l2(phi1, phi0) <= 1e-6


def test_dsa_arguments_are_checked():
    prob = si.make_config("2d_sine_q2_p1_s4", n=4)
    ctx, _ = gpu_ctx(prob, "face")
    for args in ((2, 1e-4, 10), (1, 0.0, 10), (1, 1.5, 10), (1, 1e-4, 0)):
        with pytest.raises(g.SnError) as ex:
            ctx.sn_set_dsa(*args)
        assert ex.value.status == g.SN_EINVAL
