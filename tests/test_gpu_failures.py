"""Failure handling through the C ABI: every error path returns its status code and leaves the
context usable.  No GPU fault is provoked: the dataflow timeout is made to happen by lowering the
poll limit of the bounded dependency wait (the kernel gives up, sets its error word and returns),
and every other failure is an invalid input rejected on the host."""
import numpy as np
import pytest

import sn_inputs as si
from gpu_util import oracle_graph, gpu_ctx, rel_l2, random_state
from oracle.sweep import Sweeper

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1810_11080_gb300 as g   # noqa: E402


def _status(fn, *a, **k):
    try:
        fn(*a, **k)
    except g.SnError as ex:
        return ex.status
    return g.SN_OK


@pytest.mark.parametrize("prec", [0, 2, 3, 4])
def test_dataflow_wait_limit_gives_timeout_then_recovers(prec):
    prob = si.make_config("2d_smooth_q3_p3_s8", n=24)
    ctx, _ = gpu_ctx(prob, "face")
    phi, psi_old = random_state(prob, seed=11)
    ref = np.zeros_like(psi_old)
    ctx.sn_set_launch(g.SN_LAUNCH_LEVELS)
    ctx.sn_sweep(phi, psi_old, ref, prec)
    ctx.sn_set_launch(g.SN_LAUNCH_DATAFLOW)
    ctx.sn_set_spin_limit(1)      # a wait that polls its flag twice without success gives up
    out = np.zeros_like(psi_old)
    assert _status(ctx.sn_sweep, phi, psi_old, out, prec) == g.SN_ETIMEOUT
    assert "spin limit" in g.lib().sn_last_error(ctx._c).decode()
    # the source iteration path reports the same status
    ctx.sn_si_begin(None)
    assert _status(ctx.sn_si_step, prec) == g.SN_ETIMEOUT
    # default limit again: the same context sweeps correctly, bit for bit as the level schedule
    ctx.sn_set_spin_limit(0)
    out = np.full_like(psi_old, np.nan)
    ctx.sn_sweep(phi, psi_old, out, prec)
    assert np.array_equal(out, ref)
    assert _status(ctx.sn_set_spin_limit, -1) == g.SN_EINVAL


def test_source_iteration_not_converged_still_writes_results():
    prob = si.make_config("2d_sine_q2_p1_s4", n=8, p=2)
    disc, G = oracle_graph(prob, "face")
    ref = Sweeper(disc, G).source_iterate(tol=1e-8, max_iter=2)
    ctx, _ = gpu_ctx(prob, "face")
    phi = np.full((disc.E, disc.N), np.nan)
    res = ctx.sn_source_iterate(1e-8, 2, g.SN_PREC_FP64, phi_out=phi, history_cap=4)
    assert res["status"] == g.SN_ENOTCONVERGED and not res["converged"] and res["iters"] == 2
    assert rel_l2(phi, ref["phi"]) <= 1e-11
    np.testing.assert_allclose(res["history"], ref["history"], rtol=1e-9)


def test_mesh_errors():
    prob = si.make_config("2d_sine_q2_p1_s4", n=4)
    m = prob.mesh
    ctx = g.Context(0, torch.cuda.Stream().cuda_stream)
    bad = m.face_nbr.copy()
    e = 5
    f = int(np.nonzero(bad[e] >= 0)[0][0])
    other = [x for x in range(m.n_elem) if x not in (e, bad[e, f])][0]
    bad[e, f] = other                                   # e names `other`, which does not name e back
    assert _status(ctx.sn_set_mesh, m.dim, m.n_elem, m.r, np.ascontiguousarray(m.ctrl), bad.astype(np.int64),
                   np.ascontiguousarray(m.nbr_face, dtype=np.int32),
                   np.ascontiguousarray(m.orient, dtype=np.int32)) == g.SN_EMESH
    # a mirrored element: its map reverses orientation, det J < 0 at every volume point
    ctrl = m.ctrl.copy()
    r = m.r
    for b in range(r + 1):
        for a in range(r + 1):
            ctrl[e, a + (r + 1) * b] = m.ctrl[e, (r - a) + (r + 1) * b]
    bad_prob = si.make_config("2d_sine_q2_p1_s4", n=4)
    bad_prob.mesh.ctrl = ctrl
    ctx2 = g.setup_problem(bad_prob, device=0, stream=torch.cuda.Stream().cuda_stream)
    assert _status(ctx2.sn_build_graph, "face", 10) == g.SN_EMESH
    assert "det J" in g.lib().sn_last_error(ctx2._c).decode()
    # state is clean afterwards: a sweep is refused, the valid mesh builds
    assert _status(ctx2.sn_sweep, np.zeros((16, 4)), np.zeros((12, 16, 4)), np.zeros((12, 16, 4)), 0) == g.SN_ESTATE
    g.setup_problem(prob, ctx=ctx2)
    ctx2.sn_build_graph("face", 10)


def test_invalid_inputs():
    prob = si.make_config("2d_sine_q2_p1_s4", n=4)
    ctx = g.setup_problem(prob, device=0, stream=torch.cuda.Stream().cuda_stream)
    st = prob.sigma_t.copy()
    st[3] = np.nan
    assert _status(ctx.sn_set_materials, st, prob.sigma_s, prob.q) == g.SN_EINVAL
    assert _status(ctx.sn_set_materials, prob.sigma_t, -prob.sigma_s, prob.q) == g.SN_EINVAL
    assert _status(ctx.sn_set_materials, 0.0 * prob.sigma_t, prob.sigma_s, prob.q) == g.SN_EINVAL
    w = prob.w.copy()
    w[2] = 0.0
    assert _status(ctx.sn_set_quadrature, np.ascontiguousarray(prob.omega), w) == g.SN_EINVAL
    om = np.ascontiguousarray(prob.omega).copy()
    om[0, 0] = np.inf
    assert _status(ctx.sn_set_quadrature, om, prob.w) == g.SN_EINVAL
    assert _status(ctx.sn_set_discretization, 4, 2) == g.SN_EINVAL
    assert _status(ctx.sn_build_graph, 3, 10) == g.SN_EINVAL
    assert _status(ctx.sn_set_launch, 7, 0) == g.SN_EINVAL
    ctx.sn_build_graph("face", 10)
    z = np.zeros((len(prob.w), prob.mesh.n_elem, 4))
    assert _status(ctx.sn_sweep, np.zeros((prob.mesh.n_elem, 4)), z, z.copy(), 5) == g.SN_EINVAL
    assert _status(ctx.sn_prepare_inverse, g.SN_PREC_MIXED_DS) == g.SN_EINVAL


def test_calls_out_of_order():
    prob = si.make_config("2d_sine_q2_p1_s4", n=4)
    ctx = g.Context(0, torch.cuda.Stream().cuda_stream)
    assert _status(ctx.sn_set_discretization, 1, 2) == g.SN_ESTATE              # before the mesh
    ctx = g.setup_problem(prob, device=0, stream=torch.cuda.Stream().cuda_stream)
    E, N, M = prob.mesh.n_elem, 4, len(prob.w)
    z = np.zeros((M, E, N))
    assert _status(ctx.sn_sweep, np.zeros((E, N)), z, z.copy(), 0) == g.SN_ESTATE   # before the graph
    assert _status(ctx.sn_si_begin, None) == g.SN_ESTATE
    assert _status(ctx.sn_autotune, 0) == g.SN_ESTATE
    assert _status(ctx.sn_prepare_inverse) == g.SN_ESTATE
    ctx.sn_build_graph("face", 10)
    assert _status(ctx.sn_si_step, 0) == g.SN_ESTATE                            # before sn_si_begin
    ctx.sn_si_begin(None)
    ctx.sn_si_step(0)
    # changing the materials drops the graph: sweeps are refused until it is rebuilt
    ctx.sn_set_materials(prob.sigma_t * 2, prob.sigma_s, prob.q)
    assert _status(ctx.sn_sweep, np.zeros((E, N)), z, z.copy(), 0) == g.SN_ESTATE
