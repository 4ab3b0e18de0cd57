"""Batched persistent sweeps over many uneven problems: identical to solving each problem alone,
and converged to the oracle."""
import numpy as np
import pytest

import sn_inputs as si
from gpu_util import oracle_graph, gpu_ctx, rel_l2
from oracle.sweep import Sweeper

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def small_batch(count=9, seed=31):
    probs = si.batch_problems(count=count, seed=seed, nmin=3, nmax=9)
    return probs


def make_ctxs(probs, stream):
    import paper_1810_11080_gb300 as g
    ctxs = []
    for prob in probs:
        c = g.setup_problem(prob, device=0, stream=stream.cuda_stream)
        c.sn_build_graph("face", 10)
        ctxs.append(c)
    return ctxs


@pytest.mark.parametrize("prec", [0, 2, 3, 4])
@pytest.mark.parametrize("mode", [0, 1])
def test_batch_steps_equal_single_problem_steps(prec, mode):
    import paper_1810_11080_gb300 as g
    probs = small_batch()
    assert len({p.p for p in probs}) > 1 and len({p.mesh.n_elem for p in probs}) > 1
    stream = torch.cuda.Stream()
    solo = make_ctxs(probs, stream)
    team = make_ctxs(probs, stream)
    batch = g.Batch(team, stream.cuda_stream)
    batch.sn_batch_set_launch(mode, 0)
    batch.sn_batch_si_begin()
    for c in solo:
        c.sn_si_begin()
    for step in range(4):
        res_b, _ = batch.sn_batch_si_step(prec)
        for k, c in enumerate(solo):
            r, _ = c.sn_si_step(prec)
            assert r == res_b[k], (step, k, r, res_b[k])
    for k, (a, b) in enumerate(zip(solo, team)):
        E, N, M = probs[k].mesh.n_elem, (probs[k].p + 1) ** 2, len(probs[k].w)
        pa, pb = np.zeros((E, N)), np.zeros((E, N))
        sa, sb = np.zeros((M, E, N)), np.zeros((M, E, N))
        a.sn_si_result(pa, sa)
        b.sn_si_result(pb, sb)
        assert np.array_equal(pa, pb) and np.array_equal(sa, sb), k


def test_batch_source_iteration_matches_oracle():
    import paper_1810_11080_gb300 as g
    probs = small_batch(count=5, seed=7)
    stream = torch.cuda.Stream()
    ctxs = make_ctxs(probs, stream)
    batch = g.Batch(ctxs, stream.cuda_stream)
    out = batch.sn_batch_source_iterate(1e-11, 2000, 2)
    assert out["status"] == 0 and np.all(out["iters"] > 0)
    for k, prob in enumerate(probs):
        disc, G = oracle_graph(prob, "face")
        ref = Sweeper(disc, G).source_iterate(tol=1e-12)
        phi = np.zeros((prob.mesh.n_elem, (prob.p + 1) ** 2))
        ctxs[k].sn_si_result(phi, None)
        assert rel_l2(phi, ref["phi"]) <= 1e-9, (k, rel_l2(phi, ref["phi"]))


def test_autotuners_pick_a_valid_schedule():
    import paper_1810_11080_gb300 as g
    probs = small_batch(count=4, seed=3)
    stream = torch.cuda.Stream()
    ctxs = make_ctxs(probs, stream)
    batch = g.Batch(ctxs, stream.cuda_stream)
    mode, bps = batch.sn_batch_tune(2)
    assert mode in (0, 1) and 0 <= bps <= 64
    res, _ = batch.sn_batch_si_step(2)
    assert np.all(np.isfinite(res))
    m1, b1 = ctxs[0].sn_autotune(2)
    assert m1 in (0, 1)
