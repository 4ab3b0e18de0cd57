"""Learned flux predictor: the library's MLP kernels against the FP64 oracle MLP, predictor data,
and source iteration with the predictor (same fixed point as plain source iteration; gain)."""
import os

import numpy as np
import pytest

import sn_inputs as si
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1810_11080_gb300",
                     "models", "predictor_3d_q2_p2_s12.npz")


def effective_params(theta, n_in, n_out):
    """The parameters the device uses: weights rounded to BF16, biases FP32."""
    th = np.asarray(theta, dtype=np.float32).astype(np.float64)
    o = 0
    for shape in omlp.shapes(n_in, n_out):
        k = int(np.prod(shape))
        if len(shape) == 2:
            th[o:o + k] = omlp.bf16_round(th[o:o + k])
        o += k
    return th


@pytest.mark.parametrize("n_in,n_out", [(16, 27), (18, 1), (16, 9)])
def test_mlp_forward_and_gradient_match_oracle(n_in, n_out):
    import paper_1810_11080_gb300 as g
    rng = np.random.default_rng(n_in + n_out)
    net = g.MLP(n_in, n_out, seed=5)
    theta = rng.normal(0, 0.2, size=net.sn_mlp_num_params()).astype(np.float32)
    net.set_params(theta)
    x = rng.normal(size=(1000, n_in)).astype(np.float32)
    t = rng.normal(size=(1000, n_out)).astype(np.float32)
    th = effective_params(theta, n_in, n_out)
    y_ref, _ = omlp.forward(th, x.astype(np.float64), n_out)
    y = net.sn_mlp_forward(x)
    assert np.abs(y - y_ref).max() <= 1e-4 * max(1.0, np.abs(y_ref).max())
    L, grad = net.sn_mlp_grad(x, t)
    L_ref, g_ref = omlp.loss_grad(th, x.astype(np.float64), t.astype(np.float64), n_out)
    assert abs(L - L_ref) <= 1e-5 * L_ref
    rel = np.linalg.norm(grad - g_ref) / np.linalg.norm(g_ref)
    print(f"MLP gradient rel L2 vs FP64 oracle ({n_in}->{n_out}): {rel:.2e}")
    assert rel <= 1e-4


def test_mlp_training_reduces_loss():
    import paper_1810_11080_gb300 as g
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, size=(20000, 6)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0] + x[:, 1]), x[:, 2] * x[:, 3]], 1).astype(np.float32)
    net = g.MLP(6, 2, seed=1)
    L0, _ = net.sn_mlp_grad(x, t)
    net.sn_mlp_train(x, t, epochs=30, batch_rows=512, lr=3e-3, seed=2)
    L1, _ = net.sn_mlp_grad(x, t)
    assert L1 < 0.05 * L0, (L0, L1)


def test_predictor_features():
    import paper_1810_11080_gb300 as g
    prob = si.make_config("3d_smooth_q2_p2_s12", n=4, sn=4, seed=5000)
    ctx = g.setup_problem(prob)
    ctx.sn_build_graph("face", 10)
    feat, ref = ctx.sn_predictor_features()
    assert feat.shape == (64, 16)
    np.testing.assert_allclose(feat[:, 0], prob.sigma_t, rtol=1e-6)
    np.testing.assert_allclose(feat[:, 1], prob.sigma_s, rtol=1e-6)
    assert abs(feat[:, 8].sum() - 1.0) < 1e-5                      # volumes of the unit cube
    nb = (prob.mesh.face_nbr < 0).sum(1)
    np.testing.assert_array_equal(feat[:, 11], nb)
    phi = np.ones((64, 27))
    t = ctx.sn_predictor_init_targets(phi)
    np.testing.assert_allclose(t, np.broadcast_to(1.0 / ref[:, None], t.shape), rtol=1e-6)


def small_model(stream):
    from paper_1810_11080_gb300 import learned
    probs = [si.make_config("3d_smooth_q2_p2_s12", n=4, sn=4, seed=1000 + 2 * k) for k in range(24)]
    data = learned.generate(probs, stream=stream.cuda_stream)
    return learned.train(data, epochs=30, batch_rows=1024, lr=3e-3, stream=stream.cuda_stream)


def test_learned_source_iteration_keeps_the_fixed_point():
    import paper_1810_11080_gb300 as g
    from paper_1810_11080_gb300 import learned
    stream = torch.cuda.Stream()
    model = small_model(stream)
    init, corr, cfg = learned.build(model, stream=stream.cuda_stream)
    prob = si.make_config("3d_smooth_q2_p2_s12", n=6, sn=4, seed=5000)
    ctx = g.setup_problem(prob, stream=stream.cuda_stream)
    ctx.sn_build_graph("face", 10)
    E, N = prob.mesh.n_elem, 27
    phi_plain, phi_learn = np.zeros((E, N)), np.zeros((E, N))
    plain = ctx.sn_source_iterate(1e-11, 3000, 0, phi_out=phi_plain)
    res = ctx.sn_source_iterate_learned(1e-11, 3000, 0, init, corr, cfg, phi_out=phi_learn)
    print(f"plain {plain['iters']} iterations, learned {res['iters']} (accepted {res['accepted']}, "
          f"rejected {res['rejected']})")
    assert res["converged"]
    assert np.linalg.norm(phi_learn - phi_plain) / np.linalg.norm(phi_plain) <= 1e-8
    assert res["iters"] <= plain["iters"] + 2


@pytest.mark.skipif(not os.path.exists(MODEL), reason="trained predictor not present")
def test_trained_predictor_gains_over_plain_source_iteration():
    import paper_1810_11080_gb300 as g
    from paper_1810_11080_gb300 import learned
    stream = torch.cuda.Stream()
    init, corr, cfg = learned.build(learned.load(MODEL), stream=stream.cuda_stream)
    total_plain = total_learned = 0
    for seed in (5000, 5002):
        prob = si.make_config("3d_smooth_q2_p2_s12", n=12, seed=seed)
        ctx = g.setup_problem(prob, stream=stream.cuda_stream)
        ctx.sn_build_graph("face", 10)
        E, N = prob.mesh.n_elem, 27
        phi_plain, phi_learn = np.zeros((E, N)), np.zeros((E, N))
        plain = ctx.sn_source_iterate(1e-8, 5000, 0, phi_out=phi_plain)
        res = ctx.sn_source_iterate_learned(1e-8, 5000, 0, init, corr, cfg, phi_out=phi_learn)
        print(f"seed {seed}: plain {plain['iters']} it {plain['ms_total']:.0f} ms; learned {res['iters']} it "
              f"{res['ms_total']:.0f} ms (accepted {res['accepted']}, rejected {res['rejected']})")
        assert res["converged"] and res["iters"] < plain["iters"]
        assert np.linalg.norm(phi_learn - phi_plain) / np.linalg.norm(phi_plain) <= 1e-6
        total_plain += plain["iters"]
        total_learned += res["iters"]
    assert total_learned <= 0.9 * total_plain, (total_learned, total_plain)
