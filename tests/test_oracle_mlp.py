"""Pins of the reference MLP: back-propagation against central finite differences, the BF16
rounding against a brute-force nearest-representable search, and a closed-form special case."""
import numpy as np
import pytest

from oracle import mlp


@pytest.mark.parametrize("n_in,n_out", [(16, 27), (18, 1), (5, 3)])
def test_backprop_matches_finite_differences(n_in, n_out):
    rng = np.random.default_rng(n_in)
    theta = rng.normal(0, 0.3, size=mlp.n_params(n_in, n_out))
    x = rng.normal(size=(23, n_in))
    t = rng.normal(size=(23, n_out))
    L, g = mlp.loss_grad(theta, x, t, n_out)
    idx = rng.choice(len(theta), size=40, replace=False)
    fd = mlp.finite_difference_grad(theta, x, t, n_out, idx)
    assert np.allclose(g[idx], fd, rtol=1e-6, atol=1e-9)


def test_linear_output_layer_special_case():
    """With W1 = W2 = 0 the hidden states are tanh(b), constant: y = tanh(tanh(b1) W2 + b2) W3 + b3."""
    n_in, n_out = 4, 2
    rng = np.random.default_rng(1)
    theta = np.zeros(mlp.n_params(n_in, n_out))
    W1, b1, W2, b2, W3, b3 = mlp.unpack(theta, n_in, n_out)
    o = n_in * 64
    theta[o:o + 64] = rng.normal(size=64)            # b1
    o2 = o + 64 + 64 * 64
    theta[o2:o2 + 64] = rng.normal(size=64)          # b2
    o3 = o2 + 64
    theta[o3:o3 + 64 * n_out] = rng.normal(size=64 * n_out)
    y, _ = mlp.forward(theta, rng.normal(size=(3, n_in)), n_out)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(theta, n_in, n_out)
    expect = np.tanh(b2) @ W3 + b3
    assert np.allclose(y, expect[None, :], atol=1e-14)


def test_bf16_rounding_is_nearest_even():
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.normal(size=200), [1.0, -2.5, 3.0e-3, 0.0]]).astype(np.float32)
    r = mlp.bf16_round(v)
    for a, b in zip(v.astype(np.float64), r):
        # brute force: neighbours on the bf16 grid around a
        u = np.array([a], dtype=np.float32).view(np.uint32)[0] & 0xFFFF0000
        cands = [np.array([u], dtype=np.uint32).view(np.float32)[0],
                 np.array([u + 0x10000], dtype=np.uint32).view(np.float32)[0]]
        best = min(cands, key=lambda c: (abs(float(c) - a), int(np.array([c], np.float32).view(np.uint32)[0] >> 16) & 1))
        assert b == float(best), (a, b, best)
