"""Reference per-element MLP of the learned flux predictor (not from the paper: the learned
predictor is this project's addition).  FP64, plain numpy.

Architecture: x [rows, n_in] -> tanh(x W1 + b1) -> tanh(h1 W2 + b2) -> h2 W3 + b3, width 64.
Packed parameter order (shared with the library): W1 [n_in][64] row-major, b1 [64],
W2 [64][64], b2 [64], W3 [64][n_out], b3 [n_out].
Loss: L = sum (y - t)^2 / (2 rows n_out).
"""
import numpy as np

HIDDEN = 64


def shapes(n_in, n_out, h=HIDDEN):
    return [(n_in, h), (h,), (h, h), (h,), (h, n_out), (n_out,)]


def n_params(n_in, n_out, h=HIDDEN):
    return sum(int(np.prod(s)) for s in shapes(n_in, n_out, h))


def unpack(theta, n_in, n_out, h=HIDDEN):
    out, o = [], 0
    for s in shapes(n_in, n_out, h):
        k = int(np.prod(s))
        out.append(np.asarray(theta[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def bf16_round(a):
    """Round float values to bfloat16 (round to nearest even on the top 16 bits of the FP32
    pattern), returned as float64."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, x, n_out):
    x = np.asarray(x, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(theta, x.shape[1], n_out)
    h1 = np.tanh(x @ W1 + b1)
    h2 = np.tanh(h1 @ W2 + b2)
    return h2 @ W3 + b3, (x, h1, h2)


def loss_grad(theta, x, t, n_out):
    """(L, dL/dtheta) by back-propagation."""
    y, (x, h1, h2) = forward(theta, x, n_out)
    rows = x.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    L = 0.5 * np.sum(r * r) / (rows * n_out)
    dy = r / (rows * n_out)
    W1, b1, W2, b2, W3, b3 = unpack(theta, x.shape[1], n_out)
    gW3 = h2.T @ dy
    gb3 = dy.sum(0)
    dz2 = (dy @ W3.T) * (1.0 - h2 * h2)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2.T) * (1.0 - h1 * h1)
    gW1 = x.T @ dz1
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def finite_difference_grad(theta, x, t, n_out, idx, eps=1e-6):
    """Central differences of the loss for the parameter indices idx."""
    out = []
    for i in idx:
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += eps
        tm[i] -= eps
        out.append((loss_grad(tp, x, t, n_out)[0] - loss_grad(tm, x, t, n_out)[0]) / (2 * eps))
    return np.array(out)
