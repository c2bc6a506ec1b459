"""Plain numpy reference of the surrogate network (test infrastructure).

The MLP 4 -> 128 -> 128 -> 1 with SiLU, parameters in the flat FP32 layout
of the library (W1 [128][16] with input columns 4..15 zero, b1 [128],
W2 [128 out][128 in], b2 [128], w3 [128], b3).  The tensor-core operands
are bf16: the network input X, the weights W1 and W2, the activations H1,
and in the backward pass dZ2 and dZ1; everything else is exact (float64
here).  forward() and grads() restate the textbook forward pass and its
reverse-mode derivative of the batch-mean squared error with those
roundings applied at those points.
"""
import numpy as np

from . import quant

P_W1, P_b1 = 0, 128 * 16
P_W2 = P_b1 + 128
P_b2 = P_W2 + 128 * 128
P_w3 = P_b2 + 128
P_b3 = P_w3 + 128
P_N = P_b3 + 1


def bf16(a):
    """Round to bfloat16 (through float32, round to nearest even)."""
    a32 = np.asarray(a, np.float32)
    return quant.bf16_value(quant.bf16_bits(a32)).astype(np.float64)


def unpack(p):
    p = np.asarray(p, np.float64)
    W1 = p[P_W1:P_b1].reshape(128, 16)[:, :4]
    return (W1, p[P_b1:P_W2], p[P_W2:P_b2].reshape(128, 128), p[P_b2:P_w3], p[P_w3:P_b3], p[P_b3])


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _rnd(rounding):
    return bf16 if rounding else (lambda a: np.asarray(a, np.float64))


def forward(p, x, rounding=True):
    """Network output (standardised units) at normalised points x [n][4]."""
    bf16 = _rnd(rounding)
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = bf16(x)
    z1 = X @ bf16(W1).T + b1
    h1 = bf16(silu(z1))
    z2 = h1 @ bf16(W2).T + b2
    return silu(z2) @ w3 + b3


def grads(p, x, y, rounding=True):
    """(flat gradient [P_N], loss) of mean((f(x) - y)^2)."""
    bf16 = _rnd(rounding)
    W1, b1, W2, b2, w3, b3 = unpack(p)
    n = x.shape[0]
    X = bf16(x)
    z1 = X @ bf16(W1).T + b1
    h1 = bf16(silu(z1))
    z2 = h1 @ bf16(W2).T + b2
    h2 = silu(z2)
    r = h2 @ w3 + b3 - y
    dy = 2.0 * r / n
    dz2 = (dy[:, None] * w3[None, :]) * dsilu(z2)
    dz2b = bf16(dz2)
    dW2 = dz2b.T @ h1
    dh1 = dz2b @ bf16(W2)
    dz1 = dh1 * dsilu(z1)
    dW1 = bf16(dz1).T @ X
    g = np.zeros(P_N)
    g[P_W1:P_b1] = np.pad(dW1, ((0, 0), (0, 12))).reshape(-1)
    g[P_b1:P_W2] = dz1.sum(0)
    g[P_W2:P_b2] = dW2.reshape(-1)
    g[P_b2:P_w3] = dz2.sum(0)
    g[P_w3:P_b3] = (dy[:, None] * h2).sum(0)
    g[P_b3] = dy.sum()
    return g, float(np.mean(r * r))
