"""Plain numpy reference of the surrogate network (test infrastructure).

The MLP 4 -> 128 -> 128 -> 1 with SiLU, parameters in the flat FP32 layout
of the library (W1 [128][16]: columns 0..3 weigh the four coordinates,
column 4 the side of the K2 switch, columns 5..15 zero; b1 [128], W2 [128
out][128 in], b2 [128], w3 [128], b3).

Network input: each normalised coordinate x_d enters as hi = bf16(x_d)
and lo = bf16(x_d - hi), both weighted by W1[:, d]; the switch side s = +1
where x_T > xs (xs the normalised log2 of the K2 switch temperature), -1
otherwise, weighted by W1[:, 4].  The tensor-core operands are bf16: the
input parts, the weights W1 and W2, the activations H1, and in the
backward pass dZ2 and dZ1; everything else is exact (float64 here).
forward() and grads() restate the textbook forward pass and its
reverse-mode derivative of the batch-mean squared error with those
roundings applied at those points.  With rounding off, hi = x and lo = 0.
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
    W1 = p[P_W1:P_b1].reshape(128, 16)[:, :5]
    return (W1, p[P_b1:P_W2], p[P_W2:P_b2].reshape(128, 128), p[P_b2:P_w3], p[P_w3:P_b3], p[P_b3])


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _rnd(rounding):
    return bf16 if rounding else (lambda a: np.asarray(a, np.float64))


def features(x, xs, rounding=True):
    """Input parts [n][9]: hi (4), lo (4), switch side."""
    rnd = _rnd(rounding)
    x = np.asarray(x, np.float64)
    if rounding:
        x = x.astype(np.float32).astype(np.float64)
    hi = rnd(x)
    lo = rnd(x - hi)
    side = np.where(x[:, 3] > np.float64(np.float32(xs)), 1.0, -1.0)
    return np.concatenate([hi, lo, side[:, None]], axis=1)


def first_layer(W1, rounding=True):
    """Operand weights [128][9] for the parts of features()."""
    W = _rnd(rounding)(W1)
    return np.concatenate([W[:, :4], W[:, :4], W[:, 4:5]], axis=1)


def forward(p, x, xs, rounding=True):
    """Network output (standardised units) at normalised points x [n][4]."""
    rnd = _rnd(rounding)
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = features(x, xs, rounding)
    z1 = X @ first_layer(W1, rounding).T + b1
    h1 = rnd(silu(z1))
    z2 = h1 @ rnd(W2).T + b2
    return silu(z2) @ w3 + b3


def grads(p, x, y, xs, rounding=True):
    """(flat gradient [P_N], loss) of mean((f(x) - y)^2)."""
    rnd = _rnd(rounding)
    W1, b1, W2, b2, w3, b3 = unpack(p)
    n = x.shape[0]
    X = features(x, xs, rounding)
    z1 = X @ first_layer(W1, rounding).T + b1
    h1 = rnd(silu(z1))
    z2 = h1 @ rnd(W2).T + b2
    h2 = silu(z2)
    r = h2 @ w3 + b3 - y
    dy = 2.0 * r / n
    dz2 = (dy[:, None] * w3[None, :]) * dsilu(z2)
    dz2b = rnd(dz2)
    dW2 = dz2b.T @ h1
    dh1 = dz2b @ rnd(W2)
    dz1 = dh1 * dsilu(z1)
    dX = rnd(dz1).T @ X                       # [128][9] over the operand columns
    dW1 = np.zeros((128, 16))
    dW1[:, :4] = dX[:, :4] + dX[:, 4:8]       # hi and lo parts share W1[:, d]
    dW1[:, 4] = dX[:, 8]
    g = np.zeros(P_N)
    g[P_W1:P_b1] = dW1.reshape(-1)
    g[P_b1:P_W2] = dz1.sum(0)
    g[P_W2:P_b2] = dW2.reshape(-1)
    g[P_b2:P_w3] = dz2.sum(0)
    g[P_w3:P_b3] = (dy[:, None] * h2).sum(0)
    g[P_b3] = dy.sum()
    return g, float(np.mean(r * r))
