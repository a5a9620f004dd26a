"""FP32 CPU reference of the surrogate's layers (numpy), for checking the
BF16 tensor-core kernels and their gradients.

TEST INFRASTRUCTURE ONLY.  Layout: NHWC [nb][h][w][c], periodic boundaries,
3x3 weights w[tap][cout][cin] with tap = 3 (dy + 1) + (dx + 1).
"""
import numpy as np

TAPS = [(t // 3 - 1, t % 3 - 1) for t in range(9)]


def shift(x, dy, dx):
    """x[p + (dy, dx)] with periodic wrap: out[:, y, x] = x[:, y + dy, x + dx]."""
    return np.roll(x, (-dy, -dx), axis=(1, 2))


def conv3x3(x, w, bias=None, relu=False):
    y = np.zeros(x.shape[:3] + (w.shape[1],), np.float64)
    for t, (dy, dx) in enumerate(TAPS):
        y += np.einsum("bhwc,nc->bhwn", shift(x, dy, dx).astype(np.float64), w[t].astype(np.float64))
    if bias is not None:
        y += bias
    if relu:
        y = np.maximum(y, 0.0)
    return y


def conv3x3_dgrad(dy, w):
    """dx[p][c] = sum_{tap, n} dy[p - off(tap)][n] w[tap][n][c]."""
    dx = np.zeros(dy.shape[:3] + (w.shape[2],), np.float64)
    for t, (ddy, ddx) in enumerate(TAPS):
        dx += np.einsum("bhwn,nc->bhwc", shift(dy, -ddy, -ddx).astype(np.float64),
                        w[t].astype(np.float64))
    return dx


def conv3x3_wgrad(x, dy):
    """dw[tap][n][c] = sum_p x[p + off(tap)][c] dy[p][n]."""
    return np.stack([np.einsum("bhwc,bhwn->nc", shift(x, ddy, ddx).astype(np.float64),
                               dy.astype(np.float64)) for ddy, ddx in TAPS])


def pool2(x):
    return 0.25 * (x[:, 0::2, 0::2] + x[:, 1::2, 0::2] + x[:, 0::2, 1::2] + x[:, 1::2, 1::2])


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)
