"""CPU reference of the surrogate network (numpy, FP64 sums), for checking the
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


def pool2_backward(dy):
    return 0.25 * up2(dy)


def up2_backward(dy):
    return 4.0 * pool2(dy)


def net_forward(x, w, b):
    """The surrogate network on x [nb][n][n][16]: returns (y, activations)
    with w[i] [9][cout][cin], b[i] [cout] for the five layers
    16->32 (n), 32->64 (n/2), 64->128 (n/4), 128->64 (n/2), 64->16 (n);
    pooling after layers 1 and 2, upsampling before layers 4 and 5, and the
    skip a4 + a2 before the last upsampling."""
    a1 = conv3x3(x, w[0], b[0], True)
    p1 = pool2(a1)
    a2 = conv3x3(p1, w[1], b[1], True)
    p2 = pool2(a2)
    a3 = conv3x3(p2, w[2], b[2], True)
    u3 = up2(a3)
    a4 = conv3x3(u3, w[3], b[3], True)
    s4 = a4 + a2
    u4 = up2(s4)
    y = conv3x3(u4, w[4], b[4], False)
    return y, dict(a1=a1, p1=p1, a2=a2, p2=p2, a3=a3, u3=u3, a4=a4, u4=u4)


def flux_div(y):
    """Increment as minus the divergence of the flux J = (y[..., 0], y[..., 1])
    with backward differences on the periodic grid: -(dJx/dx + dJy/dy)."""
    jx, jy = y[..., 0].astype(np.float64), y[..., 1].astype(np.float64)
    return -((jx - shift(jx[..., None], 0, -1)[..., 0]) + (jy - shift(jy[..., None], -1, 0)[..., 0]))


def flux_div_backward(dinc, c):
    """Adjoint of flux_div: the gradient with respect to y [..][c] (channels 0
    and 1; the others 0) of sum(dinc * flux_div(y))."""
    d = dinc[..., None].astype(np.float64)
    dy = np.zeros(dinc.shape + (c,))
    dy[..., 0] = -(d - shift(d, 0, 1))[..., 0]
    dy[..., 1] = -(d - shift(d, 1, 0))[..., 0]
    return dy


def net_loss(y, base, target, flux=False, jweight=None):
    """Residual MSE: mean over pixels of (base + inc - target)^2 with the
    increment inc = y[..., 0], or flux_div(y) with `flux`.  With `jweight`
    (the momentum state) base and target are [3][..] (density, jx, jy) and
    jweight times the MSE of base[a] + y[..., a + 1] - target[a], a = 1, 2, is
    added.  Returns (loss, residuals)."""
    b0, t0 = (base[0], target[0]) if jweight is not None else (base, target)
    inc = flux_div(y) if flux else y[..., 0]
    if jweight is None:
        d = b0 + inc - t0
        return float(np.mean(d * d)), d
    d = np.stack([b0 + inc - t0] + [base[a] + y[..., a + 1] - target[a] for a in (1, 2)])
    return float(np.mean(d[0] ** 2) + jweight * (np.mean(d[1] ** 2) + np.mean(d[2] ** 2))), d


def net_backward(x, w, acts, d, flux=False, jweight=None, want_dx=False):
    """Parameter gradients of net_loss by reverse-mode differentiation of
    net_forward (chain rule layer by layer).  Returns (dw list, db list), and
    with want_dx also the gradient with respect to the input x."""
    d0 = d[0] if jweight is not None else d
    if flux:
        dy = flux_div_backward(2.0 * d0 / d0.size, w[4].shape[1])
    else:
        dy = np.zeros(d0.shape + (w[4].shape[1],))
        dy[..., 0] = 2.0 * d0 / d0.size
    if jweight is not None:
        for a in (1, 2):
            dy[..., a + 1] += 2.0 * jweight * d[a] / d[a].size
    return backward_from_dy(x, w, acts, dy, want_dx)


def backward_from_dy(x, w, acts, dy, want_dx=False):
    """Parameter gradients (and optionally the input gradient) of the network
    for a given output gradient dy."""
    dw, db = [None] * 5, [None] * 5
    ins = [x, acts["p1"], acts["p2"], acts["u3"], acts["u4"]]

    def layer(i, dz):
        dw[i] = conv3x3_wgrad(ins[i], dz)
        db[i] = dz.sum(axis=(0, 1, 2))

    layer(4, dy)
    ds4 = up2_backward(conv3x3_dgrad(dy, w[4]))
    dz4 = ds4 * (acts["a4"] > 0)
    layer(3, dz4)
    da3 = up2_backward(conv3x3_dgrad(dz4, w[3]))
    dz3 = da3 * (acts["a3"] > 0)
    layer(2, dz3)
    da2 = pool2_backward(conv3x3_dgrad(dz3, w[2])) + ds4
    dz2 = da2 * (acts["a2"] > 0)
    layer(1, dz2)
    da1 = pool2_backward(conv3x3_dgrad(dz2, w[1]))
    dz1 = da1 * (acts["a1"] > 0)
    layer(0, dz1)
    if want_dx:
        return dw, db, conv3x3_dgrad(dz1, w[0])
    return dw, db


def two_stride_loss(x0, w, b, base0, t1, t2):
    """The loss of two surrogate strides in a row (plain increments): the
    first prediction s1 = base0 + y0[..., 0] becomes the next input (channel
    0 the field, channel 2 its increment, the other channels as in x0), and
    L = mean((s1 - t1)^2) + mean((s1 + y1[..., 0] - t2)^2).  Returns
    (L, intermediates for two_stride_backward)."""
    y0, a0 = net_forward(x0, w, b)
    inc0 = y0[..., 0]
    s1 = base0 + inc0
    x1 = np.array(x0, dtype=np.float64)
    x1[..., 0] = s1
    x1[..., 2] = inc0
    y1, a1 = net_forward(x1, w, b)
    p2 = s1 + y1[..., 0]
    L = float(np.mean((s1 - t1) ** 2) + np.mean((p2 - t2) ** 2))
    return L, dict(a0=a0, a1=a1, x1=x1, s1=s1, p2=p2)


def two_stride_backward(x0, w, b, t1, t2, mid):
    """Parameter gradients of two_stride_loss: the second stride's output
    gradient, then through its input (channels 0 and 2) and its base (s1) into
    the first stride's increment."""
    s1, p2 = mid["s1"], mid["p2"]
    n = s1.size
    d2 = 2.0 * (p2 - t2) / n
    dy1 = np.zeros(s1.shape + (w[4].shape[1],))
    dy1[..., 0] = d2
    dw1, db1, dx1 = backward_from_dy(mid["x1"], w, mid["a1"], dy1, want_dx=True)
    dinc0 = 2.0 * (s1 - t1) / n + d2 + dx1[..., 0] + dx1[..., 2]
    dy0 = np.zeros(s1.shape + (w[4].shape[1],))
    dy0[..., 0] = dinc0
    dw0, db0 = backward_from_dy(x0, w, mid["a0"], dy0)
    return [a + c for a, c in zip(dw0, dw1)], [a + c for a, c in zip(db0, db1)]
