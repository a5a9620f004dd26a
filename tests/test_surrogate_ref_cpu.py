"""Pins of the CPU reference of the surrogate network: the convolution
against an explicit loop over pixels and taps, its input and weight
gradients as the adjoints of the forward map, pooling and upsampling as
mutual adjoints, and the whole-network backward pass against central finite
differences of the loss."""
import numpy as np
import pytest

from oracle import surrogate_ref as R


def _rand(shape, seed, scale=1.0):
    return scale * np.random.default_rng(seed).standard_normal(shape)


def test_conv_matches_explicit_loop():
    x = _rand((1, 4, 6, 3), 1)
    w = _rand((9, 2, 3), 2)
    b = _rand(2, 3)
    y = R.conv3x3(x, w, b)
    h, wd = 4, 6
    for yy in range(h):
        for xx in range(wd):
            for n in range(2):
                s = b[n]
                for t in range(9):
                    dy, dx = t // 3 - 1, t % 3 - 1          # tap = 3 (dy + 1) + (dx + 1)
                    s += np.dot(x[0, (yy + dy) % h, (xx + dx) % wd], w[t, n])
                assert abs(y[0, yy, xx, n] - s) < 1e-12


def test_gradients_are_adjoints():
    x = _rand((2, 4, 4, 3), 4)
    w = _rand((9, 5, 3), 5)
    dy = _rand((2, 4, 4, 5), 6)
    lhs = np.sum(R.conv3x3(x, w) * dy)
    assert abs(lhs - np.sum(x * R.conv3x3_dgrad(dy, w))) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(w * R.conv3x3_wgrad(x, dy))) < 1e-10 * abs(lhs)
    a = _rand((1, 4, 6, 2), 7)
    c = _rand((1, 2, 3, 2), 8)
    assert abs(np.sum(R.pool2(a) * c) - np.sum(a * R.pool2_backward(c))) < 1e-12
    assert abs(np.sum(R.up2(c) * a) - np.sum(c * R.up2_backward(a))) < 1e-12


def _net(seed, n=8):
    chans = [(16, 32), (32, 64), (64, 128), (128, 64), (64, 16)]
    w = [_rand((9, co, ci), seed + i, np.sqrt(2.0 / (9 * ci))) for i, (ci, co) in enumerate(chans)]
    b = [_rand(co, seed + 10 + i, 0.1) for i, (ci, co) in enumerate(chans)]
    x = _rand((1, n, n, 16), seed + 20)
    base = _rand((1, n, n), seed + 21)
    tgt = _rand((1, n, n), seed + 22)
    return x, w, b, base, tgt


@pytest.mark.parametrize("flux,jw", [(False, None), (True, None), (True, 0.7)])
def test_network_backward_matches_finite_differences(flux, jw):
    x, w, b, base, tgt = _net(30)
    if jw is not None:                       # density, jx, jy state
        base = np.stack([base, _rand(base.shape, 23), _rand(base.shape, 24)])
        tgt = np.stack([tgt, _rand(tgt.shape, 25), _rand(tgt.shape, 26)])
    y, acts = R.net_forward(x, w, b)
    _, d = R.net_loss(y, base, tgt, flux, jw)
    dw, db = R.net_backward(x, w, acts, d, flux, jw)
    rng = np.random.default_rng(0)
    h = 1e-5
    for i in range(5):
        for _ in range(4):
            idx = tuple(int(rng.integers(s)) for s in w[i].shape)
            old = w[i][idx]
            w[i][idx] = old + h
            lp, _ = R.net_loss(R.net_forward(x, w, b)[0], base, tgt, flux, jw)
            w[i][idx] = old - h
            lm, _ = R.net_loss(R.net_forward(x, w, b)[0], base, tgt, flux, jw)
            w[i][idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - dw[i][idx]) <= 1e-4 * abs(fd) + 1e-9, (i, idx, fd, dw[i][idx])
        j = int(rng.integers(b[i].size))
        old = b[i][j]
        b[i][j] = old + h
        lp, _ = R.net_loss(R.net_forward(x, w, b)[0], base, tgt, flux, jw)
        b[i][j] = old - h
        lm, _ = R.net_loss(R.net_forward(x, w, b)[0], base, tgt, flux, jw)
        b[i][j] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - db[i][j]) <= 1e-4 * abs(fd) + 1e-9, (i, j, fd, db[i][j])


def test_flux_divergence_definition_conservation_and_adjoint():
    """flux_div against its definition written as loops on a 3 x 5 grid, the
    telescoping sum (every increment has zero mean per image), zero increment
    for a uniform flux, and the adjoint identity of its backward."""
    y = _rand((2, 3, 5, 4), 41)
    inc = R.flux_div(y)
    H, W = 3, 5
    for b in range(2):
        for i in range(H):
            for j in range(W):
                ref = -((y[b, i, j, 0] - y[b, i, (j - 1) % W, 0]) +
                        (y[b, i, j, 1] - y[b, (i - 1) % H, j, 1]))
                assert abs(inc[b, i, j] - ref) < 1e-14
    assert np.abs(inc.sum(axis=(1, 2))).max() < 1e-13
    u = np.zeros((1, 3, 5, 4))
    u[..., 0], u[..., 1] = 0.7, -1.3
    assert np.abs(R.flux_div(u)).max() == 0.0
    d = _rand((2, 3, 5), 42)
    lhs = np.sum(inc * d)
    rhs = np.sum(y * R.flux_div_backward(d, 4))
    assert abs(lhs - rhs) < 1e-12


def test_input_gradient_and_two_stride_backward_match_finite_differences():
    """The network's input gradient, and the gradient of the two-stride loss
    (the first prediction fed back as the next input), against central
    finite differences."""
    x, w, b, base, tgt = _net(50)
    t2 = _rand(tgt.shape, 53)
    y, acts = R.net_forward(x, w, b)
    _, d = R.net_loss(y, base, tgt)
    _, _, dx = R.net_backward(x, w, acts, d, want_dx=True)
    rng = np.random.default_rng(3)
    h = 1e-5
    for _ in range(6):
        idx = tuple(int(rng.integers(s)) for s in x.shape)
        old = x[idx]
        x[idx] = old + h
        lp, _ = R.net_loss(R.net_forward(x, w, b)[0], base, tgt)
        x[idx] = old - h
        lm, _ = R.net_loss(R.net_forward(x, w, b)[0], base, tgt)
        x[idx] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - dx[idx]) <= 1e-4 * abs(fd) + 1e-9, (idx, fd, dx[idx])
    L, mid = R.two_stride_loss(x, w, b, base, tgt, t2)
    dw, db = R.two_stride_backward(x, w, b, tgt, t2, mid)
    for i in range(5):
        for _ in range(3):
            idx = tuple(int(rng.integers(s)) for s in w[i].shape)
            old = w[i][idx]
            w[i][idx] = old + h
            lp, _ = R.two_stride_loss(x, w, b, base, tgt, t2)
            w[i][idx] = old - h
            lm, _ = R.two_stride_loss(x, w, b, base, tgt, t2)
            w[i][idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - dw[i][idx]) <= 1e-4 * abs(fd) + 1e-9, (i, idx, fd, dw[i][idx])
        j = int(rng.integers(b[i].size))
        old = b[i][j]
        b[i][j] = old + h
        lp, _ = R.two_stride_loss(x, w, b, base, tgt, t2)
        b[i][j] = old - h
        lm, _ = R.two_stride_loss(x, w, b, base, tgt, t2)
        b[i][j] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - db[i][j]) <= 1e-4 * abs(fd) + 1e-9, (i, j, fd, db[i][j])
