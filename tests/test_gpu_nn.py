"""Surrogate kernels against the FP32 CPU reference: tensor-core 3x3
convolution (forward, input gradient, weight gradient), pooling and
upsampling forward/backward, ReLU mask, Adam.  Inputs are BF16; the
reference sums their exact values in FP64, so the tolerance covers the FP32
accumulation order and the BF16 rounding of the output only."""
import ctypes as C

import numpy as np
import pytest

from oracle import surrogate_ref as R

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    from paper_2212_07848_gb300 import abi
    L = abi.load()
    P = C.c_void_p
    L.lb_nn_conv3x3.argtypes = [P, P, P, P] + [C.c_int] * 7 + [P]
    L.lb_nn_conv3x3_wgrad.argtypes = [P, P, P, P] + [C.c_int] * 5 + [P, C.c_size_t, P]
    L.lb_nn_wgrad_workspace.argtypes = [C.c_int] * 5
    L.lb_nn_wgrad_workspace.restype = C.c_size_t
    L.lb_nn_pool2.argtypes = [P, P] + [C.c_int] * 5 + [P]
    L.lb_nn_up2.argtypes = [P, P] + [C.c_int] * 5 + [P]
    L.lb_nn_relu_mask.argtypes = [P, P, P, C.c_size_t, P]
    L.lb_nn_adam.argtypes = [P, P, P, P, P, C.c_size_t, C.c_double, C.c_double, C.c_double,
                             C.c_double, C.c_longlong, P]
    return L


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _bf(shape, scale=1.0, seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    return (scale * torch.randn(shape, generator=g)).to(torch.bfloat16).cuda()


def _np(t):
    return t.float().cpu().numpy()


def _close(got, ref, tol):
    scale = np.sqrt(np.mean(ref ** 2)) + 1e-30
    err = np.abs(got - ref).max() / scale
    assert err < tol, err


def _close_bf16(got, ref, tol=2e-3):
    """BF16 outputs: rounding to nearest costs up to 2^-8 of each value, plus a
    small FP32 accumulation error relative to the field's RMS."""
    scale = np.sqrt(np.mean(ref ** 2)) + 1e-30
    excess = np.abs(got - ref) - 2.0 ** -8 * np.abs(ref)
    assert excess.max() < tol * scale, excess.max() / scale


CONV = [(2, 4, 128, 16, 32), (1, 3, 256, 64, 128), (2, 2, 128, 128, 64), (1, 2, 128, 32, 16),
        (2, 16, 16, 64, 32),   # tiles span rows (h w % 128 == 0 only)
        (1, 6, 128, 32, 128),  # several 128-pixel tiles, widest tcgen05 N
        # more output rows than SMs: persistent CTAs walk runs of rows that
        # cross bands, images and (128 input channels) channel blocks
        (2, 96, 256, 128, 64), (3, 80, 128, 64, 128)]


@pytest.mark.parametrize("path", [0, 1, 2, 3])  # auto, mma.sync, tcgen05 per tile, persistent
@pytest.mark.parametrize("nb,h,w,cin,cout", CONV)
def test_conv_forward(nb, h, w, cin, cout, path):
    from paper_2212_07848_gb300 import abi
    L = _lib()
    assert L.lb_nn_set_conv_path(path) == 0
    x = _bf((nb, h, w, cin), seed=1)
    wt = _bf((9, cout, cin), 0.1, seed=2)
    b = torch.randn(cout, device="cuda")
    y = torch.empty((nb, h, w, cout), dtype=torch.bfloat16, device="cuda")
    for relu in (0, 1):
        assert L.lb_nn_conv3x3(_p(x), _p(wt), _p(b), _p(y), nb, h, w, cin, cout, relu, 0, None) == 0
        torch.cuda.synchronize()
        ref = R.conv3x3(_np(x), _np(wt), b.cpu().numpy(), bool(relu))
        _close_bf16(_np(y), ref)
    assert L.lb_nn_status() == abi.LB_OK             # no tensor-core wait gave up
    assert L.lb_nn_set_conv_path(0) == 0


@pytest.mark.parametrize("path", [0, 1])        # auto (persistent tcgen05 where it applies), mma.sync
@pytest.mark.parametrize("nb,h,w,cin,cout", CONV)
def test_conv_input_gradient(nb, h, w, cin, cout, path):
    from paper_2212_07848_gb300 import abi
    L = _lib()
    assert L.lb_nn_set_conv_path(path) == 0
    dy = _bf((nb, h, w, cout), seed=3)
    wt = _bf((9, cout, cin), 0.1, seed=4)
    dx = torch.empty((nb, h, w, cin), dtype=torch.bfloat16, device="cuda")
    assert L.lb_nn_conv3x3(_p(dy), _p(wt), None, _p(dx), nb, h, w, cout, cin, 0, 1, None) == 0
    torch.cuda.synchronize()
    _close_bf16(_np(dx), R.conv3x3_dgrad(_np(dy), _np(wt)))
    assert L.lb_nn_status() == abi.LB_OK
    assert L.lb_nn_set_conv_path(0) == 0


# the surrogate's layers at their training sizes (batch 2 instead of 8)
WGRAD_EXTRA = [(2, 64, 512, 16, 32), (2, 32, 256, 32, 64), (2, 16, 128, 64, 128),
               (2, 32, 256, 128, 64), (2, 64, 512, 64, 16), (1, 4, 128, 128, 128),
               (1, 3, 128, 16, 16), (1, 5, 256, 128, 16), (1, 4, 128, 64, 32)]


@pytest.mark.parametrize("path", [0, 1])   # tcgen05 where it applies (w % 128 == 0), mma.sync
@pytest.mark.parametrize("nb,h,w,cin,cout", CONV + WGRAD_EXTRA)
def test_conv_weight_gradient(nb, h, w, cin, cout, path):
    from paper_2212_07848_gb300 import abi
    L = _lib()
    assert L.lb_nn_set_conv_path(path) == 0
    x = _bf((nb, h, w, cin), seed=5)
    dy = _bf((nb, h, w, cout), seed=6)
    dw = torch.zeros((9, cout, cin), device="cuda")
    db = torch.zeros(cout, device="cuda")
    nbytes = L.lb_nn_wgrad_workspace(nb, h, w, cin, cout)
    assert nbytes > 0
    ws = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    assert L.lb_nn_conv3x3_wgrad(_p(x), _p(dy), _p(dw), _p(db), nb, h, w, cin, cout, _p(ws),
                                 nbytes - 4, None) == -1          # short workspace
    for _ in range(2):                       # accumulates
        assert L.lb_nn_conv3x3_wgrad(_p(x), _p(dy), _p(dw), _p(db), nb, h, w, cin, cout, _p(ws),
                                     nbytes, None) == 0
    torch.cuda.synchronize()
    first = dw.clone()
    _close(dw.cpu().numpy(), 2 * R.conv3x3_wgrad(_np(x), _np(dy)), 1e-3)
    _close(db.cpu().numpy(), 2 * _np(dy).sum(axis=(0, 1, 2)), 1e-3)
    # deterministic: the same inputs give the same bits (weights and biases)
    first_b = db.clone()
    dw.zero_()
    db.zero_()
    for _ in range(2):
        assert L.lb_nn_conv3x3_wgrad(_p(x), _p(dy), _p(dw), _p(db), nb, h, w, cin, cout, _p(ws),
                                     nbytes, None) == 0
    torch.cuda.synchronize()
    assert torch.equal(dw, first)
    assert torch.equal(db, first_b)
    assert L.lb_nn_status() == abi.LB_OK
    assert L.lb_nn_set_conv_path(0) == 0


def test_pool_up_relu_adam():
    L = _lib()
    x = _bf((2, 8, 16, 16), seed=7)
    y = torch.empty((2, 4, 8, 16), dtype=torch.bfloat16, device="cuda")
    assert L.lb_nn_pool2(_p(x), _p(y), 2, 8, 16, 16, 0, None) == 0
    dx = torch.empty_like(x)
    assert L.lb_nn_pool2(_p(y), _p(dx), 2, 8, 16, 16, 1, None) == 0
    u = torch.empty_like(x)
    assert L.lb_nn_up2(_p(y), _p(u), 2, 4, 8, 16, 0, None) == 0
    du = torch.empty_like(y)
    assert L.lb_nn_up2(_p(x), _p(du), 2, 4, 8, 16, 1, None) == 0
    torch.cuda.synchronize()
    _close(_np(y), R.pool2(_np(x)), 1e-2)
    _close(_np(dx), 0.25 * R.up2(_np(y)), 1e-2)
    _close(_np(u), R.up2(_np(y)), 1e-2)
    _close(_np(du), 4 * R.pool2(_np(x)), 1e-2)
    a = _bf((1000,), seed=8)
    m = torch.empty_like(a)
    assert L.lb_nn_relu_mask(_p(a), _p(a), _p(m), 1000, None) == 0
    torch.cuda.synchronize()
    assert np.array_equal(_np(m), np.where(_np(a) > 0, _np(a), 0.0))
    n = 513
    gen = torch.Generator(device="cpu").manual_seed(10)
    w = torch.randn(n, generator=gen).cuda()
    g = torch.randn(n, generator=gen).cuda()
    mo = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    w0 = w.cpu().numpy().copy()
    assert L.lb_nn_adam(_p(w), _p(g), _p(mo), _p(v), _p(wb), n, 1e-3, 0.9, 0.999, 1e-8, 1, None) == 0
    torch.cuda.synchronize()
    gg = g.cpu().numpy()
    mm, vv = 0.1 * gg, 0.001 * gg * gg
    ref = w0 - 1e-3 * (mm / 0.1) / (np.sqrt(vv / 0.001) + 1e-8)
    assert np.abs(w.cpu().numpy() - ref).max() < 1e-6
    # the BF16 copy rounds to nearest: within half an ulp, at most 2^-8 relative
    assert np.all(np.abs(_np(wb) - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6)


def test_coarse_expand_mse_residual():
    from paper_2212_07848_gb300 import abi
    L = abi.load()
    nx, ny, f = 96, 64, 4
    df = torch.randn((9, ny, nx), device="cuda") * 0.01
    out = torch.empty((ny // f, nx // f), device="cuda")
    assert L.lb_nn_coarse_grain(_p(df), nx, ny, f, 0.5, _p(out), None) == 0
    assert L.lb_nn_coarse_grain(_p(df), nx, ny, 5, 0.5, _p(out), None) == abi.LB_ERR_ARG
    d = df.cpu().double().numpy().sum(axis=0)
    ref = d.reshape(ny // f, f, nx // f, f).mean(axis=(1, 3)) / 0.5
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-6
    n = out.numel()
    x = torch.empty((n, 16), dtype=torch.bfloat16, device="cuda")
    prev = out * 0.5
    assert L.lb_nn_expand(_p(out), _p(prev), 0.75, _p(x), 16, n, None) == 0
    torch.cuda.synchronize()
    xe = _np(x)
    assert np.array_equal(xe[:, 0], out.to(torch.bfloat16).float().cpu().numpy().ravel())
    assert np.array_equal(xe[:, 2], (out - prev).to(torch.bfloat16).float().cpu().numpy().ravel())
    assert np.all(xe[:, 1] == 0.75) and np.all(xe[:, 3:] == 0)
    assert L.lb_nn_expand(_p(out), None, 0.75, _p(x), 16, n, None) == 0
    torch.cuda.synchronize()
    assert np.all(_np(x)[:, 2:] == 0)
    y = _bf((n, 16), 0.1, seed=9)
    base = out.flatten().clone()
    tgt = base + 0.05 * torch.randn(n, device="cuda")
    loss = torch.zeros(1, device="cuda")
    dy = torch.empty_like(y)
    assert L.lb_nn_mse(_p(y), 16, _p(tgt), _p(base), n, _p(loss), _p(dy), None) == 0
    torch.cuda.synchronize()
    e = base.cpu().double().numpy() + _np(y)[:, 0] - tgt.cpu().double().numpy()
    assert abs(float(loss.item()) - np.mean(e * e)) < 1e-5 * np.mean(e * e)
    ge = _np(dy)
    assert np.abs(ge[:, 0] - 2 * e / n).max() < 1e-2 * np.abs(2 * e / n).max()
    assert np.all(ge[:, 1:] == 0)
    state = base.clone()
    assert L.lb_nn_residual(_p(state), _p(y), 16, _p(x), 16, n, None, None) == 0
    torch.cuda.synchronize()
    sref = base.cpu().numpy() + _np(y)[:, 0]
    assert np.abs(state.cpu().numpy() - sref).max() < 1e-6
    xr = _np(x)
    assert np.array_equal(xr[:, 0], state.to(torch.bfloat16).float().cpu().numpy())
    assert np.all(xr[:, 1] == 0.75)
    assert np.array_equal(xr[:, 2], _np(y)[:, 0])          # the increment just applied
    # zero-mean increments: the mass of the state is conserved
    mean = torch.zeros(513, device="cuda")
    state2 = base.clone()
    assert L.lb_nn_residual(_p(state2), _p(y), 16, _p(x), 16, n, _p(mean), None) == 0
    torch.cuda.synchronize()
    mu = _np(y)[:, 0].astype(np.float64).mean()
    assert abs(float(mean[0].item()) - mu) < 1e-6 * max(1.0, abs(mu)) + 1e-7
    assert abs(float(state2.double().sum() - base.double().sum())) < 1e-4
    assert np.abs(state2.cpu().numpy() - (base.cpu().numpy() + _np(y)[:, 0] - mu)).max() < 1e-6


def test_flux_divergence_forward_and_adjoint():
    """lb_nn_flux_div against the CPU reference on a ragged 3 x 40 x 24 x 16
    batch: forward to the BF16 rounding of its output, backward likewise,
    channels beyond the flux exactly 0."""
    from paper_2212_07848_gb300 import abi
    L = abi.load()
    nb, h, w, c = 3, 40, 24, 16
    y = _bf((nb, h, w, c), seed=51)
    inc = torch.empty((nb, h, w), dtype=torch.bfloat16, device="cuda")
    assert L.lb_nn_flux_div(_p(y), _p(inc), c, nb, h, w, 0, None) == 0
    d = _bf((nb, h, w), seed=52)
    dy = torch.full((nb, h, w, c), 7.0, dtype=torch.bfloat16, device="cuda")
    assert L.lb_nn_flux_div(_p(d), _p(dy), c, nb, h, w, 1, None) == 0
    assert L.lb_nn_flux_div(_p(y), _p(inc), 1, nb, h, w, 0, None) == -1
    torch.cuda.synchronize()
    _close_bf16(_np(inc), R.flux_div(_np(y)))
    ref = R.flux_div_backward(_np(d), c)
    _close_bf16(_np(dy)[..., :2], ref[..., :2])
    assert not _np(dy)[..., 2:].any()


def test_momentum_state_kernels():
    """lb_nn_coarse_momentum against block means of sum_i c_i df_i, and the
    channel forms of expand, MSE and the residual update (through a
    channel-offset pointer) that carry the momentum state."""
    from paper_2212_07848_gb300 import abi
    L = abi.load()
    nx, ny, f = 96, 64, 4
    df = torch.randn((9, ny, nx), device="cuda") * 0.01
    jx = torch.empty((ny // f, nx // f), device="cuda")
    jy = torch.empty_like(jx)
    assert L.lb_nn_coarse_momentum(_p(df), nx, ny, f, 0.25, _p(jx), _p(jy), None) == 0
    assert L.lb_nn_coarse_momentum(_p(df), nx, ny, 5, 0.25, _p(jx), _p(jy), None) == abi.LB_ERR_ARG
    c = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)])
    d = df.cpu().double().numpy()
    for a, got in ((0, jx), (1, jy)):
        j = np.tensordot(c[:, a].astype(float), d, axes=1)
        ref = j.reshape(ny // f, f, nx // f, f).mean(axis=(1, 3)) / 0.25
        torch.cuda.synchronize()
        assert np.abs(got.cpu().numpy() - ref).max() < 1e-5 * np.abs(ref).max()
    n = jx.numel()
    x = torch.zeros((n, 16), dtype=torch.bfloat16, device="cuda")
    prev = jx * 0.5
    assert L.lb_nn_expand_channel(_p(jx), _p(prev), _p(x), 16, 3, n, None) == 0
    assert L.lb_nn_expand_channel(_p(jy), None, _p(x), 16, 4, n, None) == 0
    assert L.lb_nn_expand_channel(_p(jy), _p(prev), _p(x), 16, 14, n, None) == abi.LB_ERR_ARG
    torch.cuda.synchronize()
    xe = _np(x)
    assert np.array_equal(xe[:, 3], jx.to(torch.bfloat16).float().cpu().numpy().ravel())
    assert np.array_equal(xe[:, 5], (jx - prev).to(torch.bfloat16).float().cpu().numpy().ravel())
    assert np.array_equal(xe[:, 4], jy.to(torch.bfloat16).float().cpu().numpy().ravel())
    assert np.all(xe[:, [0, 1, 2, 6]] == 0) and np.all(xe[:, 7:] == 0)
    y = _bf((n, 16), 0.1, seed=19)
    base = jx.flatten().clone()
    tgt = base + 0.05 * torch.randn(n, device="cuda")
    loss = torch.zeros(1, device="cuda")
    dy = torch.full((n, 16), 3.0, dtype=torch.bfloat16, device="cuda")
    assert L.lb_nn_mse_channel(_p(y), 16, 2, _p(tgt), _p(base), n, 0.5, _p(loss), _p(dy),
                               None) == 0
    torch.cuda.synchronize()
    e = base.cpu().double().numpy() + _np(y)[:, 2] - tgt.cpu().double().numpy()
    assert abs(float(loss.item()) - 0.5 * np.mean(e * e)) < 1e-5 * np.mean(e * e)
    ge = _np(dy)
    assert np.abs(ge[:, 2] - e / n).max() < 1e-2 * np.abs(e / n).max()
    assert np.all(ge[:, [0, 1]] == 3.0) and np.all(ge[:, 3:] == 3.0)     # untouched
    # residual on channel 2 of y into channel 3 of x (increment lands in 5)
    state = base.clone()
    yc = C.c_void_p(y.data_ptr() + 2 * 2)
    xc = C.c_void_p(x.data_ptr() + 2 * 3)
    assert L.lb_nn_residual(_p(state), yc, 16, xc, 16, n, None, None) == 0
    torch.cuda.synchronize()
    sref = base.cpu().numpy() + _np(y)[:, 2]
    assert np.abs(state.cpu().numpy() - sref).max() < 1e-6
    xr = _np(x)
    assert np.array_equal(xr[:, 3], state.to(torch.bfloat16).float().cpu().numpy())
    assert np.array_equal(xr[:, 5], _np(y)[:, 2])
    assert np.array_equal(xr[:, 4], xe[:, 4])


def test_block_mse():
    """lb_nn_mse_blocks against numpy: the loss from 8 x 8 tile means of the
    residual on a 2 x 32 x 48 batch, and its gradient added to dy."""
    from paper_2212_07848_gb300 import abi
    L = abi.load()
    nb, h, w, c, B = 2, 32, 48, 16, 8
    n = nb * h * w
    y = _bf((n, c), 0.1, seed=61)
    base = torch.randn(n, device="cuda") * 0.1
    tgt = torch.randn(n, device="cuda") * 0.1
    loss = torch.zeros(1, device="cuda")
    dy = torch.full((n, c), 0.5, dtype=torch.bfloat16, device="cuda")
    dy[:, 0] = 0.0
    assert L.lb_nn_mse_blocks(_p(y), c, _p(tgt), _p(base), nb, h, w, B, 3.0, _p(loss), _p(dy),
                              None) == 0
    assert L.lb_nn_mse_blocks(_p(y), c, _p(tgt), _p(base), nb, h, w, 7, 3.0, _p(loss), _p(dy),
                              None) == abi.LB_ERR_ARG
    torch.cuda.synchronize()
    d = (base.cpu().double().numpy() + _np(y)[:, 0] - tgt.cpu().double().numpy())
    tiles = d.reshape(nb, h // B, B, w // B, B).mean(axis=(2, 4))
    ref_loss = 3.0 * np.mean(tiles ** 2)
    assert abs(float(loss.item()) - ref_loss) < 1e-4 * ref_loss
    g = 2 * 3.0 * tiles / tiles.size / (B * B)
    gref = np.repeat(np.repeat(g, B, axis=1), B, axis=2).reshape(-1)
    got = _np(dy)
    assert np.abs(got[:, 0] - gref).max() <= 1e-2 * np.abs(gref).max()
    assert np.all(got[:, 1:] == 0.5)
