"""Learned surrogate: a small convolutional operator that advances the 4x
coarse-grained density of an unstable-branch quench by a fixed stride of
lattice steps, trained on trajectories of the solver (which stays its
reference and its fallback).  The paper has no such part; it serves the
long quench runs behind the paper's unstable-branch experiment.

Network (NHWC BF16 activations, FP32 master weights, periodic boundaries):
    a1 = relu(conv(x, 16 -> 32))            at N x N
    a2 = relu(conv(pool(a1), 32 -> 64))     at N/2
    a3 = relu(conv(pool(a2), 64 -> 128))    at N/4
    a4 = relu(conv(up(a3), 128 -> 64))      at N/2
    y  = conv(up(a4 + a2), 64 -> 16)        at N
    prediction = x[..., 0] + inc, inc = y[..., 0], or in the flux form
    inc = -div(y[..., 0], y[..., 1]) (the increment conserves mass locally as
    the lattice does, so rollout errors cannot pile up at long wavelengths)
Input channel 0 is the coarse density deviation rho - rho0, channel 1 the
coupling feature (G + 4.8) / 0.4, channel 2 the last density increment; with
`momentum` the coarse momentum (jx, jy) / J_SCALE is state too: input
channels 3, 4 (and its last increments 5, 6), output channels 2, 3 its
increments, so the network sees the flow that carries mass between domains.
The other channels are zero.  Every operation is a
kernel of liblbsc.so (tensor-core convolutions, elementwise pieces, Adam);
torch only provides device memory.
"""
import ctypes as C
import math
import time

import numpy as np

from . import abi

CIN = 16
LAYERS = [(16, 32), (32, 64), (64, 128), (128, 64), (64, 16)]   # (cin, cout)


J_SCALE = 0.01     # coarse momentum is stored and fed as j / J_SCALE


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _pc(t, ch):
    """Pointer to channel ch of a BF16 NHWC tensor (its first pixel)."""
    return C.c_void_p(t.data_ptr() + 2 * ch)


def _check(rc, what):
    if rc != 0:
        raise abi.LbError(rc, what)


def gfeat(G):
    return (G + 4.8) / 0.4


class SurrogateNet:
    def __init__(self, n, batch, seed=0, stream=None, flux=False, momentum=False, jweight=1.0,
                 block_loss=()):
        import torch
        self.torch = torch
        self.n, self.batch, self.flux = n, batch, flux
        self.momentum, self.jweight = momentum, jweight
        # (block, weight) pairs: the density residual averaged over block x
        # block tiles enters the loss with that weight (long-wavelength error)
        self.block_loss = tuple(block_loss)
        self.L = abi.load()
        self.s = stream
        g = torch.Generator(device="cpu").manual_seed(seed)
        self.w, self.b, self.wb, self.dw, self.db = [], [], [], [], []
        self.mw, self.vw, self.mb, self.vb = [], [], [], []
        for ci, co in LAYERS:
            std = math.sqrt(2.0 / (9 * ci))
            w = (std * torch.randn((9, co, ci), generator=g)).cuda()
            if co == 16:                       # output layer starts near zero
                w *= 0.01
            self.w.append(w)
            self.b.append(torch.zeros(co, device="cuda"))
            self.wb.append(w.to(torch.bfloat16))
            for lst, like in ((self.dw, w), (self.mw, w), (self.vw, w)):
                lst.append(torch.zeros_like(like))
            for lst in (self.db, self.mb, self.vb):
                lst.append(torch.zeros(co, device="cuda"))
        self.step_count = 0
        self._alloc(batch)

    def _alloc(self, nb):
        t, n, bf = self.torch, self.n, self.torch.bfloat16
        self._stride_graph = None   # a captured stride refers to the old buffers
        z = lambda h, c: t.empty((nb, h, h, c), dtype=bf, device="cuda")
        self.nb = nb
        self.a1, self.p1, self.a2, self.p2 = z(n, 32), z(n // 2, 32), z(n // 2, 64), z(n // 4, 64)
        self.a3, self.u3, self.a4, self.s4 = z(n // 4, 128), z(n // 2, 128), z(n // 2, 64), z(n // 2, 64)
        self.u4, self.y = z(n, 64), z(n, 16)
        self.inc, self.dinc = (z(n, 1), z(n, 1)) if self.flux else (None, None)
        # gradients
        self.dy, self.du4, self.ds4, self.dz4 = z(n, 16), z(n, 64), z(n // 2, 64), z(n // 2, 64)
        self.du3, self.da3, self.dz3, self.dp2 = z(n // 2, 128), z(n // 4, 128), z(n // 4, 128), z(n // 4, 64)
        self.da2, self.dz2, self.dp1 = z(n // 2, 64), z(n // 2, 64), z(n // 2, 32)
        self.da1, self.dz1, self.tmp2 = z(n, 32), z(n, 32), z(n // 2, 64)
        sizes = [n, n // 2, n // 4, n // 2, n]
        ws = max(self.L.lb_nn_wgrad_workspace(nb, h, h, ci, co)
                 for h, (ci, co) in zip(sizes, LAYERS))
        self.ws_bytes = ws
        self.ws = t.empty(ws // 4, dtype=t.float32, device="cuda")

    def _conv(self, x, i, out, relu, h):
        ci, co = LAYERS[i]
        _check(self.L.lb_nn_conv3x3(_p(x), _p(self.wb[i]), _p(self.b[i]), _p(out), self.nb, h, h,
                                    ci, co, relu, 0, self.s), "conv")

    def forward(self, x):
        """x: [nb][n][n][16] BF16; returns y [nb][n][n][16] (channel 0 = increment)."""
        n, L, nb = self.n, self.L, self.nb
        self._conv(x, 0, self.a1, 1, n)
        _check(L.lb_nn_pool2(_p(self.a1), _p(self.p1), nb, n, n, 32, 0, self.s), "pool")
        self._conv(self.p1, 1, self.a2, 1, n // 2)
        _check(L.lb_nn_pool2(_p(self.a2), _p(self.p2), nb, n // 2, n // 2, 64, 0, self.s), "pool")
        self._conv(self.p2, 2, self.a3, 1, n // 4)
        _check(L.lb_nn_up2(_p(self.a3), _p(self.u3), nb, n // 4, n // 4, 128, 0, self.s), "up")
        self._conv(self.u3, 3, self.a4, 1, n // 2)
        _check(L.lb_nn_add(_p(self.a4), _p(self.a2), _p(self.s4), self.s4.numel(), self.s), "add")
        _check(L.lb_nn_up2(_p(self.s4), _p(self.u4), nb, n // 2, n // 2, 64, 0, self.s), "up")
        self._conv(self.u4, 4, self.y, 0, n)
        if self.flux:
            _check(L.lb_nn_flux_div(_p(self.y), _p(self.inc), 16, nb, n, n, 0, self.s), "flux")
        return self.y

    @property
    def out(self):
        """The density increment of the last forward: [nb][n][n][out_c], channel 0."""
        return self.inc if self.flux else self.y

    @property
    def out_c(self):
        return 1 if self.flux else 16

    def twin(self):
        """A second set of activation buffers on the same parameters (the
        weights, their BF16 copies, biases and gradient sums are shared), for
        training through two strides."""
        t = object.__new__(SurrogateNet)
        t.__dict__.update({k: v for k, v in self.__dict__.items()
                           if k not in ("_stride_graph",)})
        t._alloc(self.nb)
        return t

    def two_stride_loss_and_grad(self, x, base, t1, t2):
        """Gradients of the two-stride loss mean((s1 - t1)^2) + mean((s1 +
        inc1 - t2)^2), s1 = base + inc0, where the second stride's input is
        the first prediction (channel 0 = s1, channel 2 = inc0): forward both
        strides, backward the second (with its input gradient), gather the
        gradient of inc0 (its own loss, the second loss through s1, and input
        channels 0 and 2), backward the first.  Plain increments only.
        Accumulates into the shared parameter gradients; returns the loss."""
        if self.flux or self.momentum:
            raise ValueError("two-stride training is for plain increments")
        t = self.torch
        if getattr(self, "_tw", None) is None or self._tw.nb != self.nb:
            self._tw = self.twin()
            self._x1 = t.empty_like(x)
            self._dx1 = t.empty_like(x)
            self._s1 = t.empty_like(base)
        tw, x1, dx1, s1 = self._tw, self._x1, self._dx1, self._s1
        L, npx = self.L, base.numel()
        self.forward(x)
        s1.copy_(base)
        x1.copy_(x)
        _check(L.lb_nn_residual(_p(s1), _p(self.y), 16, _p(x1), CIN, npx, None, self.s),
               "residual")
        tw.forward(x1)
        loss = self.loss_and_grad(x, t1, base)
        loss += tw.loss_and_grad(x1, t2, s1)
        tw.backward(x1, dx=dx1)
        for src, ch in ((tw.dy, 0), (dx1, 0), (dx1, 2)):
            _check(L.lb_nn_add_channel(_p(self.dy), 16, 0, _p(src), 16, ch, npx, self.s),
                   "add channel")
        self.backward(x)
        return loss

    def backward(self, x, dx=None):
        """Accumulate parameter gradients from self.dy (dL/dy); with `dx` (a
        BF16 [nb][n][n][16] buffer) also write dL/dx, the input gradient."""
        n, L, nb, s = self.n, self.L, self.nb, self.s
        wg = lambda inp, dz, i, h: _check(L.lb_nn_conv3x3_wgrad(
            _p(inp), _p(dz), _p(self.dw[i]), _p(self.db[i]), nb, h, h, LAYERS[i][0], LAYERS[i][1],
            _p(self.ws), self.ws_bytes, s), "wgrad")
        dg = lambda dz, i, out, h: _check(L.lb_nn_conv3x3(
            _p(dz), _p(self.wb[i]), None, _p(out), nb, h, h, LAYERS[i][1], LAYERS[i][0], 0, 1, s), "dgrad")
        wg(self.u4, self.dy, 4, n)
        dg(self.dy, 4, self.du4, n)
        _check(L.lb_nn_up2(_p(self.du4), _p(self.ds4), nb, n // 2, n // 2, 64, 1, s), "upb")
        _check(L.lb_nn_relu_mask(_p(self.ds4), _p(self.a4), _p(self.dz4), self.dz4.numel(), s), "relu")
        wg(self.u3, self.dz4, 3, n // 2)
        dg(self.dz4, 3, self.du3, n // 2)
        _check(L.lb_nn_up2(_p(self.du3), _p(self.da3), nb, n // 4, n // 4, 128, 1, s), "upb")
        _check(L.lb_nn_relu_mask(_p(self.da3), _p(self.a3), _p(self.dz3), self.dz3.numel(), s), "relu")
        wg(self.p2, self.dz3, 2, n // 4)
        dg(self.dz3, 2, self.dp2, n // 4)
        _check(L.lb_nn_pool2(_p(self.dp2), _p(self.tmp2), nb, n // 2, n // 2, 64, 1, s), "poolb")
        _check(L.lb_nn_add(_p(self.tmp2), _p(self.ds4), _p(self.da2), self.da2.numel(), s), "add")
        _check(L.lb_nn_relu_mask(_p(self.da2), _p(self.a2), _p(self.dz2), self.dz2.numel(), s), "relu")
        wg(self.p1, self.dz2, 1, n // 2)
        dg(self.dz2, 1, self.dp1, n // 2)
        _check(L.lb_nn_pool2(_p(self.dp1), _p(self.da1), nb, n, n, 32, 1, s), "poolb")
        _check(L.lb_nn_relu_mask(_p(self.da1), _p(self.a1), _p(self.dz1), self.dz1.numel(), s), "relu")
        wg(x, self.dz1, 0, n)
        if dx is not None:
            dg(self.dz1, 0, dx, n)

    def zero_grad(self):
        for t in self.dw + self.db:
            t.zero_()

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        for i in range(len(LAYERS)):
            _check(self.L.lb_nn_adam(_p(self.w[i]), _p(self.dw[i]), _p(self.mw[i]), _p(self.vw[i]),
                                     _p(self.wb[i]), self.w[i].numel(), lr, b1, b2, eps,
                                     self.step_count, self.s), "adam")
            _check(self.L.lb_nn_adam(_p(self.b[i]), _p(self.db[i]), _p(self.mb[i]), _p(self.vb[i]),
                                     None, self.b[i].numel(), lr, b1, b2, eps, self.step_count,
                                     self.s), "adam")

    def loss_and_grad(self, x, target, base, grad=True):
        """MSE of the residual prediction base + increment against the FP32
        target; fills self.dy when `grad` (through the flux divergence's
        adjoint in the flux form).  With `momentum`, target and base are
        [3][nb][n][n] (density, jx, jy) and the momentum MSE of output channels
        2 and 3, weighted by jweight, is added.  Returns the loss as a device
        tensor."""
        loss = self.torch.zeros(1, device="cuda")
        n, nb = self.n, self.nb
        npx = nb * n * n
        t0, b0 = (target[0], base[0]) if self.momentum else (target, base)
        d_out = self.dinc if self.flux else self.dy
        _check(self.L.lb_nn_mse(_p(self.out), self.out_c, _p(t0), _p(b0), npx, _p(loss),
                                _p(d_out) if grad else None, self.s), "mse")
        for blk, wgt in self.block_loss:
            _check(self.L.lb_nn_mse_blocks(_p(self.out), self.out_c, _p(t0), _p(b0), nb, n, n, blk,
                                           wgt, _p(loss), _p(d_out) if grad else None, self.s),
                   "block mse")
        if grad and self.flux:
            _check(self.L.lb_nn_flux_div(_p(self.dinc), _p(self.dy), 16, nb, n, n, 1, self.s),
                   "flux backward")
        if self.momentum:
            for a in (1, 2):
                _check(self.L.lb_nn_mse_channel(_p(self.y), 16, a + 1, _p(target[a]), _p(base[a]),
                                                npx, self.jweight, _p(loss),
                                                _p(self.dy) if grad else None, self.s), "mse j")
        return loss


def generate(n_traj, size, steps, stride, G_range=(-5.2, -4.4), coarse=4, kT=1e-6, seed0=1000,
             rho0=math.log(2.0), stencil=4, momentum=False):
    """Quench trajectories of the lattice solver from a homogeneous density
    rho0 with thermal noise, coarse-grained every `stride` steps.  Returns
    (frames, the couplings G, seconds spent): frames FP32
    [n_traj][steps // stride + 1][size/coarse][size/coarse] of rho - rho0, or
    with `momentum` [n_traj][nf][3][m][m] holding rho - rho0, jx / J_SCALE and
    jy / J_SCALE."""
    import torch

    from .lattice import Lattice
    L = abi.load()
    rng = np.random.default_rng(seed0)
    Gs = rng.uniform(G_range[0], G_range[1], n_traj)
    nf = steps // stride + 1
    m = size // coarse
    shape = (n_traj, nf, 3, m, m) if momentum else (n_traj, nf, m, m)
    frames = torch.empty(shape, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(n_traj):
        lat = Lattice(size, size, float(Gs[k]), 1.0, kT, stencil=stencil)
        lat.init(rho0, seed0 + k, 0.0)
        df = C.c_void_p(lat.device_ptr(abi.LB_PTR_POPULATIONS))
        st = C.c_void_p(lat.stream())
        for f in range(nf):
            if f:
                lat.step(stride)
            rho = frames[k, f, 0] if momentum else frames[k, f]
            _check(L.lb_nn_coarse_grain(df, size, size, coarse, 1.0, _p(rho), st), "coarse")
            if momentum:
                _check(L.lb_nn_coarse_momentum(df, size, size, coarse, J_SCALE, _p(frames[k, f, 1]),
                                               _p(frames[k, f, 2]), st), "coarse momentum")
        lat.sync()
        lat.close()
    torch.cuda.synchronize()
    return frames, Gs, time.perf_counter() - t0


def expand(L, field, G, out, prev=None, stream=None):
    """16-channel BF16 network input [..][m][m][16] from an FP32 field [..][m][m]:
    the field, the coupling feature and (with `prev`) the field's last increment."""
    _check(L.lb_nn_expand(_p(field), _p(prev), gfeat(G), _p(out), CIN, field.numel(), stream),
           "expand")


def expand_state(L, frame, G, out, prev=None, stream=None):
    """Network input from one frame: [m][m] (density only) or [3][m][m]
    (density, jx, jy: momentum in channels 3, 4 and its last increment in 5, 6)."""
    if frame.dim() == 2:
        return expand(L, frame, G, out, prev, stream)
    expand(L, frame[0], G, out, prev[0] if prev is not None else None, stream)
    for a in (1, 2):
        _check(L.lb_nn_expand_channel(_p(frame[a]), _p(prev[a]) if prev is not None else None,
                                      _p(out), CIN, a + 2, frame[a].numel(), stream), "expand j")


def advance(net, state, x, npx, mean=None):
    """Apply the network's last output to the FP32 state (density [..] or
    [3][..]) and refresh the matching input channels of x: the density by
    the increment (projected to zero mean when `mean` is a buffer), the
    momentum by output channels 2, 3 (likewise; the lattice conserves it)."""
    L, s = net.L, net.s
    rho = state[0] if net.momentum else state
    _check(L.lb_nn_residual(_p(rho), _p(net.out), net.out_c, _p(x), CIN, npx, _p(mean), s),
           "residual")
    if net.momentum:
        for a in (1, 2):
            _check(L.lb_nn_residual(_p(state[a]), _pc(net.y, a + 1), 16, _pc(x, a + 2), CIN, npx,
                                    _p(mean), s), "residual j")


def train(net, frames, Gs, train_ids, iters, lr=1e-3, seed=0, log_every=0, t_min=1, lr_end=None,
          pushforward=0.0, pf_depth=1, two_stride=0.0):
    """Adam on random (trajectory, time) pairs of consecutive frames, the frame
    before each pair giving the last-increment input; the learning rate decays
    from `lr` to `lr_end` on a cosine (constant without `lr_end`).  With
    probability `pushforward` an iteration first advances the batch one stride
    with the network itself (no gradient) and trains on that prediction as the
    input (the pushforward trick: the network learns to correct its own
    rollout errors); with pf_depth > 1 that advance is 1 .. pf_depth strides
    (uniform), so it also learns from errors compounded over several strides.
    With probability `two_stride` an iteration instead trains through two
    strides with gradients (two_stride_loss_and_grad; plain increments).
    Returns the losses logged every `log_every` iterations."""
    import torch
    L = net.L
    if net.nb != net.batch:
        net._alloc(net.batch)
    nb, m = net.nb, net.n
    mom = frames.dim() == 5
    if mom != net.momentum:
        raise ValueError("frames and network disagree on the momentum state")
    x = torch.empty((nb, m, m, CIN), dtype=torch.bfloat16, device="cuda")
    shape = (3, nb, m, m) if mom else (nb, m, m)
    base = torch.empty(shape, dtype=torch.float32, device="cuda")
    tgt = torch.empty(shape, dtype=torch.float32, device="cuda")
    bview = (lambda j: base[:, j]) if mom else (lambda j: base[j])
    tview = (lambda j: tgt[:, j]) if mom else (lambda j: tgt[j])
    rng = np.random.default_rng(seed)
    nf = frames.shape[1]
    losses = []
    t2 = torch.empty((nb, m, m), dtype=torch.float32, device="cuda") if two_stride > 0 else None
    for it in range(iters):
        if two_stride > 0.0 and rng.random() < two_stride:
            for j in range(nb):
                k = int(rng.choice(train_ids))
                f = int(rng.integers(t_min, nf - 2))
                base[j].copy_(frames[k, f])
                tgt[j].copy_(frames[k, f + 1])
                t2[j].copy_(frames[k, f + 2])
                expand_state(L, frames[k, f], Gs[k], x[j], frames[k, f - 1] if f > 0 else None,
                             net.s)
            net.zero_grad()
            loss = net.two_stride_loss_and_grad(x, base, tgt, t2)
            _adam_step(net, it, iters, lr, lr_end)
            if log_every and it % log_every == 0:
                losses.append(float(loss.item()))
            continue
        pf = pushforward > 0.0 and rng.random() < pushforward
        depth = (int(rng.integers(1, pf_depth + 1)) if pf_depth > 1 else 1) if pf else 0
        for j in range(nb):
            k = int(rng.choice(train_ids))
            f = int(rng.integers(max(t_min, depth + 1) if pf else t_min, nf - 1))
            src = f - depth
            bview(j).copy_(frames[k, src])
            tview(j).copy_(frames[k, f + 1])
            expand_state(L, frames[k, src], Gs[k], x[j], frames[k, src - 1] if src > 0 else None,
                         net.s)
        for _ in range(depth):
            # strides by the network itself: base becomes its prediction of
            # frame f, x the matching input (with the increments just applied)
            net.forward(x)
            advance(net, base, x, nb * m * m)
        net.zero_grad()
        net.forward(x)
        loss = net.loss_and_grad(x, tgt, base)
        net.backward(x)
        _adam_step(net, it, iters, lr, lr_end)
        if log_every and it % log_every == 0:
            losses.append(float(loss.item()))
    return losses


def _adam_step(net, it, iters, lr, lr_end):
    if lr_end is None:
        net.adam(lr)
    else:
        net.adam(lr_end + 0.5 * (lr - lr_end) * (1.0 + math.cos(math.pi * it / max(iters - 1, 1))))


def one_step_mse(net, frames, Gs, ids, t_min=1):
    """Mean one-stride MSE of the surrogate's density and of persistence (no
    change) over all consecutive frame pairs of the trajectories `ids`,
    `net.nb` pairs per forward pass (unused slots of the last pass repeat its
    last pair)."""
    import torch
    L, nb, m = net.L, net.nb, net.n
    mom = frames.dim() == 5
    x = torch.empty((nb, m, m, CIN), dtype=torch.bfloat16, device="cuda")
    base = torch.empty((nb, m, m), dtype=torch.float32, device="cuda")
    tgt = torch.empty((nb, m, m), dtype=torch.float32, device="cuda")
    rho = (lambda fr: fr[0]) if mom else (lambda fr: fr)
    pairs = [(k, f) for k in ids for f in range(t_min, frames.shape[1] - 1)]
    s_net, s_id = 0.0, 0.0
    for i in range(0, len(pairs), nb):
        chunk = pairs[i:i + nb]
        chunk = chunk + [chunk[-1]] * (nb - len(chunk))
        for j, (k, f) in enumerate(chunk):
            base[j].copy_(rho(frames[k, f]))
            tgt[j].copy_(rho(frames[k, f + 1]))
            expand_state(L, frames[k, f], Gs[k], x[j], frames[k, f - 1] if f > 0 else None, net.s)
        net.forward(x)
        used = len(pairs[i:i + nb])
        d2 = ((tgt - base) ** 2).mean(dim=(1, 2))
        y0 = net.out[..., 0].float()
        e2 = ((base + y0 - tgt) ** 2).mean(dim=(1, 2))
        s_net += float(e2[:used].sum())
        s_id += float(d2[:used].sum())
    return s_net / len(pairs), s_id / len(pairs)


class _StrideGraph:
    """One surrogate stride (network forward + state update) captured once
    as a CUDA graph on a private stream, on fixed input/state buffers."""

    def __init__(self, net):
        import torch
        self.torch = torch
        m = net.n
        self.net = net
        self.stream = torch.cuda.Stream()
        self.x = torch.zeros((1, m, m, CIN), dtype=torch.bfloat16, device="cuda")
        shape = (3, m, m) if net.momentum else (m, m)
        self.state = torch.zeros(shape, dtype=torch.float32, device="cuda")
        self.mean = torch.zeros(513, dtype=torch.float32, device="cuda")
        saved = net.s
        net.s = self.stream.cuda_stream
        try:
            torch.cuda.synchronize()
            with torch.cuda.stream(self.stream):
                net.forward(self.x)          # first launches (kernel attributes) outside capture
            self.stream.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream):
                net.forward(self.x)
                advance(net, self.state, self.x, m * m, self.mean)
        finally:
            net.s = saved

    def run(self, frame0, G, strides, prev0, out):
        torch = self.torch
        net = self.net
        rho = self.state[0] if net.momentum else self.state
        with torch.cuda.stream(self.stream):
            self.stream.wait_stream(torch.cuda.current_stream())
            self.state.copy_(frame0)
            expand_state(net.L, self.state, G, self.x, prev0, self.stream.cuda_stream)
            for s in range(strides):
                self.graph.replay()
                out[s].copy_(rho)
        torch.cuda.current_stream().wait_stream(self.stream)
        return out


def rollout(net, frame0, G, strides, prev0=None, graph=True):
    """Apply the surrogate `strides` times from an FP32 frame ([m][m], or
    [3][m][m] with momentum) and the frame one stride earlier (for the
    last-increment inputs); the state stays FP32 (only the network input is
    BF16) and each increment is projected to zero mean, so the field's mass
    (and momentum) is conserved as on the lattice.  Returns the FP32 density
    after each stride as one tensor [strides][m][m].  With `graph` each
    stride replays a CUDA graph captured on the first call."""
    import torch
    L, m = net.L, net.n
    if net.nb != 1:
        net._alloc(1)
        net._stride_graph = None
    out = torch.empty((strides, m, m), dtype=torch.float32, device="cuda")
    if graph:
        if getattr(net, "_stride_graph", None) is None:
            net._stride_graph = _StrideGraph(net)
        return net._stride_graph.run(frame0, G, strides, prev0, out)
    x = torch.empty((1, m, m, CIN), dtype=torch.bfloat16, device="cuda")
    mean = torch.zeros(513, dtype=torch.float32, device="cuda")
    state = frame0.clone()
    expand_state(L, state, G, x, prev0, net.s)
    for s in range(strides):
        net.forward(x)
        advance(net, state, x, m * m, mean)
        out[s].copy_(state[0] if net.momentum else state)
    return out


def guarded_rollout(net, frame0, G, strides, prev0=None, mass_tol=1e-3, bound=None):
    """Rollout with the checks that decide when the solver has to take over:
    the lattice conserves mass exactly, so the coarse field's mean must stay
    within `mass_tol` of its initial mean, and the field must stay inside
    `bound` (default: 1.5 x the initial field's largest |value|, at least 1).
    Returns (fields [n][m][m] accepted, n): n < strides means the surrogate
    left its domain after n strides and the caller continues with the solver
    from the last accepted state."""
    out = rollout(net, frame0, G, strides, prev0)
    rho0 = frame0[0] if frame0.dim() == 3 else frame0
    means = out.mean(dim=(1, 2)).cpu().numpy()
    peaks = out.abs().amax(dim=(1, 2)).cpu().numpy()
    m0 = float(rho0.mean())
    lim = bound if bound is not None else max(1.0, 1.5 * float(rho0.abs().max()))
    ok = (np.abs(means - m0) <= mass_tol) & np.isfinite(means) & (peaks <= lim)
    n = int(np.argmin(ok)) if not ok.all() else strides
    return out[:n], n


def compare_ensembles(out, ref):
    """The ensemble metrics of evaluate_rollouts for rollouts `out` and solver
    frames `ref` (lists over trajectories of [nroll][m][m] arrays)."""
    Ls, Lr, Ss, Sr, per = [], [], [], [], []
    for o, r in zip(out, ref):
        a = [radial_sk(f) for f in o]
        b = [radial_sk(f) for f in r]
        Ls.append([v[1] for v in a])
        Lr.append([v[1] for v in b])
        Ss.append([v[0] for v in a])
        Sr.append([v[0] for v in b])
        per.append(np.max(np.abs(np.array(Ls[-1]) - np.array(Lr[-1])) / np.array(Lr[-1])))
    Ls, Lr = np.mean(Ls, axis=0), np.mean(Lr, axis=0)
    Ss, Sr = np.mean(Ss, axis=0), np.mean(Sr, axis=0)
    s_peak, s_l1 = 0.0, 0.0
    for t in range(len(Ls)):
        sel = Sr[t] >= 0.25 * Sr[t].max()
        s_peak = max(s_peak, float(np.max(np.abs(Ss[t][sel] - Sr[t][sel]) / Sr[t][sel])))
        s_l1 = max(s_l1, float(np.abs(Ss[t] - Sr[t]).sum() / Sr[t].sum()))
    return {"L_surrogate": Ls.tolist(), "L_solver": Lr.tolist(),
            "L_mean_max_rel_err": float(np.max(np.abs(Ls - Lr) / Lr)),
            "L_traj_max_rel_err": float(np.max(per)), "Sk_peak_max_rel_err": s_peak,
            "Sk_l1_rel_err": s_l1, "Sk_surrogate": Ss, "Sk_solver": Sr}


def solver_reseeded(frames, Gs, ids, f0, nroll, size, stride, seed0, coarse=4, kT=1e-6,
                    rho0=math.log(2.0), stencil=4):
    """The floor of any predictor of S(k, t): each trajectory of `ids` is
    re-run by the solver to frame f0 (the same fine state as in `generate`
    with the same seed0), then continued on an independent noise stream
    (replica counter 1) for `nroll` strides and compared with its own frames
    by the metrics of evaluate_rollouts."""
    import torch

    from .lattice import Lattice
    L = abi.load()
    m = size // coarse
    outs, refs = [], []
    buf = torch.empty((nroll, m, m), dtype=torch.float32, device="cuda")
    for k in ids:
        lat = Lattice(size, size, float(Gs[k]), 1.0, kT, stencil=stencil)
        lat.init(rho0, seed0 + k, 0.0)
        lat.step(f0 * stride)
        lat.set_replica(1)
        df = C.c_void_p(lat.device_ptr(abi.LB_PTR_POPULATIONS))
        for s in range(nroll):
            lat.step(stride)
            _check(L.lb_nn_coarse_grain(df, size, size, coarse, 1.0, _p(buf[s]),
                                        C.c_void_p(lat.stream())), "coarse")
        lat.sync()
        lat.close()
        outs.append(buf.cpu().numpy().copy())
        ref = frames[k, f0 + 1:f0 + 1 + nroll]
        refs.append((ref[:, 0] if frames.dim() == 5 else ref).cpu().numpy())
    return compare_ensembles(outs, refs)


def evaluate_rollouts(net, frames, Gs, ids, f0, nroll):
    """Score the surrogate against the solver: from frame f0 of each trajectory
    in `ids` (with frame f0 - 1 for the increment input) roll out `nroll`
    strides and compare with the solver's frames f0+1 .. f0+nroll.  Returns
    the ensemble-mean domain size L(t) of both, their largest relative gap,
    the largest per-trajectory L gap, and two measures of the ensemble-mean
    radial S(k, t) gap, each the worst over the rollout: the largest relative
    gap over the peak shells (solver S at least a quarter of its maximum) and
    the L1 gap sum |S_sur - S_sol| / sum S_sol over all shells."""
    outs, refs = [], []
    for k in ids:
        outs.append(rollout(net, frames[k, f0].clone(), float(Gs[k]), nroll,
                            frames[k, f0 - 1] if f0 > 0 else None).cpu().numpy())
        ref = frames[k, f0 + 1:f0 + 1 + nroll]
        refs.append((ref[:, 0] if frames.dim() == 5 else ref).cpu().numpy())
    return compare_ensembles(outs, refs)


def radial_sk(field):
    """Radial S(k) (mean |FFT|^2 / N per integer shell) and L = 2 pi sum S / sum |k| S
    of a periodic 2D field (host analysis of evaluation frames)."""
    f = np.asarray(field, np.float64)
    f = f - f.mean()
    n = f.shape[0]
    S = np.abs(np.fft.fft2(f)) ** 2 / f.size
    k = np.fft.fftfreq(n) * n
    kk = np.hypot(*np.meshgrid(k, k))
    b = np.rint(kk).astype(int)
    S[0, 0] = 0.0
    sums = np.bincount(b.ravel(), S.ravel(), minlength=n)
    cnt = np.bincount(b.ravel(), minlength=n)
    Sb = np.where(cnt > 0, sums / np.maximum(cnt, 1), 0.0)
    kabs = 2 * np.pi * kk / n
    Ld = 2 * np.pi * S.sum() / (kabs * S).sum()
    return Sb, Ld
