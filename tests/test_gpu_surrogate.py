"""The learned surrogate end to end on the GPU: the whole network's forward
pass, loss and parameter gradients (all liblbsc kernels) against the FP64
CPU reference; then training on solver quench trajectories, where the
trained operator must beat persistence on held-out trajectories, roll out
stably, and take less time per stride than the solver's steps it replaces."""
import math
import time

import numpy as np
import pytest

from oracle import surrogate_ref as R

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(got, ref):
    return float(np.sqrt(np.mean((got - ref) ** 2)) / (np.sqrt(np.mean(ref ** 2)) + 1e-30))


@pytest.mark.parametrize("flux,mom,n", [(False, False, 64), (True, False, 64), (True, True, 64),
                                        (False, False, 128)])
def test_network_gradients_match_reference(flux, mom, n):
    """Plain increment, flux form, and flux form with the momentum state; at
    n = 128 the full-resolution layers (rows of 128 pixels) run on the
    persistent tensor-core kernel, forward and input gradient."""
    from paper_2212_07848_gb300.surrogate import LAYERS, SurrogateNet
    nb = 2 if n == 64 else 1
    net = SurrogateNet(n, nb, seed=3, flux=flux, momentum=mom, jweight=0.7)
    g = torch.Generator(device="cpu").manual_seed(4)
    for i in range(len(LAYERS)):                   # a non-trivial output layer and biases
        net.w[i].copy_(torch.randn(net.w[i].shape, generator=g).cuda()
                       * math.sqrt(2.0 / (9 * LAYERS[i][0])))
        net.wb[i].copy_(net.w[i].to(torch.bfloat16))
        net.b[i].copy_(0.1 * torch.randn(net.b[i].shape, generator=g).cuda())
    x = torch.randn((nb, n, n, 16), generator=g).to(torch.bfloat16).cuda()
    base = torch.randn((nb, n, n), generator=g).cuda()
    tgt = torch.randn((nb, n, n), generator=g).cuda()
    if flux:
        # A smooth residual: the flux adjoint differentiates d, and the coarse
        # layers then sum the derivative over blocks, which for a white-noise d
        # would cancel down to the BF16 rounding of the intermediate gradients.
        yy, xx = torch.meshgrid(torch.arange(n), torch.arange(n), indexing="ij")
        sm = sum(torch.sin(2 * math.pi * (kx * xx + ky * yy) / n + ph)
                 for kx, ky, ph in ((1, 0, 0.3), (0, 2, 1.1), (1, 1, 2.0), (3, 1, 0.7)))
        tgt = base - 10.0 * sm.float().cuda()[None]
    if mom:                                   # density, jx, jy planes
        base = torch.stack([base] + [torch.randn((nb, n, n), generator=g).cuda() for _ in range(2)])
        tgt = torch.stack([tgt] + [torch.randn((nb, n, n), generator=g).cuda() for _ in range(2)])
    net.zero_grad()
    net.forward(x)
    loss = net.loss_and_grad(x, tgt, base)
    net.backward(x)
    torch.cuda.synchronize()

    w = [t.float().cpu().numpy().astype(np.float64) for t in net.wb]
    b = [t.cpu().numpy().astype(np.float64) for t in net.b]
    xr = x.float().cpu().numpy().astype(np.float64)
    y, acts = R.net_forward(xr, w, b)
    jw = 0.7 if mom else None
    ref_loss, d = R.net_loss(y, base.cpu().numpy(), tgt.cpu().numpy(), flux, jw)
    dw, db = R.net_backward(xr, w, acts, d, flux, jw)
    assert _rel(net.y.float().cpu().numpy(), y) < 2e-2
    if flux:
        inc = net.out[..., 0].float().cpu().numpy()
        assert _rel(inc, R.flux_div(net.y.float().cpu().numpy())) < 1e-2
        assert _rel(inc, R.flux_div(y)) < 5e-2
    assert abs(float(loss.item()) - ref_loss) < 1e-2 * ref_loss
    # The flux adjoint differences BF16 gradients, and its output sums to zero
    # over each image, so the bias gradients (pixel sums) are small residues
    # of cancellation that only the ReLU masks leave: looser bounds there.
    # Measured on GB300 (relative RMS errors, BF16 activations and gradients
    # between layers): plain increments at most 0.012 (the first layer's
    # weights, whose gradient sums BF16 gradients over every pixel) and 0.0024
    # for biases; the flux form with the momentum state 0.038; the flux form
    # alone 0.072 / 0.082, its adjoint differencing BF16 gradients.
    tol, tol_b = (8e-2, 1.5e-1) if flux else (2.5e-2, 1e-2)
    if flux and mom:
        tol, tol_b = 6e-2, 4e-2
    for i in range(len(LAYERS)):
        assert _rel(net.dw[i].cpu().numpy(), dw[i]) < tol, i
        if flux and i == len(LAYERS) - 1:
            # exactly 0 in exact arithmetic for the flux channels 0, 1: bound
            # the sum of P BF16-rounded dy values by its rounding error (the
            # momentum channels 2, 3 also get 2% of their value)
            dyg = net.dy.float().cpu().numpy().reshape(-1, LAYERS[i][1])
            bound = 4.0 * np.sqrt(dyg.shape[0]) * 2.0 ** -8 * np.sqrt((dyg ** 2).mean(axis=0))
            err = np.abs(net.db[i].cpu().numpy() - db[i])
            assert np.all(err <= bound + 2e-2 * np.abs(db[i]) + 1e-12), err
            continue
        assert _rel(net.db[i].cpu().numpy(), db[i]) < tol_b, i


@pytest.fixture(scope="module")
def trained():
    from paper_2212_07848_gb300 import surrogate as S
    frames, Gs, gen_s = S.generate(12, 256, 3000, 200, seed0=2000)
    net = S.SurrogateNet(64, 8, seed=0)
    # the first stride (uniform noise -> separated domains) carries no
    # information at the coarse scale: train and score from frame 1 on
    before = S.one_step_mse(net, frames, Gs, [10, 11], t_min=1)
    losses = S.train(net, frames, Gs, list(range(10)), 1000, lr=1e-3, seed=1, log_every=50,
                     t_min=1)
    return S, net, frames, Gs, losses, before


def test_training_beats_persistence(trained):
    S, net, frames, Gs, losses, before = trained
    assert np.all(np.isfinite(losses))
    assert before[0] > 0.9 * before[1]             # starts out as (nearly) persistence
    mse, persist = S.one_step_mse(net, frames, Gs, [10, 11], t_min=1)
    print(f"held-out one-stride MSE {mse:.3e} vs persistence {persist:.3e}")
    assert mse < 0.7 * persist


def test_rollout_stable_and_faster_than_solver(trained):
    S, net, frames, Gs, _, _ = trained
    from paper_2212_07848_gb300.lattice import Lattice
    k, f0, strides = 10, 3, 8
    out = S.rollout(net, frames[k, f0].clone(), float(Gs[k]), strides, frames[k, f0 - 1])
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.all(np.isfinite(o)) and np.abs(o).max() < 3.0
    # the captured-graph rollout replays exactly the eager one
    eager = S.rollout(net, frames[k, f0].clone(), float(Gs[k]), strides, frames[k, f0 - 1],
                      graph=False)
    assert torch.equal(eager, out)
    # time per stride of the surrogate against the 200 solver steps it stands for
    x0 = frames[k, f0].clone()
    S.rollout(net, x0, float(Gs[k]), 2, frames[k, f0 - 1])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S.rollout(net, x0, float(Gs[k]), 20, frames[k, f0 - 1])
    torch.cuda.synchronize()
    t_net = (time.perf_counter() - t0) / 20
    lat = Lattice(256, 256, float(Gs[k]), 1.0, 1e-6)
    lat.init(math.log(2.0), 5, 0.0)
    lat.step(200)
    lat.sync()
    t0 = time.perf_counter()
    lat.step(2000)
    lat.sync()
    t_lb = (time.perf_counter() - t0) / 10
    lat.close()
    print(f"surrogate {t_net * 1e3:.3f} ms/stride, solver {t_lb * 1e3:.3f} ms per 200 steps")
    assert t_net < t_lb


# Rollout scores of the small training case (12 quenches of 256^2 -> 64^2,
# 1000 iterations, held-out quenches 10 and 11 from frame 3 over 10 strides),
# the regression bounds of the bench's surrogate metrics at this size.  The
# training is bit-reproducible, so on the same GPU the scores are fixed, but
# one short training is chaotic in its rounding: a change of the summation
# order of a gradient kernel moved seed 0's S(k, t) L1 gap from 0.28 to 0.41
# and 0.54, and over initial seeds 0-3 it measured 0.25-0.41 (L(t) gap
# 0.05-0.12).  So the test scores three networks (initial seeds 0, 1, 2) and
# bounds their mean, about 30% above the largest mean seen (0.41 and 0.11);
# each network must stay clear of a failed training (scores below 1).  A
# short training on a 64^2 grid is far from the 2% of the paper-scale target,
# whose figures are the bench's.
ROLLOUT_BOUNDS = {"L_mean_max_rel_err": 0.15, "Sk_l1_rel_err": 0.55}


def test_rollout_scores_against_the_solver(trained):
    S, net, frames, Gs, _, _ = trained
    keys = ("L_mean_max_rel_err", "L_traj_max_rel_err", "Sk_peak_max_rel_err", "Sk_l1_rel_err")
    scores = []
    for seed in (0, 1, 2):
        if seed == 0:
            n = net
        else:
            n = S.SurrogateNet(64, 8, seed=seed)
            S.train(n, frames, Gs, list(range(10)), 1000, lr=1e-3, seed=1, t_min=1)
        ev = S.evaluate_rollouts(n, frames, Gs, [10, 11], 3, 10)
        got = {k: ev[k] for k in keys}
        print("rollout scores, seed", seed, got)
        for k in ROLLOUT_BOUNDS:
            assert np.isfinite(got[k]) and got[k] < 1.0, (seed, k, got[k])
        scores.append(got)
    for k, bound in ROLLOUT_BOUNDS.items():
        mean = float(np.mean([g[k] for g in scores]))
        assert mean < bound, (k, mean)


def test_guarded_rollout_hands_back_to_the_solver(trained):
    """Rollout increments have zero mean, so the field's mass stays at its
    initial value to FP32 rounding and the mass guard accepts the rollout
    whole; a bound the field cannot meet hands over to the solver at once."""
    S, net, frames, Gs, _, _ = trained
    k, f0 = 11, 4
    fields, n = S.guarded_rollout(net, frames[k, f0].clone(), float(Gs[k]), 6, frames[k, f0 - 1],
                                  mass_tol=1e-4, bound=10.0)
    assert n == 6 and fields.shape[0] == 6
    drift = (fields.double().mean(dim=(1, 2)) - frames[k, f0].double().mean()).abs().max()
    assert float(drift) < 1e-5
    fields, n = S.guarded_rollout(net, frames[k, f0].clone(), float(Gs[k]), 6, frames[k, f0 - 1],
                                  mass_tol=0.0, bound=1e-9)
    assert n == 0 and fields.shape[0] == 0


def test_training_is_reproducible():
    """Two trainings from the same seed on the same frames give the same
    weights bit for bit (every gradient sum runs in a fixed order)."""
    from paper_2212_07848_gb300 import surrogate as S
    frames, Gs, _ = S.generate(3, 256, 800, 200, seed0=3000)
    ws = []
    for _ in range(2):
        net = S.SurrogateNet(64, 4, seed=5)
        S.train(net, frames, Gs, [0, 1, 2], 40, lr=1e-3, seed=2, pushforward=0.5)
        torch.cuda.synchronize()
        ws.append([w.clone() for w in net.w] + [b.clone() for b in net.b])
    for a, b in zip(*ws):
        assert torch.equal(a, b)


def test_two_stride_gradients_match_reference():
    """Training through two strides: the gradients of the two-stride loss
    (the first prediction fed back as the second input) against the FP64
    CPU reference."""
    from paper_2212_07848_gb300.surrogate import LAYERS, SurrogateNet
    n, nb = 64, 2
    net = SurrogateNet(n, nb, seed=7)
    g = torch.Generator(device="cpu").manual_seed(8)
    for i in range(len(LAYERS)):
        net.w[i].copy_(torch.randn(net.w[i].shape, generator=g).cuda()
                       * math.sqrt(2.0 / (9 * LAYERS[i][0])) * (0.3 if i == 4 else 1.0))
        net.wb[i].copy_(net.w[i].to(torch.bfloat16))
        net.b[i].copy_(0.1 * torch.randn(net.b[i].shape, generator=g).cuda())
    x = torch.randn((nb, n, n, 16), generator=g).to(torch.bfloat16).cuda()
    base = x[..., 0].float().contiguous()
    t1 = base + 0.3 * torch.randn((nb, n, n), generator=g).cuda()
    t2 = t1 + 0.3 * torch.randn((nb, n, n), generator=g).cuda()
    net.zero_grad()
    loss = net.two_stride_loss_and_grad(x, base, t1, t2)
    torch.cuda.synchronize()
    w = [t.float().cpu().numpy().astype(np.float64) for t in net.wb]
    b = [t.cpu().numpy().astype(np.float64) for t in net.b]
    xr = x.float().cpu().numpy().astype(np.float64)
    ref_loss, mid = R.two_stride_loss(xr, w, b, base.cpu().numpy(), t1.cpu().numpy(),
                                      t2.cpu().numpy())
    dw, db = R.two_stride_backward(xr, w, b, t1.cpu().numpy(), t2.cpu().numpy(), mid)
    assert abs(float(loss.item()) - ref_loss) < 2e-2 * ref_loss
    # measured on GB300: at most 0.022 (first layer's weights), biases 0.0034
    for i in range(len(LAYERS)):
        assert _rel(net.dw[i].cpu().numpy(), dw[i]) < 4e-2, i
        assert _rel(net.db[i].cpu().numpy(), db[i]) < 1e-2, i
