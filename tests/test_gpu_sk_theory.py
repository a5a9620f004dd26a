"""FP32 ensemble S(k) against the paper's theory, Eq. (16) on lattice axes,
and against the FP64 path on the same noise.

Ensembles of 64 replicas of 128^2 (the batched-ensemble kernel), 2000 steps,
S(k) sampled every step over the last 1000.  Axis modes k = 2 pi m / 128
with m >= 4 have relaxed (nu k^2 x 1000 >= 8); each of them must agree with
the closed form within 2% or, where the ensemble's own statistical error is
larger, within 4 of its standard errors (estimated from the spread of the
128 per-replica, per-axis means).  States: the supercritical C1 state
(G = -3.6, rho0 = ln 2) and a metastable gas between coexistence and the
gas spinodal at G = -4.5, where the low-k modes are enhanced about
fifteen-fold."""
import numpy as np
import pytest

from oracle import theory as T
from pairs import LN2

pytestmark = pytest.mark.gpu

L, NREP, STEPS, START = 128, 64, 2000, 1001


def _axis_means(e, nrep):
    """Per replica and axis, the time-averaged S at k = 2 pi m / L, m = 1..L/2."""
    vals = []
    for r in range(nrep):
        S, n = e.structure_factor(r)
        assert n == STEPS - START + 1
        vals.append(S[0, 1:L // 2 + 1])          # k along x
        vals.append(S[1:L // 2 + 1, 0])          # k along y
    return np.array(vals)


@pytest.mark.parametrize("G,rho0,kT", [(-3.6, LN2, 1e-5), (-4.5, 0.35, 1e-6)])
def test_ensemble_sk_matches_eq16_on_axes(G, rho0, kT):
    from paper_2212_07848_gb300.ensemble import Ensemble
    if G == -4.5:
        g_sp = T.spinodal(G)[0]
        g_co = T.coexistence(G, eps=0.0)[0]
        assert g_co < rho0 < g_sp                # metastable gas
    e = Ensemble([(L, L, G, 1.0, kT, rho0)] * NREP, seed=11)
    e.init(0.0)
    e.sk_config(1, START)
    e.step(STEPS)
    e.sync()
    v = _axis_means(e, NREP)
    m = np.arange(1, L // 2 + 1)
    th = T.sk_axis(2 * np.pi * m / L, rho0, G, kT)
    mean = v.mean(axis=0)
    sem = v.std(axis=0, ddof=1) / np.sqrt(v.shape[0])
    sel = m >= 4
    dev = np.abs(mean - th)
    ok = (dev <= 0.02 * th) | (dev <= 4 * sem)
    assert ok[sel].all(), [(int(mm), float(a / b - 1), float(s / b))
                           for mm, a, b, s, o in zip(m, mean, th, sem, ok) if not o and mm >= 4]
    # no systematic bias beyond the statistics
    chi2 = np.mean(((mean[sel] - th[sel]) / sem[sel]) ** 2)
    assert chi2 < 2.0, chi2
    if G == -4.5:
        assert th[3] > 8 * rho0 * kT / T.CS2     # the enhancement is really probed


def test_fp32_sk_agrees_with_fp64_on_the_same_noise():
    """Same seeds and replica indices: the FP32 deviation storage reproduces
    the FP64 S(k) of each replica far inside 2% per mode."""
    from paper_2212_07848_gb300.lattice import Lattice
    worst = 0.0
    for r in range(4):
        S = []
        for prec in ("fp32", "fp64"):
            g = Lattice(L, L, -3.6, 1.0, 1e-5, precision=prec)
            g.set_replica(r)
            g.init(LN2, 11, 0.0)
            g.sk_config(1, START)
            g.step(STEPS)
            S.append(g.structure_factor()[0])
            g.close()
        a, b = S
        nz = b > 0
        worst = max(worst, float(np.max(np.abs(a[nz] - b[nz]) / b[nz])))
    assert worst < 0.02, worst


def test_uneven_c4_ensemble_sk_matches_eq16_per_k_bin():
    """The batched-ensemble workload itself: 256 replicas with sides drawn from
    {64, 128, 256, 512}, G ~ U[-4.8, -3.6], rho0 = ln 2 (1 + U[-0.1, 0.1]),
    kT = 1e-6, 2e4 steps, S(k) sampled every 5 steps after 2000.  The mix sits
    around the critical point (rho0 near rho_c = ln 2, T_hat = -4/G from 0.83
    to 1.11): the replicas with G < -4 are quenched inside the spinodal and
    phase separate, those with G > -4 stay homogeneous with 1 + G psi psi'
    between 0 and 0.1.  The homogeneous replicas with 1 + G psi psi' >= 0.03
    are compared on their axis modes with |k| >= 0.25 (relaxed within the
    first 2000 steps) with Eq. (16) at their own G and rho0: in every k-bin of
    width 0.25 the ensemble mean of S / S_theory is within 2% of 1, or within
    4 standard errors where those exceed 2%."""
    from paper_2212_07848_gb300.ensemble import Ensemble
    rng = np.random.default_rng(7)
    nrep = 256
    sizes = rng.choice([64, 128, 256, 512], size=nrep)
    Gs = rng.uniform(-4.8, -3.6, nrep)
    rhos = LN2 * (1.0 + rng.uniform(-0.1, 0.1, nrep))
    kT = 1e-6
    reps = [(int(n), int(n), float(g), 1.0, kT, float(r)) for n, g, r in zip(sizes, Gs, rhos)]
    e = Ensemble(reps, seed=7)
    e.init(0.0)
    e.sk_config(5, 2005)
    e.step(20000)
    e.sync()
    ratios, ks = [], []
    nstable = 0
    for r, (n, _, G, _, _, rho0) in enumerate(reps):
        c = 1.0 + G * float(T.psi(rho0) * T.dpsi(rho0))
        if c < 0.03:
            continue
        nstable += 1
        S, ns = e.structure_factor(r)
        assert ns == 3600
        m = np.arange(1, n // 2 + 1)
        k = 2 * np.pi * m / n
        th = T.sk_axis(k, rho0, G, kT)
        sel = k >= 0.25
        for axis in (S[0, 1:n // 2 + 1], S[1:n // 2 + 1, 0]):
            ratios.append(axis[sel] / th[sel])
            ks.append(k[sel])
    assert nstable >= 30, nstable
    ratios, ks = np.concatenate(ratios), np.concatenate(ks)
    edges = np.arange(0.25, np.pi + 0.25, 0.25)
    chi = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        b = (ks >= lo) & (ks < hi)
        if b.sum() < 20:
            continue
        mean = ratios[b].mean()
        sem = ratios[b].std(ddof=1) / np.sqrt(b.sum())
        assert abs(mean - 1.0) <= max(0.02, 4 * sem), (lo, hi, mean, sem, int(b.sum()))
        chi.append(((mean - 1.0) / sem) ** 2)
    assert len(chi) >= 8 and np.mean(chi) < 2.0, chi
