"""Ensemble experiments on the static structure factor: S(k) of homogeneous
states approaching the spinodal along an isotherm (the metastable branches of
Fig. 2, top) and approaching the critical point along the binodal (Fig. 2,
bottom), and the long-wavelength limit S(k -> 0) whose scaling Fig. 3 shows.

All lattice work runs in liblbsc.so through one batched ensemble; the caller
supplies the state points (G, rho0).  S(0) is obtained from the axis modes by
the exact lattice form of the E4 structure factor, in which 1/S is linear in
(1 - cos k): a straight-line fit of 1/S against 1 - cos k over the lowest
relaxed modes gives 1/S(0) as its intercept.
"""
import numpy as np

from .ensemble import Ensemble


def axis_structure_factor(states, L=128, steps=30000, start=10000, seeds_per_state=32, kT=1e-6,
                          tau=1.0, stencil=4, seed=0, stream=None):
    """Run one ensemble with `seeds_per_state` replicas (distinct Philox
    replica indices) of each state (G, rho0) on an L x L lattice, sampling S(k)
    at every step from `start` on.  Returns (k, mean, sem): k = 2 pi m / L for
    m = 1 .. L/2, and per state the mean over replicas and both axes of S at
    those modes with its standard error ([nstates][L/2] each)."""
    reps = [(L, L, float(G), tau, kT, float(rho0)) for G, rho0 in states
            for _ in range(seeds_per_state)]
    e = Ensemble(reps, stencil=stencil, seed=seed, stream=stream)
    try:
        e.init(0.0)
        e.sk_config(1, start)
        e.step(steps)
        e.sync()
        m = L // 2
        mean, sem = [], []
        for i in range(len(states)):
            vals = []
            for r in range(i * seeds_per_state, (i + 1) * seeds_per_state):
                S, n = e.structure_factor(r)
                if n != steps - start + 1:
                    raise RuntimeError("unexpected number of S(k) samples")
                vals.append(S[0, 1:m + 1])     # k along x
                vals.append(S[1:m + 1, 0])     # k along y
            v = np.array(vals)
            mean.append(v.mean(axis=0))
            sem.append(v.std(axis=0, ddof=1) / np.sqrt(len(v)))
    finally:
        e.close()
    k = 2.0 * np.pi * np.arange(1, L // 2 + 1) / L
    return k, np.array(mean), np.array(sem)


def s0_from_axis(k, S, modes=slice(0, 8), sem=None):
    """S(k -> 0) from axis modes: weighted straight-line fit of 1/S against
    1 - cos k over `modes`; returns (S0, its standard error)."""
    x = 1.0 - np.cos(k[modes])
    y = 1.0 / S[modes]
    if sem is None:
        w = np.ones_like(y)
    else:
        w = (S[modes] ** 2 / sem[modes]) ** 2   # 1 / var(1/S)
    W = np.sum(w)
    xm, ym = np.sum(w * x) / W, np.sum(w * y) / W
    sxx = np.sum(w * (x - xm) ** 2)
    b = np.sum(w * (x - xm) * (y - ym)) / sxx
    a = ym - b * xm
    var_a = 1.0 / W + xm ** 2 / sxx
    return 1.0 / a, np.sqrt(var_a) / a ** 2


def power_law(x, y):
    """Exponent and prefactor of y = c x^p by least squares in log-log."""
    p, lc = np.polyfit(np.log(np.asarray(x, float)), np.log(np.asarray(y, float)), 1)
    return p, np.exp(lc)
