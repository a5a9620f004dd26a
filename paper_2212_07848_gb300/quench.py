"""Unstable-branch quench: phase separation after an instantaneous quench
into the unstable region (the experiment behind Fig. 1's upper panels of
arXiv:2212.07848, here in two dimensions).

`run_quench` advances one lattice from a homogeneous density with thermal
noise and records, every `every` steps, the instantaneous radial S(k, t)
and the domain size L(t) = 2 pi sum_k S / sum_k |k| S (a definition of this
library; the paper gives none).  `classify_topology` names the final
morphology of a periodic density field: droplets (liquid minority, no
component wrapping the box), stripes (a component that wraps in one
direction: a flat slab in 2D) or bubbles (gas minority, no wrapping).  The
lattice work runs in liblbsc.so; the classification is host-side analysis.
"""
from collections import deque

import numpy as np

from .lattice import Lattice


def _components(mask):
    """Connected components of a periodic boolean field (4-neighbour).
    Returns a list of (size, wraps_x, wraps_y)."""
    ny, nx = mask.shape
    seen = np.zeros(mask.shape, dtype=bool)
    # unwrapped coordinates of the first visit of each cell
    ux = np.zeros(mask.shape, dtype=np.int64)
    uy = np.zeros(mask.shape, dtype=np.int64)
    comps = []
    for y0, x0 in zip(*np.nonzero(mask)):
        if seen[y0, x0]:
            continue
        seen[y0, x0] = True
        ux[y0, x0], uy[y0, x0] = x0, y0
        q = deque([(y0, x0)])
        size, wx, wy = 0, False, False
        while q:
            y, x = q.popleft()
            size += 1
            for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                yy, xx = (y + dy) % ny, (x + dx) % nx
                if not mask[yy, xx]:
                    continue
                px, py = ux[y, x] + dx, uy[y, x] + dy
                if seen[yy, xx]:
                    if ux[yy, xx] != px:
                        wx = True
                    if uy[yy, xx] != py:
                        wy = True
                    continue
                seen[yy, xx] = True
                ux[yy, xx], uy[yy, xx] = px, py
                q.append((yy, xx))
        comps.append((size, wx, wy))
    return comps


def classify_topology(rho, threshold):
    """'droplet', 'stripe', 'bubble' or 'mixed' for a periodic 2D density
    field, liquid where rho > threshold; also returns the liquid fraction and
    the component list of the minority phase."""
    liquid = rho > threshold
    phi = float(liquid.mean())
    minority = liquid if phi <= 0.5 else ~liquid
    comps = _components(minority)
    if not comps:
        return "homogeneous", phi, comps
    wrap = [c for c in comps if c[1] or c[2]]
    if wrap:
        one_dir = all((c[1] != c[2]) for c in wrap)
        return ("stripe" if one_dir else "mixed"), phi, comps
    return ("droplet" if phi <= 0.5 else "bubble"), phi, comps


def run_quench(nx, ny, G, rho0, kT=1e-6, steps=50000, every=500, seed=100, tau=1.0,
               stencil=4, nbins=None, init_amp=0.0, precision="fp32"):
    """Quench a homogeneous lattice and record S(k, t) and L(t) every `every`
    steps.  Returns a dict with times, L, radial S (rows = samples), the
    final density and its topology classification."""
    lat = Lattice(nx, ny, G, tau, kT, stencil=stencil, precision=precision)
    lat.init(rho0, seed, init_amp)
    lat.sk_config(0, 0)
    nbins = nbins or max(nx, ny) // 2
    times, L, S = [], [], []
    done = 0
    while done < steps:
        n = min(every, steps - done)
        lat.step(n)
        done += n
        lat.sk_reset()
        lat.sk_sample_now()
        bins, _ = lat.structure_factor(nbins)
        times.append(done)
        S.append(bins)
        L.append(lat.domain_size())
    rho = lat.density()
    lat.close()
    topo, phi, comps = classify_topology(rho, threshold=rho0)
    return {"t": np.array(times), "L": np.array(L), "S": np.array(S), "density": rho,
            "topology": topo, "liquid_fraction": phi, "components": comps}


def growth_exponent(t, L, t_min):
    """Least-squares slope of log L against log t over t >= t_min."""
    t, L = np.asarray(t, float), np.asarray(L, float)
    sel = t >= t_min
    return float(np.polyfit(np.log(t[sel]), np.log(L[sel]), 1)[0])


def block_mean(field, b):
    """b x b block means of a 2D field (for classifying large lattices)."""
    ny, nx = field.shape
    return field.reshape(ny // b, b, nx // b, b).mean(axis=(1, 3))


if __name__ == "__main__":
    import argparse
    import json
    import math
    ap = argparse.ArgumentParser(description="2D unstable-branch quenches: S(k,t), L(t), topology")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--G", type=float, default=-5.0)
    ap.add_argument("--steps", type=int, default=50000)
    ap.add_argument("--every", type=int, default=500)
    ap.add_argument("--seeds", default="100,101")
    ap.add_argument("--rho0", default=f"{math.log(2.0)},0.422",
                    help="the critical density and a 15%% liquid-fraction state at G = -5")
    ap.add_argument("--block", type=int, default=4, help="block mean before classification")
    ap.add_argument("--out", default=None, help="npz with t, L and S(k, t) of every run")
    a = ap.parse_args()
    saved = {}
    for rho0 in [float(r) for r in a.rho0.split(",")]:
        for seed in [int(s) for s in a.seeds.split(",")]:
            r = run_quench(a.n, a.n, a.G, rho0, steps=a.steps, every=a.every, seed=seed)
            coarse = block_mean(r["density"], a.block) if a.block > 1 else r["density"]
            topo, phi, _ = classify_topology(coarse, rho0)
            lo, hi = np.percentile(r["density"], [1.0, 99.0])
            t, L = r["t"], r["L"]
            line = {"n": a.n, "G": a.G, "rho0": rho0, "seed": seed, "topology": topo,
                    "liquid_fraction": phi, "rho_gas": float(lo), "rho_liquid": float(hi),
                    "L": {str(int(tt)): float(LL) for tt, LL in zip(t, L)
                          if int(tt) in (1000, 2000, 5000, 10000, 20000, 50000)},
                    "exponent_t_ge_5000": growth_exponent(t, L, 5000),
                    "exponent_t_ge_20000": growth_exponent(t, L, 20000)}
            print(json.dumps(line), flush=True)
            key = f"rho{rho0:.4f}_s{seed}"
            saved[key + "_t"], saved[key + "_L"], saved[key + "_S"] = t, L, r["S"][:, :512]
    if a.out:
        np.savez(a.out, **saved)
