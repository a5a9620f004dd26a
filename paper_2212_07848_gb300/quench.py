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
