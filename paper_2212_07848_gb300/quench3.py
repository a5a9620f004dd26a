"""Unstable-branch quenches in three dimensions: the experiment of Fig. 1
(upper panels) of arXiv:2212.07848, where densities on the unstable part of
the T_hat = 0.8 isotherm phase-separate into droplets, cylinders, flat slabs,
bubble cylinders or bubbles in a periodic box.

`run_quench3` advances one D3Q19 lattice from a homogeneous density (with a
small Philox density kick and thermal noise) and classifies the final
morphology with `classify_topology3`: the minority phase's connected
components and the number of periodic directions each one wraps (0: droplet
or bubble, 1: cylinder, 2 or 3: flat slab).  The lattice work runs in
liblbsc.so; the classification is host-side analysis.
"""
from collections import deque

import numpy as np

from .lattice3 import Lattice3


def components3(mask):
    """Connected components of a periodic boolean field [nz][ny][nx]
    (6-neighbour).  Returns a list of (size, (wraps_x, wraps_y, wraps_z))."""
    nz, ny, nx = mask.shape
    seen = np.zeros(mask.shape, dtype=bool)
    unw = np.zeros(mask.shape + (3,), dtype=np.int64)   # unwrapped (x, y, z) of the first visit
    comps = []
    steps = ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))
    for z0, y0, x0 in zip(*np.nonzero(mask)):
        if seen[z0, y0, x0]:
            continue
        seen[z0, y0, x0] = True
        unw[z0, y0, x0] = (x0, y0, z0)
        q = deque([(z0, y0, x0)])
        size, wraps = 0, [False, False, False]
        while q:
            z, y, x = q.popleft()
            size += 1
            ux, uy, uz = unw[z, y, x]
            for dx, dy, dz in steps:
                xx, yy, zz = (x + dx) % nx, (y + dy) % ny, (z + dz) % nz
                if not mask[zz, yy, xx]:
                    continue
                p = (ux + dx, uy + dy, uz + dz)
                if seen[zz, yy, xx]:
                    u = unw[zz, yy, xx]
                    for a in range(3):
                        if u[a] != p[a]:
                            wraps[a] = True
                    continue
                seen[zz, yy, xx] = True
                unw[zz, yy, xx] = p
                q.append((zz, yy, xx))
        comps.append((size, tuple(wraps)))
    return comps


def classify_topology3(rho, threshold=None, min_contrast=0.2):
    """'droplet', 'droplet-cylinder', 'flat', 'bubble-cylinder', 'bubble',
    'mixed' or 'homogeneous' for a periodic 3D density field (liquid where
    rho > threshold; default: halfway between the 1st and 99th percentiles,
    and 'homogeneous' when those differ by less than min_contrast times the
    mean density).  The minority
    phase decides: with liquid minority no wrapping is a droplet and wrapping
    in one direction a droplet-cylinder; with gas minority the same give a
    bubble and a bubble-cylinder; wrapping in two or three directions is a
    flat slab.  Several minority components of different kinds are 'mixed'.
    Also returns the liquid fraction and the minority components."""
    rho = np.asarray(rho)
    if threshold is None:
        lo, hi = np.percentile(rho, [1.0, 99.0])
        if hi - lo < min_contrast * rho.mean():
            return "homogeneous", float("nan"), []
        threshold = 0.5 * (lo + hi)
    liquid = rho > threshold
    phi = float(liquid.mean())
    minority = liquid if phi <= 0.5 else ~liquid
    comps = components3(minority)
    if not comps:
        return "homogeneous", phi, comps
    big = [c for c in comps if c[0] >= 0.01 * minority.sum()]
    kinds = set()
    for _, w in big:
        nw = sum(w)
        kinds.add("flat" if nw >= 2 else ("cylinder" if nw == 1 else "sphere"))
    if len(kinds) > 1:
        return "mixed", phi, comps
    kind = kinds.pop()
    if kind == "flat":
        return "flat", phi, comps
    side = "droplet" if phi <= 0.5 else "bubble"
    return (side if kind == "sphere" else side + "-cylinder"), phi, comps


def run_quench3(n, G, rho0, kT=1e-7, steps=20000, seed=100, tau=1.0, psi_kind=0, psi_p1=0.0,
                psi_p2=0.0, init_amp=1e-3, precision="fp32", every=0, nbins=None):
    """Quench an n^3 lattice from rho0 (plus a density kick of amplitude
    init_amp) and return the final density, its topology, the liquid
    fraction and the mass drift; with `every` > 0 (n a power of two) also the
    instantaneous radial S(k, t) and the domain size L(t) = 2 pi sum S /
    sum |k| S of the full 3D S(k) every `every` steps."""
    lat = Lattice3(n, n, n, G, tau, kT, precision=precision, psi_kind=psi_kind, psi_p1=psi_p1,
                   psi_p2=psi_p2)
    lat.init(rho0, seed, init_amp)
    m0 = lat.conserved()[0]
    times, L, S = [], [], []
    if every > 0:
        nbins = nbins or int(np.ceil(np.sqrt(3.0) * n / 2)) + 1
        lat.sk_config(every, every)
        lat.sk_full()
        done = 0
        while done < steps:
            lat.step(every)
            done += every
            bins, _ = lat.structure_factor(nbins)
            times.append(done)
            S.append(bins)
            L.append(lat.domain_size())
            lat.sk_reset()
    else:
        lat.step(steps)
    lat.sync()
    rho = lat.density()
    m1 = lat.conserved()[0]
    lat.close()
    topo, phi, comps = classify_topology3(rho)
    out = {"density": rho, "topology": topo, "liquid_fraction": phi, "components": comps,
           "mass_drift": abs(m1 - m0) / m0}
    if every > 0:
        out.update(t=np.array(times), L=np.array(L), S=np.array(S))
    return out


# Eq. (5) at T_hat = 0.8: with the lattice temperature c_s^2 = 1/3 and G = -3
# the EoS p = rho/3 + (G/6) psi^2 is the paper's p = nT - psi^2/2, so
# T_c = (1/3)/0.8 = 5/12 with n_c = 1 (reduced density n_hat = rho).
EQ5_G, EQ5_TC, EQ5_NC = -3.0, 5.0 / 12.0, 1.0


def topology_sweep(densities, seeds, n=64, steps=10000, kT=1e-6, init_amp=1e-3):
    """The experiment of Fig. 1 (upper): quench each reduced density on the
    T_hat = 0.8 isotherm of Eq. (5) once per seed and count the final
    topologies.  Returns {density: {topology: count}} and, per density, the
    mean liquid fraction and the gas and liquid densities seen."""
    table = {}
    for nh in densities:
        counts, phis, lo, hi = {}, [], [], []
        for s in seeds:
            r = run_quench3(n, EQ5_G, nh * EQ5_NC, kT=kT, steps=steps, seed=s,
                            psi_kind=1, psi_p1=EQ5_TC, psi_p2=EQ5_NC, init_amp=init_amp)
            counts[r["topology"]] = counts.get(r["topology"], 0) + 1
            if r["topology"] != "homogeneous":
                phis.append(r["liquid_fraction"])
                a, b = np.percentile(r["density"], [1.0, 99.0])
                lo.append(a)
                hi.append(b)
        table[nh] = {"counts": counts,
                     "liquid_fraction": float(np.mean(phis)) if phis else None,
                     "rho_gas": float(np.mean(lo)) if lo else None,
                     "rho_liquid": float(np.mean(hi)) if hi else None}
    return table


def growth_run(n_hat, n=128, steps=20000, every=500, seed=1, kT=1e-6, init_amp=1e-3):
    """L(t) of one Eq. (5) quench at T_hat = 0.8 from the full 3D S(k); the
    growth exponent is the log-log slope over the last decade of t."""
    r = run_quench3(n, EQ5_G, n_hat * EQ5_NC, kT=kT, steps=steps, seed=seed, psi_kind=1,
                    psi_p1=EQ5_TC, psi_p2=EQ5_NC, init_amp=init_amp, every=every)
    t, L = r["t"], r["L"]
    sel = t >= t[-1] / 10
    slope = float(np.polyfit(np.log(t[sel]), np.log(L[sel]), 1)[0])
    return {"n_hat": n_hat, "n": n, "seed": seed, "topology": r["topology"],
            "L": {str(int(tt)): float(LL) for tt, LL in zip(t, L)
                  if int(tt) in (500, 1000, 2000, 5000, 10000, 20000)},
            "exponent_last_decade": slope, "mass_drift": r["mass_drift"]}


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="3D unstable-branch quench topologies (Fig. 1)")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--seeds", type=int, default=6)
    ap.add_argument("--densities", default="0.65,0.7,0.75,0.8,0.85,0.9,0.95,1.0,1.15,1.3,1.45,"
                                           "1.5,1.55,1.6,1.62,1.64,1.66")
    ap.add_argument("--growth", action="store_true",
                    help="L(t) from the full 3D S(k) instead of the topology sweep")
    ap.add_argument("--every", type=int, default=500)
    a = ap.parse_args()
    dens = [float(x) for x in a.densities.split(",")]
    if a.growth:
        for nh in dens:
            for s in range(1, a.seeds + 1):
                print(json.dumps(growth_run(nh, n=a.n, steps=a.steps, every=a.every, seed=s)),
                      flush=True)
    else:
        res = topology_sweep(dens, range(1, a.seeds + 1), n=a.n, steps=a.steps)
        for nh, r in res.items():
            print(json.dumps({"n_hat": nh, **r}), flush=True)
