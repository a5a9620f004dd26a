"""Build a GPU lattice and an oracle lattice from the same parameters."""
import numpy as np

from oracle import oracle as O

LN2 = float(np.log(2.0))


def make_pair(nx, ny, G, tau, kT, stencil=4, kind=0, p1=0.0, p2=0.0, precision="fp64",
              rho0=LN2, seed=0, amp=0.0, replica=0, strip=None, tau_bulk=0.0, tau_ghost=0.0):
    from paper_2212_07848_gb300.lattice import Lattice
    g = Lattice(nx, ny, G, tau, kT, psi_kind=kind, stencil=stencil, precision=precision,
                psi_p1=p1, psi_p2=p2, tau_bulk=tau_bulk, tau_ghost=tau_ghost)
    if strip:
        g.set_strip_height(strip)
    g.set_replica(replica)
    g.init(rho0, seed, amp)
    o = O.OracleLattice(nx, ny, G, tau, kT, psi_kind=kind, stencil=stencil, psi_p1=p1,
                        psi_p2=p2, replica=replica, tau_bulk=tau_bulk, tau_ghost=tau_ghost)
    o.init(rho0, seed, amp)
    return g, o


def max_rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))
