"""Ensemble: many replicas of uneven size, coupling and density advanced
together on one GPU (a wrapper over the lb_ens_* calls of the C ABI)."""
import numpy as np

from . import abi


class Ensemble:
    """reps: list of (nx, ny, G, tau, kT, rho0).  Replica r draws its noise
    from key `seed`, counter word 2 = r (the same stream as a Lattice with
    that seed and set_replica(r))."""

    def __init__(self, reps, psi_kind=0, psi_p1=0.0, psi_p2=0.0, stencil=4, seed=0,
                 stream=None):
        self.reps = [tuple(r) for r in reps]
        self._h = abi.lb_ens_create(self.reps, psi_kind, psi_p1, psi_p2, stencil, seed, stream)

    def close(self):
        if getattr(self, "_h", None):
            abi.lb_ens_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.reps)

    def init(self, init_amp=0.0):
        abi.lb_ens_init(self._h, init_amp)

    def sk_config(self, every, start):
        abi.lb_ens_sk_config(self._h, every, start)

    def set_launch(self, mode):
        """abi.LB_ENS_PER_STEP or abi.LB_ENS_PERSISTENT."""
        abi.lb_ens_set_launch(self._h, mode)

    @property
    def launch(self):
        return abi.lb_ens_get_launch(self._h)

    def set_kernel(self, mode):
        """Strip layout: abi.LB_KERNEL_AUTO / LB_KERNEL_PLAIN / LB_KERNEL_OVERLAP."""
        abi.lb_ens_set_kernel(self._h, mode)

    @property
    def kernel(self):
        return abi.lb_ens_get_kernel(self._h)

    def set_resident(self, mode):
        """Shared-memory-resident replicas: abi.LB_ENS_RESIDENT_OFF / _ON / _AUTO."""
        abi.lb_ens_set_resident(self._h, mode)

    @property
    def num_resident(self):
        return abi.lb_ens_num_resident(self._h)

    def set_strip_height(self, rows):
        abi.lb_ens_set_strip_height(self._h, rows)

    def autotune(self, trial_steps=20, cache_path=None):
        return abi.lb_ens_autotune(self._h, trial_steps, cache_path)

    def step(self, n=1):
        abi.lb_ens_step(self._h, n)

    def sync(self):
        abi.lb_ens_sync(self._h)

    @property
    def t(self):
        return abi.lb_ens_get_step(self._h)

    @property
    def num_tiles(self):
        return abi.lb_ens_num_tiles(self._h)

    def populations(self, r):
        nx, ny = self.reps[r][:2]
        out = np.empty(9 * nx * ny)
        return abi.lb_ens_populations(self._h, r, out).reshape(9, ny, nx)

    def density(self, r):
        nx, ny = self.reps[r][:2]
        out = np.empty(nx * ny)
        return abi.lb_ens_density(self._h, r, out).reshape(ny, nx)

    def conserved(self, r):
        return abi.lb_ens_conserved(self._h, r)

    def structure_factor(self, r, nbins=0):
        nx, ny = self.reps[r][:2]
        if nbins == 0:
            out = np.empty(ny * (nx // 2 + 1))
            out, n = abi.lb_ens_structure_factor(self._h, r, out, 0)
            return out.reshape(ny, nx // 2 + 1), n
        return abi.lb_ens_structure_factor(self._h, r, np.empty(nbins), nbins)
