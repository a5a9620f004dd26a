"""Lattice3: a convenience wrapper over the D3Q19 part of the C ABI (one
periodic three-dimensional lattice on one GPU; all arithmetic in liblbsc.so)."""
import ctypes as C

import numpy as np

from . import abi


class Lattice3:
    """Fluctuating Shan-Chen D3Q19 lattice: nx (multiple of 32), ny (multiple
    of 8), nz (>= 3), G (< 0 attractive), tau (> 1/2), kT (>= 0), precision
    "fp32" or "fp64", stream (an int cudaStream_t or None), pseudopotential
    psi_kind with psi_p1, psi_p2 as for the 2D lattice."""

    def __init__(self, nx, ny, nz, G, tau=1.0, kT=0.0, precision="fp32", stream=None,
                 psi_kind=0, psi_p1=0.0, psi_p2=0.0):
        L = abi.load()
        self.nx, self.ny, self.nz = nx, ny, nz
        h = C.c_void_p()
        prec = abi.LB_FP32 if precision == "fp32" else abi.LB_FP64
        rc = L.lb3_create(C.byref(h), nx, ny, nz, G, tau, kT, prec,
                          C.c_void_p(stream) if stream else None)
        if rc != 0:
            raise abi.LbError(rc, "lb3_create")
        self._h = h
        if psi_kind:
            self._ck(L.lb3_set_psi(h, psi_kind, psi_p1, psi_p2), "lb3_set_psi")

    def close(self):
        if getattr(self, "_h", None):
            abi.load().lb3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc, what):
        if rc != 0:
            raise abi.LbError(rc, what)

    def init(self, rho0, seed=0, init_amp=0.0):
        self._ck(abi.load().lb3_init(self._h, rho0, seed, init_amp), "lb3_init")

    def set_replica(self, r):
        self._ck(abi.load().lb3_set_replica(self._h, r), "lb3_set_replica")

    def set_strip(self, planes):
        self._ck(abi.load().lb3_set_strip(self._h, planes), "lb3_set_strip")

    def step(self, n=1):
        self._ck(abi.load().lb3_step(self._h, int(n)), "lb3_step")

    def sync(self):
        self._ck(abi.load().lb3_sync(self._h), "lb3_sync")

    @property
    def t(self):
        return abi.load().lb3_get_step(self._h)

    def density(self):
        out = np.empty(self.nx * self.ny * self.nz)
        self._ck(abi.load().lb3_density(self._h, out), "lb3_density")
        return out.reshape(self.nz, self.ny, self.nx)

    def populations(self):
        out = np.empty(19 * self.nx * self.ny * self.nz)
        self._ck(abi.load().lb3_populations(self._h, out), "lb3_populations")
        return out.reshape(19, self.nz, self.ny, self.nx)

    def set_populations(self, f):
        f = np.ascontiguousarray(f, np.float64).ravel()
        self._ck(abi.load().lb3_set_populations(self._h, f), "lb3_set_populations")

    def conserved(self):
        out = np.zeros(4)
        self._ck(abi.load().lb3_conserved(self._h, out), "lb3_conserved")
        return out

    def sk_config(self, every, start):
        self._ck(abi.load().lb3_sk_config(self._h, int(every), int(start)), "lb3_sk_config")

    def sk_reset(self):
        self._ck(abi.load().lb3_sk_reset(self._h), "lb3_sk_reset")

    def structure_factor_axes(self):
        """(S on the x, y and z axes [nx/2 + ny/2 + nz/2], nsamples)."""
        out = np.empty(self.nx // 2 + self.ny // 2 + self.nz // 2)
        n = C.c_longlong(0)
        self._ck(abi.load().lb3_structure_factor_axes(self._h, out, C.byref(n)),
                 "lb3_structure_factor_axes")
        return out, n.value

    def sk_full(self, enable=True):
        """Accumulate the full 3D S(k) on the sampling steps of sk_config
        (power-of-two sizes)."""
        self._ck(abi.load().lb3_sk_full(self._h, 1 if enable else 0), "lb3_sk_full")

    def structure_factor(self, nbins):
        """(radial means of the full S(k) [nbins], nsamples)."""
        out = np.empty(nbins)
        n = C.c_longlong(0)
        self._ck(abi.load().lb3_structure_factor(self._h, out, int(nbins), C.byref(n)),
                 "lb3_structure_factor")
        return out, n.value

    def sk_moments(self):
        """(sum_k S, sum_k |k| S) of the mean full S(k), k != 0."""
        out = np.empty(2)
        self._ck(abi.load().lb3_sk_moments(self._h, out), "lb3_sk_moments")
        return out

    def domain_size(self):
        """L = 2 pi sum_k S / sum_k |k| S of the mean full S(k)."""
        m = self.sk_moments()
        return float(2.0 * np.pi * m[0] / m[1]) if m[1] > 0 else float("nan")
