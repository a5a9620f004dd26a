"""Lattice: a convenience wrapper over the C ABI (one periodic D2Q9 lattice).

The object owns one library context.  PyTorch supplies the CUDA stream when
one is given and can view the library's device buffers without a copy;
all lattice arithmetic runs in liblbsc.so.
"""
import ctypes as C

import numpy as np

from . import abi


class Lattice:
    """Fluctuating Shan-Chen D2Q9 lattice on one GPU.

    Parameters follow lb_params (include/lbsc.h): nx, ny (multiples of 4),
    G (< 0 attractive), tau (> 1/2), kT (>= 0), psi_kind (0: 1-exp(-rho);
    1: sqrt(Tc nc) exp(1-nc/rho); 2: a exp(-b/rho)), psi_p1/psi_p2, stencil
    (4, 6, 8), precision ("fp32" or "fp64"), stream (an int cudaStream_t,
    e.g. torch.cuda.current_stream().cuda_stream), device, tau_bulk and
    tau_ghost (0: equal to tau, the BGK collision).
    """

    def __init__(self, nx, ny, G, tau=1.0, kT=0.0, psi_kind=0, stencil=4,
                 precision="fp32", psi_p1=0.0, psi_p2=0.0, stream=None, device=-1,
                 tau_bulk=0.0, tau_ghost=0.0):
        p = abi.lb_params_init()
        p.nx, p.ny, p.G, p.tau, p.kT = nx, ny, G, tau, kT
        p.tau_bulk, p.tau_ghost = tau_bulk, tau_ghost
        p.psi_kind, p.psi_p1, p.psi_p2, p.stencil = psi_kind, psi_p1, psi_p2, stencil
        p.precision = abi.LB_FP32 if precision in ("fp32", abi.LB_FP32) else abi.LB_FP64
        p.stream = stream
        p.device = device
        self.nx, self.ny = nx, ny
        self.precision = "fp32" if p.precision == abi.LB_FP32 else "fp64"
        self.dtype = np.float32 if self.precision == "fp32" else np.float64
        self._h = abi.lb_create_ex(p)

    def close(self):
        if getattr(self, "_h", None):
            abi.lb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def init(self, rho0, seed=0, init_amp=0.0):
        abi.lb_init(self._h, rho0, seed, init_amp)

    def set_replica(self, r):
        abi.lb_set_replica(self._h, r)

    def step(self, n=1):
        abi.lb_step(self._h, n)

    def sync(self):
        abi.lb_sync(self._h)

    @property
    def t(self):
        return abi.lb_get_step(self._h)

    def density(self):
        out = np.empty(self.nx * self.ny)
        abi.lb_density(self._h, out)
        return out.reshape(self.ny, self.nx)

    def populations(self):
        out = np.empty(9 * self.nx * self.ny)
        abi.lb_populations(self._h, out)
        return out.reshape(9, self.ny, self.nx)

    def set_populations(self, f):
        abi.lb_set_populations(self._h, f)

    def set_density(self, rho):
        abi.lb_set_density(self._h, rho)

    def download_state(self, out=None):
        """Raw deviations [9][ny][nx] in the storage precision."""
        if out is None:
            out = np.empty((9, self.ny, self.nx), self.dtype)
        assert out.dtype == self.dtype and out.flags.c_contiguous and out.size == 9 * self.nx * self.ny
        abi.lb_download_state(self._h, out.ctypes.data_as(C.c_void_p))
        return out

    def upload_state(self, df):
        assert df.dtype == self.dtype and df.flags.c_contiguous and df.size == 9 * self.nx * self.ny
        abi.lb_upload_state(self._h, df.ctypes.data_as(C.c_void_p))

    def sk_config(self, every, start):
        abi.lb_sk_config(self._h, every, start)

    def sk_reset(self):
        abi.lb_sk_reset(self._h)

    def sk_sample_now(self):
        abi.lb_sk_sample_now(self._h)

    def structure_factor(self, nbins=0):
        """(S, nsamples): S is [ny][nx/2+1] for nbins == 0, else [nbins] radial means."""
        if nbins == 0:
            out = np.empty(self.ny * (self.nx // 2 + 1))
            out, n = abi.lb_structure_factor(self._h, out, 0)
            return out.reshape(self.ny, self.nx // 2 + 1), n
        out = np.empty(nbins)
        return abi.lb_structure_factor(self._h, out, nbins)

    def sk_moments(self):
        """(sum_k S, sum_k |k| S) of the mean S(k), k = 0 excluded."""
        return abi.lb_sk_moments(self._h)

    def domain_size(self):
        """L = 2 pi sum S / sum |k| S (this library's definition)."""
        m = self.sk_moments()
        return 2.0 * 3.141592653589793 * m[0] / m[1]

    def structure_factor_counts(self, nbins):
        return abi.lb_structure_factor_counts(self._h, nbins)

    def conserved(self):
        return abi.lb_conserved(self._h)

    def save(self, path):
        abi.lb_save(self._h, path)

    def load(self, path):
        abi.lb_load(self._h, path)

    def set_strip_height(self, rows):
        abi.lb_set_strip_height(self._h, rows)

    def set_kernel(self, mode):
        """abi.LB_KERNEL_AUTO / LB_KERNEL_PLAIN / LB_KERNEL_TMA / LB_KERNEL_OVERLAP."""
        abi.lb_set_kernel(self._h, mode)

    @property
    def kernel(self):
        return abi.lb_get_kernel(self._h)

    def device_ptr(self, which=abi.LB_PTR_POPULATIONS):
        return abi.lb_device_ptr(self._h, which)

    def stream(self):
        return abi.lb_stream(self._h)

    def torch_populations(self):
        """Zero-copy torch view of the current deviations [9][ny][nx] (valid until
        the next step swaps the buffers)."""
        import torch

        class _View:
            pass

        v = _View()
        v.__cuda_array_interface__ = {
            "shape": (9, self.ny, self.nx),
            "typestr": "<f4" if self.precision == "fp32" else "<f8",
            "data": (self.device_ptr(abi.LB_PTR_POPULATIONS), False),
            "version": 3,
            "strides": None,
        }
        return torch.as_tensor(v, device="cuda")
