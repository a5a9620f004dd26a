"""Seeded synthetic inputs shared by the CUDA path's tests and the oracle.

This module holds no arithmetic of the method: it only draws seeded random
numbers and builds density fields of the shapes the paper's experiments use
(homogeneous boxes with small perturbations, flat slabs, droplets).  Both
sides convert a density field into populations with their own code.
"""
import numpy as np

LN2 = float(np.log(2.0))


def rng(seed):
    return np.random.default_rng(int(seed))


def random_populations(nx, ny, seed, lo=0.05, hi=0.2):
    """Arbitrary positive populations, [9][ny][nx] float64 (a non-equilibrium state)."""
    return rng(seed).uniform(lo, hi, size=(9, ny, nx))


def perturbed_density(nx, ny, rho0, amp, seed):
    """rho0 + amp * N(0, 1) per site, [ny][nx]."""
    return rho0 + amp * rng(seed).standard_normal((ny, nx))


def sinusoid_density(nx, ny, rho0, amp, mx, my):
    """rho0 + amp * sin(2 pi (mx x / nx + my y / ny)), [ny][nx]."""
    y, x = np.mgrid[0:ny, 0:nx]
    return rho0 + amp * np.sin(2.0 * np.pi * (mx * x / nx + my * y / ny))


def slab_density(nx, ny, rho_gas, rho_liq, width, smooth=2.0):
    """A liquid slab of the given width centred in x, flat in y (two flat
    interfaces, periodic), tanh profiles of thickness `smooth`."""
    x = np.arange(nx) + 0.5
    c = nx / 2.0
    d = np.abs(x - c) - width / 2.0
    prof = rho_gas + 0.5 * (rho_liq - rho_gas) * (1.0 - np.tanh(d / smooth))
    return np.tile(prof, (ny, 1))


def droplet_density(nx, ny, radius, rho_in, rho_out, smooth=2.0):
    """A circular droplet of the given radius centred in the box."""
    y, x = np.mgrid[0:ny, 0:nx]
    r = np.hypot(x + 0.5 - nx / 2.0, y + 0.5 - ny / 2.0)
    return rho_out + 0.5 * (rho_in - rho_out) * (1.0 - np.tanh((r - radius) / smooth))


# Workloads of the kind the paper simulates (periodic boxes, homogeneous
# initial density, thermal noise).  Sizes and couplings as named.
WORKLOADS = {
    "d2q9_128sq_fp64_G-3.6": dict(nx=128, ny=128, precision="fp64", G=-3.6, tau=1.0,
                                  kT=1e-5, rho0=LN2, psi_kind=0, stencil=4, seed=0,
                                  steps=2000, sk_every=1, sk_start=1001),
    "d2q9_1024sq_fp32_G-4.5": dict(nx=1024, ny=1024, precision="fp32", G=-4.5, tau=1.0,
                                   kT=1e-6, psi_kind=0, stencil=4, seeds=list(range(1, 17)),
                                   steps=100000, sk_every=100, sk_start=20000),
    "d2q9_4096sq_fp32_G-5.0_quench": dict(nx=4096, ny=4096, precision="fp32", G=-5.0,
                                          tau=1.0, kT=1e-6, rho0=LN2, psi_kind=0,
                                          stencil=4, seed=100, steps=50000, sk_every=500,
                                          sk_start=500),
}
