"""GB300 (sm_103a) fluctuating Shan-Chen D2Q9 lattice Boltzmann library.

Method of Lulli et al., "Metastable and Unstable Dynamics in multi-phase
lattice Boltzmann" (arXiv:2212.07848).  The hot path -- the fused time step
and the on-device structure factor -- lives in liblbsc.so (CUDA, C ABI in
include/lbsc.h); `abi` binds it with ctypes under the same names and
`Lattice` wraps one context.  Importing the package does not load the
library; the first call does, and fails loudly if it is missing.
"""
from . import abi  # noqa: F401


def __getattr__(name):
    if name == "Lattice":
        from .lattice import Lattice
        return Lattice
    raise AttributeError(name)
