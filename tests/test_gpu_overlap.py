"""The overlapped-strip step kernel (strips of 128 - 2H columns, halo columns
pulled by the CTA's own threads, no halo warp) against the halo-warp kernel
(same arithmetic, so the same bits) and against the oracle."""
import numpy as np
import pytest

from pairs import LN2, make_pair, max_rel

pytestmark = pytest.mark.gpu


def _lattice(nx, ny, G, tau, kT, stencil, kernel, precision="fp32", strip=None, sk=0,
             tau_bulk=0.0):
    from paper_2212_07848_gb300.lattice import Lattice
    g = Lattice(nx, ny, G, tau, kT, stencil=stencil, precision=precision, tau_bulk=tau_bulk)
    g.set_kernel(kernel)
    if strip:
        g.set_strip_height(strip)
    g.init(LN2, 33, 0.01)
    if sk:
        g.sk_config(sk, sk)
    return g


@pytest.mark.parametrize("nx,ny,G,tau,kT,stencil,precision,strip,sk,tb", [
    (128, 64, -3.6, 1.0, 1e-5, 4, "fp32", None, 0, 0.0),     # two strips (126 + 2 columns)
    (4096, 32, -5.0, 1.0, 1e-6, 4, "fp32", 8, 5, 0.0),      # benchmark width, sampling
    (252, 36, -4.5, 0.8, 1e-5, 6, "fp32", 8, 0, 0.0),       # reach 2: exactly two strips
    (260, 20, -3.6, 1.3, 1e-5, 8, "fp32", 4, 0, 0.0),       # E8, ragged last strip
    (12, 8, -3.6, 0.9, 1e-5, 4, "fp32", None, 0, 1.2),      # narrower than one strip, MRT
    (4, 4, -3.6, 1.0, 1e-5, 6, "fp32", None, 0, 0.0),       # halo wider than half the lattice
    (132, 36, -3.6, 0.9, 1e-5, 4, "fp64", 8, 0, 0.0),       # FP64
])
def test_overlap_kernel_matches_halo_warp_kernel(nx, ny, G, tau, kT, stencil, precision, strip,
                                                 sk, tb):
    from paper_2212_07848_gb300 import abi
    a = _lattice(nx, ny, G, tau, kT, stencil, abi.LB_KERNEL_OVERLAP, precision, strip, sk, tb)
    b = _lattice(nx, ny, G, tau, kT, stencil, abi.LB_KERNEL_PLAIN, precision, strip, sk, tb)
    assert a.kernel == abi.LB_KERNEL_OVERLAP and b.kernel == abi.LB_KERNEL_PLAIN
    a.step(30)
    b.step(30)
    a.sync()
    b.sync()
    da, db = a.download_state(), b.download_state()
    assert np.array_equal(da, db), np.abs(da - db).max()
    if sk:
        sa, na = a.structure_factor()
        sb, nb = b.structure_factor()
        assert na == nb == 6 and np.array_equal(sa, sb)


def test_overlap_kernel_matches_oracle():
    from paper_2212_07848_gb300 import abi
    g, o = make_pair(260, 68, -4.5, 1.0, 1e-6, precision="fp32", rho0=0.33, seed=4, amp=0.005)
    g.set_kernel(abi.LB_KERNEL_OVERLAP)
    g.step(100)
    o.step(100)
    assert max_rel(g.populations(), o.populations()) < 1e-4
    assert max_rel(g.density(), o.density()) < 1e-4
