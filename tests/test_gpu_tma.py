"""The bulk-tensor-copy step kernel against the plain-load kernel (same
arithmetic, so the same bits) and against the oracle; kernel selection."""
import numpy as np
import pytest

from pairs import LN2, make_pair, max_rel

pytestmark = pytest.mark.gpu


def _lattice(nx, ny, G, tau, kT, stencil, kernel, strip=None, sk=0):
    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.lattice import Lattice
    g = Lattice(nx, ny, G, tau, kT, stencil=stencil, precision="fp32")
    g.set_kernel(kernel)
    if strip:
        g.set_strip_height(strip)
    g.init(LN2, 21, 0.01)
    if sk:
        g.sk_config(sk, sk)
    return g


@pytest.mark.parametrize("nx,ny,G,tau,kT,stencil,strip,sk", [
    (128, 64, -3.6, 1.0, 1e-5, 4, None, 0),    # one strip: both periodic edges
    (256, 36, -4.5, 0.8, 1e-5, 6, 8, 0),       # ragged last row strip, reach 2
    (384, 20, -3.6, 1.3, 1e-5, 8, 4, 0),       # three strips, E8
    (512, 128, -5.0, 1.0, 1e-6, 4, None, 5),   # sampling steps write delta rho
])
def test_tma_kernel_matches_plain_kernel(nx, ny, G, tau, kT, stencil, strip, sk):
    from paper_2212_07848_gb300 import abi
    a = _lattice(nx, ny, G, tau, kT, stencil, abi.LB_KERNEL_TMA, strip, sk)
    b = _lattice(nx, ny, G, tau, kT, stencil, abi.LB_KERNEL_PLAIN, strip, sk)
    assert a.kernel == abi.LB_KERNEL_TMA and b.kernel == abi.LB_KERNEL_PLAIN
    a.step(50)
    b.step(50)
    a.sync()
    b.sync()
    da, db = a.download_state(), b.download_state()
    assert np.array_equal(da, db), np.abs(da - db).max()
    if sk:
        sa, na = a.structure_factor()
        sb, nb = b.structure_factor()
        assert na == nb == 10 and np.array_equal(sa, sb)


def test_tma_kernel_matches_oracle():
    from paper_2212_07848_gb300 import abi
    g, o = make_pair(256, 64, -4.5, 1.0, 1e-6, precision="fp32", rho0=0.33, seed=4, amp=0.005)
    g.set_kernel(abi.LB_KERNEL_TMA)
    g.step(100)
    o.step(100)
    assert max_rel(g.populations(), o.populations()) < 1e-4
    assert max_rel(g.density(), o.density()) < 1e-4


def test_kernel_selection():
    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.lattice import Lattice
    assert Lattice(256, 64, -3.6).kernel == abi.LB_KERNEL_PLAIN      # auto, narrow
    assert Lattice(1024, 8, -3.6).kernel == abi.LB_KERNEL_OVERLAP    # auto, wide
    t = Lattice(256, 64, -3.6)
    t.set_kernel(abi.LB_KERNEL_TMA)
    assert t.kernel == abi.LB_KERNEL_TMA
    t.set_kernel(abi.LB_KERNEL_OVERLAP)
    assert t.kernel == abi.LB_KERNEL_OVERLAP
    t.set_kernel(abi.LB_KERNEL_PLAIN)
    assert t.kernel == abi.LB_KERNEL_PLAIN
    assert Lattice(132, 64, -3.6).kernel == abi.LB_KERNEL_PLAIN
    assert Lattice(1024, 8, -3.6, precision="fp64").kernel == abi.LB_KERNEL_OVERLAP
    g = Lattice(132, 64, -3.6)
    with pytest.raises(abi.LbError) as e:
        g.set_kernel(abi.LB_KERNEL_TMA)
    assert e.value.code == abi.LB_ERR_UNSUPPORTED
