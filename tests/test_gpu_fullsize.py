"""Full-size check at the benchmark's lattice (4096^2, FP32, G = -5.0 critical
quench, kT = 1e-6) in the benchmark's launch configuration: one GPU step is
compared with the oracle evaluated site by site on the same input state
(random sites plus every kind of strip and wrap boundary), and mass and
momentum are checked over the run."""
import numpy as np
import pytest

from oracle import oracle as O
from pairs import LN2

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def test_fullsize_4096_one_step_sampled_sites():
    from paper_2212_07848_gb300.lattice import Lattice
    nx = ny = 4096
    G, tau, kT, seed = -5.0, 1.0, 1e-6, 100
    from paper_2212_07848_gb300 import abi
    g = Lattice(nx, ny, G, tau, kT)
    assert g.kernel == abi.LB_KERNEL_OVERLAP          # the kernel the benchmark times
    g.init(LN2, seed, 0.01)
    c0 = g.conserved()
    g.step(3)
    df_in = g.download_state().copy()
    g.step(1)
    df_out = g.download_state()
    c1 = g.conserved()
    assert abs(c1[0] - c0[0]) / c0[0] < 1e-6
    assert abs(c1[1] - c0[1]) < 1e-6 * c0[0] and abs(c1[2] - c0[2]) < 1e-6 * c0[0]

    rng = np.random.default_rng(1)
    xs = list(rng.integers(0, nx, 3000))
    ys = list(rng.integers(0, ny, 3000))
    # strip boundaries of both layouts: 128-column strips (halo warp) and
    # 126-column strips (overlapped, the automatic choice; the last strip
    # starts at 32 x 126 = 4032), and row strips of 32
    edge_x = [0, 1, 2, nx - 3, nx - 2, nx - 1, 125, 126, 127, 128, 129, 251, 252, 255, 256,
              2047, 2048, 4031, 4032, 4033]
    edge_y = [0, 1, 2, ny - 3, ny - 2, ny - 1, 31, 32, 33, 63, 64, 65, 127, 128, 2047, 2048]
    for ex in edge_x:
        for ey in edge_y:
            xs.append(ex)
            ys.append(ey)
    xs = np.array(xs, np.int32)
    ys = np.array(ys, np.int32)

    f_in = df_in.astype(np.float64)
    f_in += (W * LN2)[:, None, None]
    p = O.make_params(nx, ny, G, tau, kT, stencil=4, rho0=LN2, seed=seed)
    ref = O.step_sites(p, 3, f_in, xs, ys)                 # [n][9] full populations
    got = df_out[:, ys, xs].T.astype(np.float64) + W * LN2
    rel = np.abs(got - ref) / np.abs(ref)
    assert rel.max() < 1e-5, rel.max()
    d_got = got.sum(1) - LN2
    d_ref = ref.sum(1) - LN2
    assert np.abs(d_got - d_ref).max() < 1e-4 * np.sqrt((d_ref ** 2).mean())


def test_fullsize_d3q19_256_one_step_sampled_sites():
    """The D3Q19 step at the 3D benchmark's size (256^3 FP32, G = -5.0,
    rho0 = ln 2, kT = 1e-6, tau = 1: the unit-relaxation path, strip of 16
    planes as timed) against the oracle evaluated site by site on the same
    input state: random sites plus tile, strip and wrap boundaries."""
    from paper_2212_07848_gb300.lattice3 import Lattice3
    n = 256
    G, tau, kT, seed = -5.0, 1.0, 1e-6, 100
    g = Lattice3(n, n, n, G, tau, kT)
    g.set_strip(16)
    g.init(LN2, seed, 0.01)
    c0 = g.conserved()
    g.step(3)
    f_in = g.populations()
    g.step(1)
    f_out = g.populations()
    c1 = g.conserved()
    g.close()
    assert abs(c1[0] - c0[0]) / c0[0] < 1e-6
    assert np.abs(c1[1:] - c0[1:]).max() < 1e-6 * c0[0]
    rng = np.random.default_rng(2)
    xs, ys, zs = (list(rng.integers(0, n, 1500)) for _ in range(3))
    for ex in (0, 1, 31, 32, 33, 255):
        for ey in (0, 3, 4, 5, 7, 8, 9, 255):
            for ez in (0, 15, 16, 17, 255):
                xs.append(ex)
                ys.append(ey)
                zs.append(ez)
    ref = O.step_sites3(n, n, n, G, tau, kT, seed, 3, f_in, xs, ys, zs)
    got = f_out[:, zs, ys, xs].T
    rel = np.abs(got - ref) / np.abs(ref)
    assert rel.max() < 1e-5, rel.max()


def test_largest_lattice_properties():
    """The largest lattice the 32-bit element indices allow (9 nx ny < 2^32:
    16384 x 28672, 33.8 GB of FP32 populations), checked by properties that
    hold at any size: without noise the flat equilibrium stays exactly flat in
    every element; with noise mass and momentum are conserved and the last
    element of the last population plane is updated."""
    import torch

    from paper_2212_07848_gb300.lattice import Lattice
    nx, ny = 16384, 28672
    assert 9 * nx * ny < 2 ** 32
    g = Lattice(nx, ny, -3.6, 1.0, 0.0)
    g.init(LN2)
    g.step(2)
    g.sync()
    v = g.torch_populations()
    assert v.shape == (9, ny, nx)
    assert int(torch.count_nonzero(v)) == 0
    del v
    g.close()
    g = Lattice(nx, ny, -3.6, 1.0, 1e-5)
    g.init(LN2, 3, 0.0)
    c0 = g.conserved()
    g.step(3)
    g.sync()
    c1 = g.conserved()
    assert abs(c1[0] - c0[0]) / c0[0] < 1e-6
    assert np.abs(c1[1:] - c0[1:]).max() < 1e-6 * c0[0]
    v = g.torch_populations()
    assert float(v[8, ny - 1, nx - 1]) != 0.0 and float(v[0, 0, 0]) != 0.0
    del v
    g.close()
