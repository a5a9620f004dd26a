"""Device structure factor vs the oracle's direct DFT on the same trajectory,
and the radial read-out and first moments vs the oracle's binning and sums."""
import numpy as np
import pytest

from pairs import LN2, make_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-3)])
@pytest.mark.parametrize("nx,ny", [(64, 32), (16, 128), (256, 256)])
def test_structure_factor_matches_oracle(precision, tol, nx, ny):
    g, o = make_pair(nx, ny, -3.6, 1.0, 1e-5, precision=precision, seed=2)
    for lat in (g, o):
        lat.sk_config(1, 21)
    g.step(60)
    o.step(60)
    Sg, ng = g.structure_factor()
    So, no = o.structure_factor()
    assert ng == no == 40
    assert Sg.shape == So.shape == (ny, nx // 2 + 1)
    assert Sg[0, 0] == 0.0
    scale = So + So.mean()
    assert np.max(np.abs(Sg - So) / scale) < tol


def test_sample_now_matches_oracle():
    g, o = make_pair(32, 64, -3.6, 1.0, 1e-4, precision="fp64", seed=4, amp=0.02)
    g.step(7)
    o.step(7)
    g.sk_reset()
    o.sk_reset()
    g.sk_sample_now()
    o.sk_sample_now()
    Sg, _ = g.structure_factor()
    So, _ = o.structure_factor()
    assert np.max(np.abs(Sg - So) / (So + So.mean())) < 1e-10


@pytest.mark.parametrize("nx,ny", [(64, 64), (128, 32), (32, 64)])
def test_radial_bins_match_oracle_binning(nx, ny):
    """The device's radial read-out (mean S per bin, modes per bin) equals the
    oracle's radial binning of the device's own half-plane S(k): counts index
    exact, means to FP64 rounding of the (atomic) bin sums."""
    from oracle import oracle as O
    g, _ = make_pair(nx, ny, -3.6, 1.0, 1e-5, precision="fp32", seed=9)
    g.sk_config(2, 2)
    g.step(40)
    S, n = g.structure_factor()
    for nb in (max(nx, ny) // 2 + 2, 7):
        bins, nbs = g.structure_factor(nbins=nb)
        counts = g.structure_factor_counts(nb)
        assert nbs == n
        ref_m, ref_c = O.radial_bins(S, nx, ny, nb)
        assert np.array_equal(counts, ref_c)
        ok = ref_c > 0
        assert np.allclose(bins[ok], ref_m[ok], rtol=1e-12, atol=0.0)
        assert np.all(np.isnan(bins[~ok]))


@pytest.mark.parametrize("nx,ny", [(64, 64), (128, 32)])
def test_sk_moments_match_oracle(nx, ny):
    """The device's first moments of S(k) (the domain size L(t) of the quench
    driver) equal the oracle's sums over the full plane."""
    from oracle import oracle as O
    g, _ = make_pair(nx, ny, -5.0, 1.0, 1e-5, precision="fp32", seed=3, amp=0.05)
    g.sk_config(5, 5)
    g.step(50)
    S, _ = g.structure_factor()
    m = g.sk_moments()
    s0, s1 = O.sk_first_moments(S, nx, ny)
    assert abs(m[0] / s0 - 1.0) < 1e-12
    assert abs(m[1] / s1 - 1.0) < 1e-12
    assert abs(g.domain_size() / (2 * np.pi * s0 / s1) - 1.0) < 1e-12


def test_unsupported_sizes_for_sk():
    from paper_2212_07848_gb300 import abi
    g, _ = make_pair(36, 20, -3.6, 1.0, 1e-5, precision="fp32")
    with pytest.raises(abi.LbError) as e:
        g.sk_config(1, 1)
    assert e.value.code == abi.LB_ERR_UNSUPPORTED
