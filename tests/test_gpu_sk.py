"""Device structure factor vs the oracle's direct DFT on the same trajectory,
and the radial read-out vs binning the half plane on the host."""
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


@pytest.mark.parametrize("nx,ny", [(64, 64), (128, 32)])
def test_radial_bins_match_host_binning(nx, ny):
    g, _ = make_pair(nx, ny, -3.6, 1.0, 1e-5, precision="fp32", seed=9)
    g.sk_config(2, 2)
    g.step(40)
    S, n = g.structure_factor()
    nb = max(nx, ny) // 2 + 2
    bins, nbs = g.structure_factor(nbins=nb)
    counts = g.structure_factor_counts(nb)
    assert nbs == n
    L = max(nx, ny)
    kx = np.arange(nx // 2 + 1)
    ky = np.fft.fftfreq(ny) * ny
    qx, qy = np.meshgrid(kx * (L / nx), ky * (L / ny))
    b = np.rint(np.sqrt(qx ** 2 + qy ** 2)).astype(int)
    w = np.where((kx == 0) | (2 * kx == nx), 1, 2)[None, :] * np.ones((ny, 1), int)
    w[0, 0] = 0
    ref_c = np.bincount(b.ravel(), weights=w.ravel(), minlength=nb)[:nb]
    ref_s = np.bincount(b.ravel(), weights=(w * S).ravel(), minlength=nb)[:nb]
    assert np.array_equal(counts, ref_c.astype(np.int64))
    ok = ref_c > 0
    assert np.allclose(bins[ok], ref_s[ok] / ref_c[ok], rtol=1e-12)
    assert np.all(np.isnan(bins[~ok]))


def test_unsupported_sizes_for_sk():
    from paper_2212_07848_gb300 import abi
    g, _ = make_pair(36, 20, -3.6, 1.0, 1e-5, precision="fp32")
    with pytest.raises(abi.LbError) as e:
        g.sk_config(1, 1)
    assert e.value.code == abi.LB_ERR_UNSUPPORTED
