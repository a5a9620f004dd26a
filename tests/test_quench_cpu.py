"""Topology classification of periodic 2D density fields (host analysis used
by the quench experiment): slabs, droplets, bubbles, wrapping detection."""
import numpy as np

from paper_2212_07848_gb300 import inputs
from paper_2212_07848_gb300.quench import _components, classify_topology


def test_slab_is_a_stripe():
    rho = inputs.slab_density(64, 48, 0.1, 1.9, 24)
    topo, phi, comps = classify_topology(rho, 1.0)
    assert topo == "stripe" and abs(phi - 24 / 64) < 0.05
    assert len(comps) == 1 and comps[0][2] and not comps[0][1]   # wraps in y only


def test_droplet_and_bubble():
    drop = inputs.droplet_density(64, 64, 10, 1.9, 0.1)
    assert classify_topology(drop, 1.0)[0] == "droplet"
    bub = inputs.droplet_density(64, 64, 10, 0.1, 1.9)
    assert classify_topology(bub, 1.0)[0] == "bubble"


def test_droplet_across_the_periodic_boundary_does_not_wrap():
    drop = np.roll(inputs.droplet_density(64, 64, 10, 1.9, 0.1), (32, 32), axis=(0, 1))
    topo, _, comps = classify_topology(drop, 1.0)
    assert topo == "droplet" and len(comps) == 1


def test_component_wrapping_in_both_directions():
    m = np.zeros((16, 16), bool)
    m[5, :] = True
    m[:, 9] = True
    comps = _components(m)
    assert len(comps) == 1 and comps[0][1] and comps[0][2]
    two = np.zeros((16, 16), bool)
    two[2:4, 2:4] = True
    two[10:12, 10:12] = True
    assert sorted(c[0] for c in _components(two)) == [4, 4]


def test_growth_exponent_and_block_mean():
    """The driver's helpers: the log-log slope of an exact power law over the
    chosen window, and block means of a field."""
    import numpy as np

    from paper_2212_07848_gb300.quench import block_mean, growth_exponent
    t = np.arange(500, 50001, 500)
    L = 2.5 * t ** 0.45
    L[t < 5000] *= 3.0                       # a different early regime, outside the window
    assert abs(growth_exponent(t, L, 5000) - 0.45) < 1e-12
    f = np.arange(64.0).reshape(8, 8)
    b = block_mean(f, 4)
    assert b.shape == (2, 2)
    assert b[0, 0] == f[:4, :4].mean() and b[1, 1] == f[4:, 4:].mean()
