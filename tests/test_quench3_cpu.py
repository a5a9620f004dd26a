"""The 3D topology classifier on constructed periodic fields: a sphere, a
cylinder along each axis, a slab, their gas-minority counterparts, and two
disjoint droplets."""
import numpy as np
import pytest

from paper_2212_07848_gb300.quench3 import classify_topology3, components3

N = 24
z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")


def _field(mask):
    return np.where(mask, 2.0, 0.2)


def test_sphere_and_bubble():
    r2 = (x - 8) ** 2 + (y - 12) ** 2 + (z - 20) ** 2
    topo, phi, _ = classify_topology3(_field(r2 < 25))
    assert topo == "droplet" and phi < 0.5
    topo, phi, _ = classify_topology3(_field(r2 >= 25))
    assert topo == "bubble" and phi > 0.5


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_cylinders_wrap_once(axis):
    a, b = [(y, z), (x, z), (x, y)][axis]
    cyl = (a - 5) ** 2 + (b - 18) ** 2 < 16      # centred near the box edge: wraps there
    comps = components3(cyl)
    assert len(comps) == 1 and sum(comps[0][1]) == 1 and comps[0][1][axis]
    assert classify_topology3(_field(cyl))[0] == "droplet-cylinder"
    assert classify_topology3(_field(~cyl))[0] == "bubble-cylinder"


def test_slab_and_mixed():
    slab = (z >= 20) | (z < 4)                   # across the periodic boundary
    assert classify_topology3(_field(slab))[0] == "flat"
    two = ((x - 5) ** 2 + (y - 5) ** 2 + (z - 5) ** 2 < 9) | ((x - 16) ** 2 + (y - 16) ** 2 < 9)
    comps = components3(two)
    assert len(comps) == 2
    assert classify_topology3(_field(two))[0] == "mixed"


def test_weak_fluctuations_are_homogeneous():
    rng = np.random.default_rng(0)
    assert classify_topology3(1.0 + 0.01 * rng.standard_normal((N, N, N)))[0] == "homogeneous"
