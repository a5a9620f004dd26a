"""Batched ensemble: every replica evolves exactly as a single lattice with
the same parameters, seed and replica index (the same per-site code), for
steps taken singly or replayed from captured graphs, with S(k) sampling;
small replicas also match the oracle; the autotuner leaves the state intact."""
import numpy as np
import pytest

from oracle import oracle as O
from pairs import LN2, max_rel

pytestmark = pytest.mark.gpu

REPS = [(64, 64, -3.6, 1.0, 1e-5, LN2), (128, 32, -4.2, 0.8, 1e-5, 0.7),
        (32, 32, -4.8, 1.3, 1e-5, 0.65), (256, 128, -3.9, 1.0, 1e-6, 0.75),
        (64, 64, -4.0, 1.0, 0.0, LN2), (16, 64, -3.6, 1.1, 1e-5, 0.72)]


def _single(r, rep, seed, amp, sk=None):
    from paper_2212_07848_gb300.lattice import Lattice
    nx, ny, G, tau, kT, rho0 = rep
    g = Lattice(nx, ny, G, tau, kT)
    g.set_replica(r)
    g.init(rho0, seed, amp)
    if sk:
        g.sk_config(*sk)
    return g


@pytest.mark.parametrize("kernel", [1, 3])        # strip layouts: halo warp, overlapped
@pytest.mark.parametrize("launch", [0, 1])        # per-step launches, persistent windows
@pytest.mark.parametrize("strip", [8, 32])
def test_replicas_match_single_lattices(strip, launch, kernel):
    from paper_2212_07848_gb300.ensemble import Ensemble
    e = Ensemble(REPS, seed=77)
    e.set_kernel(kernel)
    assert e.kernel == kernel
    e.set_launch(launch)
    assert e.launch == launch
    e.set_strip_height(strip)
    e.init(0.01)
    e.sk_config(5, 10)
    e.step(3)          # single launches
    e.step(64)         # graph windows of 5 steps with a sample at the end
    e.step(4)
    e.sync()
    assert e.t == 71
    for r, rep in enumerate(REPS):
        g = _single(r, rep, 77, 0.01, (5, 10))
        g.step(71)
        assert np.array_equal(e.populations(r), g.populations()), r
        Se, ne = e.structure_factor(r)
        Sg, ng = g.structure_factor()
        assert ne == ng == 13
        assert np.array_equal(Se, Sg), r


def test_plain_graph_windows_match():
    from paper_2212_07848_gb300.ensemble import Ensemble
    a = Ensemble(REPS, seed=5)
    b = Ensemble(REPS, seed=5)
    a.init(0.02)
    b.init(0.02)
    a.step(100)                      # three 32-step graph replays + 4 single steps
    for _ in range(100):
        b.step(1)                    # single launches only
    for r in range(len(REPS)):
        assert np.array_equal(a.populations(r), b.populations(r))


def test_small_replica_matches_oracle():
    from paper_2212_07848_gb300.ensemble import Ensemble
    e = Ensemble(REPS, seed=9)
    e.init(0.01)
    e.step(60)
    for r in (0, 2, 5):
        nx, ny, G, tau, kT, rho0 = REPS[r]
        o = O.OracleLattice(nx, ny, G, tau, kT, replica=r)
        o.init(rho0, 9, 0.01)
        o.step(60)
        assert max_rel(e.populations(r), o.populations()) < 1e-4
        c = e.conserved(r)
        assert abs(c[0] - o.conserved()[0]) / c[0] < 1e-6


def test_autotune_keeps_state(tmp_path):
    from paper_2212_07848_gb300.ensemble import Ensemble
    a = Ensemble(REPS, seed=3)
    b = Ensemble(REPS, seed=3)
    a.init(0.01)
    b.init(0.01)
    a.step(7)
    b.step(7)
    cache = str(tmp_path / "tune.txt")
    s = a.autotune(5, cache)
    assert s in (8, 12, 16, 24, 32, 48)
    assert a.t == 7
    a.step(10)
    b.step(10)
    for r in range(len(REPS)):
        assert np.array_equal(a.populations(r), b.populations(r))
    # a second ensemble of the same shape reads the choice from the cache
    c = Ensemble(REPS, seed=3)
    c.init(0.0)
    assert c.autotune(5, cache) == s
    assert open(cache).read().count("\n") == 1


def test_persistent_launch_many_tiles_per_cta():
    """More tiles than resident CTAs (each CTA sweeps several tiles per step and
    waits on the replica barriers): persistent windows give the per-step bits,
    including the S(k) sampling windows."""
    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.ensemble import Ensemble
    reps = [(1024, 1024, -4.4, 1.0, 1e-6, LN2), (512, 1024, -3.8, 0.9, 1e-6, 0.7),
            (1024, 256, -4.0, 1.1, 1e-6, 0.68), (256, 256, -4.6, 1.0, 1e-6, LN2)]
    a, b = Ensemble(reps, seed=9), Ensemble(reps, seed=9)
    a.set_launch(abi.LB_ENS_PERSISTENT)
    b.set_kernel(abi.LB_KERNEL_OVERLAP)         # the other strip layout: the same bits
    for e in (a, b):
        e.set_strip_height(8)
        e.init(0.01)
        e.sk_config(16, 16)
    assert a.kernel == abi.LB_KERNEL_PLAIN     # automatic layout for power-of-two widths
    assert a.num_tiles > 1000          # above the 6 x 152 resident CTAs
    a.step(3)
    a.step(16 * 4 + 5)      # sampling windows replayed as persistent launches
    a.step(40)
    b.step(3)
    b.step(16 * 4 + 5)
    b.step(40)
    a.sync()                # raises on a barrier timeout or a non-finite value
    for r in range(len(reps)):
        assert np.array_equal(a.populations(r), b.populations(r)), r
        Sa, na = a.structure_factor(r)
        Sb, nb = b.structure_factor(r)
        assert na == nb and np.array_equal(Sa, Sb), r


@pytest.mark.parametrize("kernel", [1, 3])
@pytest.mark.parametrize("taus", ["unit", "none", "mixed"])
def test_persistent_unit_modes_many_replicas(taus, kernel):
    """The persistent kernel is specialised on whether every replica, none or
    some take the unit-relaxation path; with many replicas of mixed sizes (so
    the dynamic (step, tile) hand-out crosses steps and replicas all the
    time) each specialisation gives the per-step bits, S(k) included."""
    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.ensemble import Ensemble
    rng = np.random.default_rng(21)
    n = 96
    sizes = rng.choice([64, 128, 256], size=n)
    tau = {"unit": np.ones(n), "none": rng.uniform(0.8, 1.3, n),
           "mixed": np.where(rng.random(n) < 0.5, 1.0, 0.9)}[taus]
    reps = [(int(s), int(s), float(rng.uniform(-4.8, -3.6)), float(t), 1e-6,
             float(LN2 * (1 + rng.uniform(-0.1, 0.1)))) for s, t in zip(sizes, tau)]
    a, b = Ensemble(reps, seed=13), Ensemble(reps, seed=13)
    for e in (a, b):
        e.set_kernel(kernel)
        e.set_strip_height(8)
        e.init(0.01)
        e.sk_config(10, 10)
    a.set_launch(abi.LB_ENS_PERSISTENT)
    a.step(2)
    a.step(43)
    b.step(2)
    b.step(43)
    a.sync()
    for r in range(n):
        assert np.array_equal(a.populations(r), b.populations(r)), r
        Sa, na = a.structure_factor(r)
        Sb, nb = b.structure_factor(r)
        assert na == nb == 4 and np.array_equal(Sa, Sb), r


# shapes that live in shared memory: one CTA (64^2, 32^2, 32 x 128) or a
# cluster of CTAs reading each other's rows (128 x 64: two, 128^2: four)
RESIDENT_SHAPES = [(64, 64), (32, 32), (32, 128), (128, 64), (128, 128)]


def _resident_pair(reps, stencil, launch, seed=31):
    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.ensemble import Ensemble
    a = Ensemble(reps, stencil=stencil, seed=seed)
    b = Ensemble(reps, stencil=stencil, seed=seed)
    a.set_resident(abi.LB_ENS_RESIDENT_ON)
    b.set_resident(abi.LB_ENS_RESIDENT_OFF)
    assert b.num_resident == 0
    for e in (a, b):
        e.set_launch(launch)
        e.set_strip_height(16)
        e.init(0.01)
        e.sk_config(5, 10)
        e.step(3)          # single steps
        e.step(37)         # sampling windows of 5 steps
        e.step(33)         # a plain 32-step window + 1
    a.sync()
    b.sync()
    return a, b


@pytest.mark.parametrize("stencil", [4, 6, 8])
@pytest.mark.parametrize("shape", RESIDENT_SHAPES)
def test_resident_replicas_match_tiles(shape, stencil):
    """Replicas kept in shared memory over whole windows of steps (in place,
    band by band, boundary rows copied each step, across a cluster through
    distributed shared memory) give the tile path's bits, S(k) included,
    for unit and general relaxation rates."""
    nx, ny = shape
    reps = [(nx, ny, -4.4, 1.0, 1e-5, LN2), (nx, ny, -3.9, 0.8, 1e-5, 0.7),
            (nx, ny, -4.7, 1.0, 0.0, 0.72)]
    a, b = _resident_pair(reps, stencil, 0)
    assert a.num_resident == len(reps)
    assert a.num_tiles == 0
    for r in range(len(reps)):
        assert np.array_equal(a.populations(r), b.populations(r)), r
        Sa, na = a.structure_factor(r)
        Sb, nb = b.structure_factor(r)
        assert na == nb == 13 and np.array_equal(Sa, Sb), r


@pytest.mark.parametrize("launch", [0, 1])
def test_resident_and_tiled_replicas_together(launch):
    """Resident replicas next to replicas that stay tiled (too wide or too
    narrow for shared memory), per-step and persistent tile launches: every
    replica keeps the bits of a single lattice."""
    reps = [(64, 64, -4.4, 1.0, 1e-5, LN2), (256, 64, -4.0, 1.0, 1e-5, 0.7),
            (128, 128, -4.6, 0.9, 1e-5, 0.68), (16, 64, -3.8, 1.0, 1e-5, LN2),
            (32, 32, -4.2, 1.0, 1e-5, 0.7)]
    a, b = _resident_pair(reps, 4, launch)
    assert a.num_resident == 3
    for r, rep in enumerate(reps):
        assert np.array_equal(a.populations(r), b.populations(r)), r
        Sa, na = a.structure_factor(r)
        Sb, nb = b.structure_factor(r)
        assert na == nb and np.array_equal(Sa, Sb), r
    # and against single lattices
    for r, rep in enumerate(reps):
        g = _single(r, rep, 31, 0.01, (5, 10))
        g.step(73)
        assert np.array_equal(a.populations(r), g.populations()), r


def test_resident_auto_policy():
    """AUTO keeps an ensemble in shared memory only when every replica fits
    one CTA; clusters only when asked for."""
    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.ensemble import Ensemble
    small = [(64, 64, -4.4, 1.0, 1e-6, LN2)] * 4
    e = Ensemble(small, seed=1)
    assert e.num_resident == 4 and e.num_tiles == 0
    e.set_resident(abi.LB_ENS_RESIDENT_OFF)
    assert e.num_resident == 0 and e.num_tiles > 0
    mixed = small + [(256, 256, -4.4, 1.0, 1e-6, LN2)]
    m = Ensemble(mixed, seed=1)
    assert m.num_resident == 0
    m.set_resident(abi.LB_ENS_RESIDENT_ON)
    assert m.num_resident == 4
    m.init(0.0)
    assert m.autotune(3) in (8, 12, 16, 24, 32, 48)
    c = Ensemble([(128, 128, -4.4, 1.0, 1e-6, LN2)] * 2, seed=1)
    assert c.num_resident == 0
    c.set_resident(abi.LB_ENS_RESIDENT_ON)
    assert c.num_resident == 2
    e.set_resident(abi.LB_ENS_RESIDENT_AUTO)
    e.init(0.0)
    e.autotune(3)          # nothing tiled: the call keeps the strip height
    e.step(40)
    e.sync()


@pytest.mark.parametrize("stencil", [4, 8])
@pytest.mark.parametrize("strip", [1, 3, 8])
@pytest.mark.parametrize("kernel", [1, 3])
def test_persistent_tile_dependencies(stencil, strip, kernel):
    """The persistent launch lets a tile start a step as soon as the tiles it
    pulls from (its neighbours within the stencil's reach, wrapped) finished
    the previous one.  Thin row strips (a tile's reach spans several), a
    ragged last column strip and one large replica with many tiles per step:
    the per-step bits."""
    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.ensemble import Ensemble
    reps = [(512, 256, -4.4, 1.0, 1e-5, LN2), (132, 64, -4.0, 1.0, 1e-5, 0.7),
            (32, 16, -4.6, 0.9, 1e-5, 0.68)]
    a = Ensemble(reps, stencil=stencil, seed=41)
    b = Ensemble(reps, stencil=stencil, seed=41)
    for e in (a, b):
        e.set_resident(abi.LB_ENS_RESIDENT_OFF)
        e.set_kernel(kernel)
        e.set_strip_height(strip)
        e.init(0.01)
    a.set_launch(abi.LB_ENS_PERSISTENT)
    a.step(70)
    b.step(70)
    a.sync()
    for r in range(len(reps)):
        assert np.array_equal(a.populations(r), b.populations(r)), r
