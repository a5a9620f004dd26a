"""Pins of the D3Q19 oracle (the paper's three-dimensional setting) against
what the lattice and the mathematics fix: isotropy of the velocity set, an
orthogonal moment basis whose first ten modes span the polynomials of degree
at most two, exact streaming, exact conservation, invariance of the flat
equilibrium, the BGK relaxation of every moment, the fluctuation-dissipation
variance of each noise mode after one step, the ideal-gas structure factor,
and the continuum limit of the Shan-Chen force."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O

LN2 = float(np.log(2.0))


def test_d3q19_isotropy():
    c, w = O.lattice3_constants()
    cs2 = 1.0 / 3.0
    assert abs(w.sum() - 1.0) < 1e-15
    d = np.eye(3)
    for a, b in itertools.product(range(3), repeat=2):
        assert abs((w * c[:, a]).sum()) < 1e-15
        assert abs((w * c[:, a] * c[:, b]).sum() - cs2 * d[a, b]) < 1e-15
    for a, b, e in itertools.product(range(3), repeat=3):
        assert abs((w * c[:, a] * c[:, b] * c[:, e]).sum()) < 1e-15
    for a, b, e, f in itertools.product(range(3), repeat=4):
        iso = cs2 ** 2 * (d[a, b] * d[e, f] + d[a, e] * d[b, f] + d[a, f] * d[b, e])
        assert abs((w * c[:, a] * c[:, b] * c[:, e] * c[:, f]).sum() - iso) < 1e-15
    # every velocity has its opposite
    for i in range(19):
        assert sum(np.array_equal(c[j], -c[i]) for j in range(19)) == 1


def test_moment_basis_orthogonal_and_ordered():
    c, w = O.lattice3_constants()
    M, b = O.moment_basis3()
    G = (M * w) @ M.T
    assert np.abs(G - np.diag(b)).max() < 1e-14
    assert np.all(b > 0)
    # modes 0..3: mass and momentum
    assert np.array_equal(M[0], np.ones(19))
    for a in range(3):
        assert np.array_equal(M[1 + a], c[:, a].astype(float))
    # modes 0..9 span exactly the polynomials of degree <= 2
    cx, cy, cz = c.T.astype(float)
    P2 = np.array([np.ones(19), cx, cy, cz, cx * cx, cy * cy, cz * cz, cx * cy, cy * cz, cz * cx])
    assert np.linalg.matrix_rank(P2) == 10
    assert np.linalg.matrix_rank(np.vstack([P2, M[:10]])) == 10
    assert np.linalg.matrix_rank(M) == 19


def _random_pop(shape, seed):
    rng = np.random.default_rng(seed)
    c, w = O.lattice3_constants()
    return w[:, None, None, None] * (1.0 + 0.1 * rng.standard_normal((19,) + shape))


def test_pure_streaming_brute_force():
    nx, ny, nz, n = 6, 5, 4, 3
    f0 = _random_pop((nz, ny, nx), 1)
    o = O.OracleLattice3(nx, ny, nz, 0.0, 1e30, 0.0)
    o.init(1.0)
    o.set_populations(f0)
    o.step(n)
    f = o.populations()
    c, _ = O.lattice3_constants()
    for i in range(19):
        ref = np.roll(f0[i], (n * c[i, 2], n * c[i, 1], n * c[i, 0]), axis=(0, 1, 2))
        assert np.array_equal(f[i], ref), i


def test_flat_equilibrium_is_invariant():
    """Full populations: the 19-term density sum rounds, so the state stays
    flat to a few units in the last place of FP64 rather than bit for bit; it does not drift
    and no force, velocity or gradient appears."""
    o = O.OracleLattice3(6, 4, 5, -4.5, 0.8, 0.0)
    o.init(0.35)
    f0 = o.populations().copy()
    o.step(10)
    f = o.populations()
    assert np.abs(f - f0).max() <= 1e-14 * np.abs(f0).max()
    for i in range(19):
        assert np.ptp(f[i]) == 0.0                 # still uniform in space
    assert np.abs(o.force()).max() == 0.0


def test_conservation_with_noise_and_force():
    o = O.OracleLattice3(8, 6, 5, -4.2, 0.9, 1e-4)
    o.init(LN2, 7, 0.02)
    c0 = o.conserved()
    o.step(30)
    c1 = o.conserved()
    assert abs(c1[0] - c0[0]) < 1e-13 * c0[0]
    assert np.abs(c1[1:] - c0[1:]).max() < 1e-12 * c0[0]


def test_bgk_relaxes_every_moment():
    """G = 0, kT = 0, one step from random populations: with m the moments of
    the streamed populations and u = j / rho, the stress modes 4..9 become
    gamma m + (1 - gamma) m_eq (m_eq the rho u u moments) and the ghost modes
    10..18 become gamma m; mass and momentum are unchanged."""
    nx, ny, nz, tau = 5, 4, 3, 0.7
    gam = 1.0 - 1.0 / tau
    f0 = _random_pop((nz, ny, nx), 2)
    o = O.OracleLattice3(nx, ny, nz, 0.0, tau, 0.0)
    o.init(1.0)
    o.set_populations(f0)
    o.step(1)
    f1 = o.populations()
    c, w = O.lattice3_constants()
    M, _ = O.moment_basis3()
    g = np.stack([np.roll(f0[i], (c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2)) for i in range(19)])
    m = np.einsum("ki,ixyz->kxyz", M, g)
    ms = np.einsum("ki,ixyz->kxyz", M, f1)
    rho, u = m[0], m[1:4] / m[0]
    uu = lambda a, b: rho * u[a] * u[b]
    usq = u[0] ** 2 + u[1] ** 2 + u[2] ** 2
    meq = {4: rho * usq, 5: rho * (3 * u[0] ** 2 - usq), 6: uu(1, 1) - uu(2, 2),
           7: uu(0, 1), 8: uu(1, 2), 9: uu(2, 0)}
    for k in range(4):
        assert np.abs(ms[k] - m[k]).max() < 1e-14
    for k in range(4, 10):
        assert np.abs(ms[k] - (gam * m[k] + (1 - gam) * meq[k])).max() < 1e-14, k
    for k in range(10, 19):
        assert np.abs(ms[k] - gam * m[k]).max() < 1e-14, k


def test_one_step_noise_variance():
    """From the flat state each non-conserved moment after one step is its
    noise N_k: mean 0, variance mu rho0 b_k (1 - gamma^2); conserved moments
    are unchanged and the modes are uncorrelated."""
    nx = ny = nz = 16
    tau, kT, rho0 = 0.8, 1e-3, 1.3
    gam, mu = 1.0 - 1.0 / tau, kT * 3.0
    o = O.OracleLattice3(nx, ny, nz, 0.0, tau, kT)
    o.init(rho0, 12)
    o.step(1)
    M, b = O.moment_basis3()
    m = np.einsum("ki,ixyz->kxyz", M, o.populations()).reshape(19, -1)
    assert np.abs(m[0] - rho0).max() < 1e-14 and np.abs(m[1:4]).max() < 1e-15
    n = m.shape[1]
    z = []
    for k in range(4, 19):
        var = mu * rho0 * b[k] * (1 - gam ** 2)
        zk = m[k] / np.sqrt(var)
        assert abs(zk.mean()) < 5 / np.sqrt(n), k
        assert abs(zk.var() - 1.0) < 6 * np.sqrt(2.0 / n), k
        z.append(zk)
    cc = np.corrcoef(np.array(z))
    assert np.abs(cc - np.eye(15)).max() < 6 / np.sqrt(n)


def test_normals_are_standard():
    from scipy import stats
    z = np.array([O.normals3(8, 8, 8, 5, 0, s, 3) for s in range(3000)])
    for j in range(15):
        assert stats.kstest(z[:, j], "norm").pvalue > 1e-3, j
    assert np.abs(np.corrcoef(z.T) - np.eye(15)).max() < 0.1


def test_ideal_gas_structure_factor_is_flat():
    """G = 0: every axis mode of S(k) equals rho0 kT / c_s^2 (the
    fluctuation-dissipation balance of the noise amplitude)."""
    L, kT, rho0 = 8, 1e-4, 1.0
    o = O.OracleLattice3(L, L, L, 0.0, 1.0, kT)
    o.init(rho0, 3)
    o.sk_config(1, 200)
    o.step(2200)
    S, n = o.structure_factor_axes()
    assert n == 2001
    ref = rho0 * kT * 3.0
    assert abs(S.mean() / ref - 1.0) < 0.04, S / ref
    assert np.abs(S / ref - 1.0).max() < 0.15


@pytest.mark.parametrize("axis,kind", [(0, 0), (1, 0), (2, 0), (0, 1), (2, 2)])
def test_force_continuum_limit(axis, kind):
    """A weak sinusoidal density: the force approaches -G c_s^2 psi grad psi
    with second-order accuracy in the wave number, for each pseudopotential
    (kind 1: Eq. (5) with Tc = 5/12, nc = 1; kind 2: a = 1.3, b = 0.8)."""
    p1, p2 = {0: (0.0, 0.0), 1: (5.0 / 12.0, 1.0), 2: (1.3, 0.8)}[kind]
    rho0 = {0: LN2, 1: 1.0, 2: 0.9}[kind]
    psi_f = {0: lambda r: 1 - np.exp(-r),
             1: lambda r: np.sqrt(p1 * p2) * np.exp(1 - p2 / r),
             2: lambda r: p1 * np.exp(-p2 / r)}[kind]
    dpsi_f = {0: lambda r: np.exp(-r),
              1: lambda r: psi_f(r) * p2 / r ** 2,
              2: lambda r: psi_f(r) * p2 / r ** 2}[kind]
    errs = []
    for L in (16, 32):
        shape = [4, 4, 4]
        shape[axis] = L
        nx, ny, nz = shape
        o = O.OracleLattice3(nx, ny, nz, -4.0, 1.0, 0.0, psi_kind=kind, psi_p1=p1, psi_p2=p2)
        o.init(rho0)
        c, w = O.lattice3_constants()
        zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        coord = (xx, yy, zz)[axis]
        k = 2 * np.pi / L
        rho = rho0 + 0.05 * np.sin(k * coord)
        o.set_populations(w[:, None, None, None] * rho[None])
        F = o.force()
        psi = psi_f(rho)
        dpsi = dpsi_f(rho) * 0.05 * k * np.cos(k * coord)
        ref = 4.0 / 3.0 * psi * dpsi
        errs.append(np.abs(F[axis] - ref).max() / np.abs(ref).max())
        others = [b for b in range(3) if b != axis]
        assert np.abs(F[others]).max() < 1e-15
    assert errs[1] < errs[0] / 3.5 and errs[1] < 1e-2, errs


def test_step_sites_equals_full_step():
    """The site-by-site step (for checking large lattices) reproduces the
    full-lattice step at every site of a small noisy lattice, bit for bit."""
    nx, ny, nz, G, tau, kT, seed = 6, 5, 4, -4.2, 0.9, 1e-4, 7
    o = O.OracleLattice3(nx, ny, nz, G, tau, kT)
    o.init(LN2, seed, 0.02)
    o.step(2)
    f_in = o.populations().copy()
    o.step(1)
    ref = o.populations()
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    got = O.step_sites3(nx, ny, nz, G, tau, kT, seed, 2, f_in, xx.ravel(), yy.ravel(), zz.ravel())
    assert np.array_equal(got.T.reshape(19, nz, ny, nx), ref)


def test_full_structure_factor_matches_fft_and_axes():
    """The oracle's full 3D S(k) (three separable direct DFT passes): one
    sample equals |FFT(delta rho)|^2 / N of the sampled density, and its axis
    entries equal the oracle's axis S(k) over several samples."""
    nx, ny, nz = 8, 6, 4
    o = O.OracleLattice3(nx, ny, nz, -3.6, 1.0, 1e-4)
    o.init(LN2, 9, 0.01)
    o.sk_full()
    o.sk_config(1, 5)
    o.step(5)                                   # one sample, of the state after step 5
    S, n = o.structure_factor_full()
    assert n == 1
    rho = o.density()
    ref = np.abs(np.fft.fftn(rho - rho.mean())) ** 2 / rho.size
    assert np.abs(S - ref).max() < 1e-12 * ref.max()
    o.step(20)
    S, n = o.structure_factor_full()
    Sa, na = o.structure_factor_axes()
    assert n == na == 21
    axes = np.concatenate([S[0, 0, 1:nx // 2 + 1], S[0, 1:ny // 2 + 1, 0], S[1:nz // 2 + 1, 0, 0]])
    assert np.abs(axes - Sa).max() < 1e-12 * Sa.max()


def test_ideal_gas_full_structure_factor_is_flat():
    """G = 0: every radial shell of the full S(k) approaches rho0 kT / c_s^2."""
    L, kT, rho0 = 8, 1e-4, 1.0
    o = O.OracleLattice3(L, L, L, 0.0, 1.0, kT)
    o.init(rho0, 4)
    o.sk_full()
    o.sk_config(1, 200)
    o.step(1200)
    S, n = o.structure_factor_full()
    bins = O.radial_bins3(S)[1:]
    ref = rho0 * kT * 3.0
    assert abs(bins.mean() / ref - 1.0) < 0.04, bins / ref
    assert np.abs(bins / ref - 1.0).max() < 0.1


def test_radial_bins3_on_a_known_cube():
    """radial_bins3 of S = |q|^2 (q_a = folded index x max(n) / n_a) gives in
    each shell the mean of |q|^2 over the modes with round(|q|) = b, counted by
    brute force; k = 0 is left out."""
    nx, ny, nz = 8, 4, 4
    Lm = 8
    S = np.zeros((nz, ny, nx))
    shells = {}
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                q = np.array([(x if x <= nx // 2 else x - nx) * Lm / nx,
                              (y if y <= ny // 2 else y - ny) * Lm / ny,
                              (z if z <= nz // 2 else z - nz) * Lm / nz])
                S[z, y, x] = q @ q
                if (x, y, z) != (0, 0, 0):
                    shells.setdefault(int(np.rint(np.sqrt(q @ q))), []).append(q @ q)
    bins = O.radial_bins3(S)
    for b, vals in shells.items():
        assert abs(bins[b] - np.mean(vals)) < 1e-12, b
    assert bins[0] == 0.0


def test_ring_pair22_moments_exact():
    """The 3D mapping of one word to a pair: for a fixed high 22 bits (u =
    (h + 1/2) 2^-22, R^2 = -2 ln u) the 1024 low-bit angle indices reproduce the
    isotropic moments of a normal pair exactly (as the 2D ring does)."""
    for high in (0, 4321, 2 ** 21, 2 ** 22 - 1):
        R2 = -2.0 * np.log((high + 0.5) / 2.0 ** 22)
        z = np.array([O.ring_pair22((high << 10) | a) for a in range(1024)])
        z0, z1 = z[:, 0], z[:, 1]
        assert np.allclose(np.hypot(z0, z1), np.sqrt(R2), rtol=1e-14)
        tol = 1e-13 * max(R2, 1.0) ** 2
        for m in (z0.mean(), z1.mean(), (z0 * z1).mean(), (z0 ** 3).mean(), (z0 * z1 ** 2).mean()):
            assert abs(m) < tol
        assert abs((z0 ** 2).mean() - R2 / 2) < tol and abs((z1 ** 2).mean() - R2 / 2) < tol
        assert abs((z0 ** 4).mean() - 3 * R2 ** 2 / 8) < tol
        assert abs((z0 ** 2 * z1 ** 2).mean() - R2 ** 2 / 8) < tol
    # over all 2^22 radius values the radius moment E R^2 = 2 up to the 22-bit midpoint rule
    h = np.arange(2 ** 22, dtype=np.float64)
    assert abs(np.mean(-2.0 * np.log((h + 0.5) / 2.0 ** 22)) - 2.0) < 1e-6


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_flat_interface_normal_pressure_is_constant(tau):
    """Eq. (14) in 3D: along the normal of a flat interface the D3Q19 force
    stencil's half weights add up to 1/2 (1/6 on the axis, 4 x 1/12 on the
    face diagonals), as E4's do in 2D, so the lattice normal pressure
    P_N = rho c_s^2 + (G c_s^2 / 4) psi(x) [psi(x+1) + psi(x-1)] must be
    constant across a converged slab (G = -5, T_hat = 0.8; odd side, no k = pi
    mode), and the two bulk phases sit at equal EoS pressure.  The spread is
    taken at its minimum: at tau = 0.8 a slowly growing translation of the slab
    (a counterflow, about x3.5 per 10^4 steps, the same in 2D) lifts it again
    after about 3 10^4 steps, so the bound there is 5e-13."""
    from oracle import theory as T
    from paper_2212_07848_gb300 import inputs
    G = -5.0
    nx, ny, nz = 65, 2, 2
    rg, rl = T.coexistence(G, eps=0.0)
    o = O.OracleLattice3(nx, ny, nz, G, tau, 0.0)
    o.init(LN2)
    prof = inputs.slab_density(nx, 1, rg, rl, 32, smooth=1.5)[0]
    c, w = O.lattice3_constants()
    rho = np.broadcast_to(prof, (nz, ny, nx))
    o.set_populations(w[:, None, None, None] * rho[None])
    bound = 1e-13 if tau == 1.0 else 5e-13
    spread = []
    for _ in range(40):
        o.step(1000)
        d = o.density()
        pn = T.pn_lattice(d[0, 0], G)
        spread.append((pn.max() - pn.min()) / abs(pn.mean()))
        if spread[-1] < bound:
            break
    assert np.abs(d - d[0, 0]).max() == 0.0          # flat in y and z
    assert spread[-1] < bound, spread[-5:]
    assert d[0, 0].max() - d[0, 0].min() > 1.5
    rho_g, rho_l = d[0, 0][0], d[0, 0][nx // 2]
    pg, pl = T.pressure(rho_g, G), T.pressure(rho_l, G)
    assert abs(pl - pg) / abs(pg) < 1e-7
