"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: lattice
isotropy identities, the isotropy equations that define the force stencils, a
library Philox (numpy's 4x64-10, which shares the round structure), brute-force
streaming, moment identities of the BGK/Guo collision, the fluctuation-
dissipation variance of the noise, numpy's FFT for the structure-factor sum,
and exact conservation and symmetry laws.
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import theory as T
from paper_2212_07848_gb300 import inputs

LN2 = float(np.log(2.0))


def _velocities():
    cx, cy, w, cs2 = O.lattice_constants()
    return cx.astype(float), cy.astype(float), w, cs2


# --------------------------------------------------------------------------
# Lattice constants
# --------------------------------------------------------------------------
def test_d2q9_isotropy_sums():
    cx, cy, w, cs2 = _velocities()
    c = np.stack([cx, cy], 1)
    d = np.eye(2)
    assert abs(cs2 - 1.0 / 3.0) < 1e-16
    assert abs(w.sum() - 1.0) < 1e-15
    assert len({(int(a), int(b)) for a, b in c}) == 9
    for a in range(2):
        assert abs((w * c[:, a]).sum()) < 1e-16
        for b in range(2):
            assert abs((w * c[:, a] * c[:, b]).sum() - cs2 * d[a, b]) < 1e-15
            for g in range(2):
                assert abs((w * c[:, a] * c[:, b] * c[:, g]).sum()) < 1e-16
                for h in range(2):
                    m4 = (w * c[:, a] * c[:, b] * c[:, g] * c[:, h]).sum()
                    iso = cs2 ** 2 * (d[a, b] * d[g, h] + d[a, g] * d[b, h] + d[a, h] * d[b, g])
                    assert abs(m4 - iso) < 1e-15


def test_moment_basis_orthogonal_complete_conserved_first():
    M, b = O.moment_basis()
    cx, cy, w, _ = _velocities()
    gram = (M * w) @ M.T
    assert np.abs(gram - np.diag(b)).max() < 1e-14
    assert np.all(b > 0)
    assert np.linalg.matrix_rank(M) == 9
    assert np.array_equal(M[0], np.ones(9))
    assert np.array_equal(M[1], cx) and np.array_equal(M[2], cy)
    # every basis vector is an integer polynomial of c (exact integer entries)
    assert np.array_equal(M, np.round(M))


@pytest.mark.parametrize("order,count", [(4, 8), (6, 12), (8, 24)])
def test_force_stencil_weights_solve_isotropy(order, count):
    ex, ey, w = O.stencil(order)
    assert len(ex) == count
    ref = T.isotropic_weights(order)          # exact rational solution
    shells = {}
    for x, y, ww in zip(ex, ey, w):
        e2 = int(x * x + y * y)
        assert ww == float(ref[e2])
        shells.setdefault(e2, set()).add((int(x), int(y)))
    # each shell is complete (all lattice vectors of that length, |e_x|,|e_y| <= 2)
    for e2, vecs in shells.items():
        full = {(x, y) for x in range(-2, 3) for y in range(-2, 3) if x * x + y * y == e2}
        assert vecs == full
    assert set(shells) == set(ref)
    assert abs((w * ex.astype(float) ** 2).sum() - 1.0) < 1e-15


# --------------------------------------------------------------------------
# Random numbers
# --------------------------------------------------------------------------
@pytest.mark.parametrize("key,ctr", [
    ((0, 0), (0, 0, 0, 0)),
    ((123, 456), (7, 0, 0, 0)),
    ((0xFFFFFFFFFFFFFFFF, 1), (5, 9, 0xDEADBEEF, 3)),
    ((2 ** 63 + 11, 2 ** 40), (2 ** 64 - 1, 17, 2, 2 ** 62)),   # carry into word 1
])
def test_philox4x64_matches_numpy(key, ctr):
    bg = np.random.Philox(key=np.array(key, np.uint64), counter=np.array(ctr, np.uint64))
    raw = bg.random_raw(8)
    # numpy bumps the 256-bit counter by one before each block
    c = list(ctr)
    for blk in range(2):
        v = (c[0] + (c[1] << 64) + (c[2] << 128) + (c[3] << 192) + 1) % (1 << 256)
        c = [(v >> (64 * j)) & (2 ** 64 - 1) for j in range(4)]
        out = O.philox4x64(c, key)
        assert [int(x) for x in out] == [int(x) for x in raw[4 * blk:4 * blk + 4]]


def test_philox4x32_statistics():
    """Uniform bytes and full avalanche on a one-bit counter change."""
    key = (0x12345678, 0x9ABCDEF0)
    words = np.array([O.philox4x32((s, 3, 0, 0), key) for s in range(4096)], np.uint32)
    by = words.view(np.uint8).ravel()
    counts = np.bincount(by, minlength=256)
    exp = by.size / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 256 + 6 * np.sqrt(2 * 256)
    flips = []
    for s in range(256):
        a = O.philox4x32((s, 11, 0, 1), key)
        for bit in (0, 13, 31):
            b = O.philox4x32((s ^ (1 << bit), 11, 0, 1), key)
            flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert abs(np.mean(flips) - 64.0) < 1.5


def test_box_muller_normals():
    from scipy import stats
    p = O.make_params(8, 8, 0.0, 1.0, 1.0, seed=42)
    z = np.array([O.normals(p, s, 5) for s in range(6000)])
    for j in range(6):
        assert stats.kstest(z[:, j], "norm").pvalue > 1e-3
    cc = np.corrcoef(z.T)
    assert np.abs(cc - np.eye(6)).max() < 0.06


def test_box_muller_ring_moments_exact():
    """Over the 1024 angle indices of one radius word R the pair reproduces the
    isotropic moments exactly: mean z0 = mean z1 = mean z0 z1 = 0,
    mean z0^2 = mean z1^2 = R^2 / 2, mean z0^4 = 3 R^4 / 8,
    mean z0^2 z1^2 = R^4 / 8, and R^2 = -2 ln u with u = (r + 1/2) 2^-32."""
    for word in (0, 12345, 2 ** 31, 2 ** 32 - 1):
        R2 = -2.0 * np.log((word + 0.5) / 2.0 ** 32)
        z = np.array([O.box_muller_ring(word, a) for a in range(1024)])
        z0, z1 = z[:, 0], z[:, 1]
        assert np.allclose(np.hypot(z0, z1), np.sqrt(R2), rtol=1e-14)
        tol = 1e-13 * max(R2, 1.0) ** 2
        for m in (z0.mean(), z1.mean(), (z0 * z1).mean(), (z0 ** 3).mean(), (z0 * z1 ** 2).mean()):
            assert abs(m) < tol
        assert abs((z0 ** 2).mean() - R2 / 2) < tol and abs((z1 ** 2).mean() - R2 / 2) < tol
        assert abs((z0 ** 4).mean() - 3 * R2 ** 2 / 8) < tol
        assert abs((z0 ** 2 * z1 ** 2).mean() - R2 ** 2 / 8) < tol
    # the angle index takes 10 bits: index a and a + 1024 give the same pair
    assert np.array_equal(O.box_muller_ring(777, 5), O.box_muller_ring(777, 5 + 1024))


# --------------------------------------------------------------------------
# Streaming, collision, forcing
# --------------------------------------------------------------------------
def test_pure_streaming_brute_force():
    """tau -> infinity, G = 0, kT = 0 leaves only pull streaming:
    f_i(x, t+n) = f_i(x - n c_i, t), periodic."""
    nx, ny, n = 12, 7, 5
    f0 = inputs.random_populations(nx, ny, seed=1)
    o = O.OracleLattice(nx, ny, G=0.0, tau=1e30, kT=0.0)
    o.init(1.0)
    o.set_populations(f0)
    o.step(n)
    f = o.populations()
    cx, cy, _, _ = O.lattice_constants()
    for i in range(9):
        assert np.array_equal(f[i], np.roll(f0[i], (n * cy[i], n * cx[i]), axis=(0, 1)))


def _stream(f):
    cx, cy, _, _ = O.lattice_constants()
    return np.stack([np.roll(f[i], (cy[i], cx[i]), axis=(0, 1)) for i in range(9)])


def _moments(f):
    cx, cy, _, _ = _velocities()
    rho = f.sum(0)
    jx = np.tensordot(cx, f, 1)
    jy = np.tensordot(cy, f, 1)
    pxx = np.tensordot(cx * cx, f, 1)
    pyy = np.tensordot(cy * cy, f, 1)
    pxy = np.tensordot(cx * cy, f, 1)
    return rho, jx, jy, pxx, pyy, pxy


@pytest.mark.parametrize("tau", [1.0, 0.8, 1.7])
def test_bgk_relaxes_second_moments(tau):
    """G = 0, kT = 0: mass and momentum are kept and the second moments relax
    as Pi* = Pi_eq + (1 - 1/tau)(Pi - Pi_eq), Pi_eq = rho (c_s^2 I + u u);
    the 3rd/4th-order Hermite moments relax towards zero at the same rate."""
    nx, ny = 10, 6
    f0 = inputs.random_populations(nx, ny, seed=2)
    o = O.OracleLattice(nx, ny, G=0.0, tau=tau, kT=0.0)
    o.init(1.0)
    o.set_populations(f0)
    o.step(1)
    g = _stream(f0)
    f1 = o.populations()
    rho, jx, jy, pxx, pyy, pxy = _moments(g)
    r1, jx1, jy1, pxx1, pyy1, pxy1 = _moments(f1)
    gam = 1.0 - 1.0 / tau
    ux, uy = jx / rho, jy / rho
    cs2 = 1.0 / 3.0
    for a, b in [(r1, rho), (jx1, jx), (jy1, jy)]:
        assert np.abs(a - b).max() < 1e-15
    for post, pre, eq in [(pxx1, pxx, rho * (cs2 + ux * ux)), (pyy1, pyy, rho * (cs2 + uy * uy)),
                          (pxy1, pxy, rho * ux * uy)]:
        assert np.abs(post - (eq + gam * (pre - eq))).max() < 1e-14
    M, _ = O.moment_basis()
    for k in (6, 7, 8):
        assert np.abs(np.tensordot(M[k], f1, 1) - gam * np.tensordot(M[k], g, 1)).max() < 1e-14


@pytest.mark.parametrize("stencil,tau", [(4, 0.9), (6, 1.3), (8, 0.6)])
def test_guo_forcing_moments(stencil, tau):
    """Guo, Zheng and Shi (2002): with u = (j + F/2)/rho the post-collision
    momentum is j + F and the source adds (1 - 1/(2 tau)) (u F + F u) to the
    second moments; the force is the Shan-Chen force of the streamed density."""
    nx, ny = 16, 12
    rho_in = inputs.perturbed_density(nx, ny, LN2, 0.05, seed=3)
    f0 = inputs.random_populations(nx, ny, seed=4, lo=-0.01, hi=0.01)
    o = O.OracleLattice(nx, ny, G=-3.6, tau=tau, kT=0.0, stencil=stencil)
    o.init(LN2)
    o.set_density(rho_in)
    f0 = o.populations() + f0
    o.set_populations(f0)
    o.step(1)
    f1 = o.populations()
    g = _stream(f0)
    probe = O.OracleLattice(nx, ny, G=-3.6, tau=tau, kT=0.0, stencil=stencil)
    probe.init(LN2)
    probe.set_populations(g)
    Fx, Fy = probe.force()          # force of the streamed density
    rho, jx, jy, pxx, pyy, pxy = _moments(g)
    r1, jx1, jy1, pxx1, pyy1, pxy1 = _moments(f1)
    assert np.abs(r1 - rho).max() < 1e-15
    assert np.abs(jx1 - (jx + Fx)).max() < 1e-15
    assert np.abs(jy1 - (jy + Fy)).max() < 1e-15
    ux, uy = (jx + Fx / 2) / rho, (jy + Fy / 2) / rho
    gam, cs2, s = 1.0 - 1.0 / tau, 1.0 / 3.0, 1.0 - 1.0 / (2.0 * tau)
    eq = [rho * (cs2 + ux * ux), rho * (cs2 + uy * uy), rho * ux * uy]
    src = [2 * ux * Fx, 2 * uy * Fy, ux * Fy + uy * Fx]
    for post, pre, e, sr in zip([pxx1, pyy1, pxy1], [pxx, pyy, pxy], eq, src):
        assert np.abs(post - (e + gam * (pre - e) + s * sr)).max() < 1e-14


# psi kinds: 0 = 1 - exp(-rho); 1 = Eq. (5) with (T_c, n_c); 2 = a exp(-b/n),
# the form introduced before Eq. (3), here with (a, b) away from the
# critical-point constants of Eq. (4) so that it is not kind 1 in disguise.
PSI_KINDS = [(0, 0.0, 0.0), (1, 0.5, 0.9), (2, 1.3, 0.8)]


@pytest.mark.parametrize("kind,p1,p2", PSI_KINDS)
@pytest.mark.parametrize("stencil", [4, 6, 8])
def test_force_sums_to_zero_and_continuum_limit(stencil, kind, p1, p2):
    """Sum of F over the lattice vanishes (pair antisymmetry of Eq. (1)), and
    for a long-wave density F -> -G c_s^2 psi grad psi (the continuum limit of
    Eq. (1) with sum_a w_a e_a e_a = I), for each pseudopotential form.  The
    expected psi and psi' are written here from the paper's formulas, and
    psi' is checked against a central difference of psi."""
    def psi_ref(r):
        if kind == 0:
            return 1.0 - np.exp(-r)
        if kind == 1:
            return np.sqrt(p1 * p2) * np.exp(1.0 - p2 / r)
        return p1 * np.exp(-p2 / r)

    def dpsi_ref(r):
        if kind == 0:
            return np.exp(-r)
        return psi_ref(r) * p2 / r ** 2

    r = np.linspace(0.3, 2.0, 7)
    fd = (psi_ref(r + 1e-6) - psi_ref(r - 1e-6)) / 2e-6
    assert np.allclose(dpsi_ref(r), fd, rtol=1e-8)
    kw = dict(psi_kind=kind, psi_p1=p1, psi_p2=p2)
    nx, ny = 24, 20
    o = O.OracleLattice(nx, ny, G=-4.2, tau=1.0, kT=0.0, stencil=stencil, **kw)
    o.init(LN2)
    o.set_density(inputs.perturbed_density(nx, ny, LN2, 0.1, seed=5))
    Fx, Fy = o.force()
    assert abs(Fx.sum()) < 1e-14 and abs(Fy.sum()) < 1e-14
    assert np.abs(Fx).max() > 1e-3                # the force is not trivially zero
    for mx, my in [(1, 0), (0, 1), (1, 1)]:
        errs = []
        for L in (128, 256):
            o = O.OracleLattice(L, L, G=-4.2, tau=1.0, kT=0.0, stencil=stencil, **kw)
            o.init(LN2)
            rho = inputs.sinusoid_density(L, L, LN2, 0.02, mx, my)
            o.set_density(rho)
            Fx, Fy = o.force()
            y, x = np.mgrid[0:L, 0:L]
            ph = 2 * np.pi * (mx * x / L + my * y / L)
            grx = 0.02 * np.cos(ph) * 2 * np.pi * mx / L
            gry = 0.02 * np.cos(ph) * 2 * np.pi * my / L
            ps, dps = psi_ref(rho), dpsi_ref(rho)
            ex_x = 4.2 / 3.0 * ps * dps * grx
            ex_y = 4.2 / 3.0 * ps * dps * gry
            scale = np.abs(np.hypot(ex_x, ex_y)).max()
            errs.append(max(np.abs(Fx - ex_x).max(), np.abs(Fy - ex_y).max()) / scale)
        assert errs[1] < 5e-4
        assert errs[1] < errs[0] / 3.0           # second-order convergence in k


def test_psi_kind2_at_critical_constants_is_eq5():
    """Eq. (4): with a = e sqrt(T_c n_c) and b = n_c the form a exp(-b/n)
    becomes Eq. (5).  The oracle run with kind 2 at those constants must
    reproduce the kind-1 run (same noisy state, same Philox stream) up to
    rounding, and or_psi must agree pointwise."""
    Tc, nc = 0.41, 1.1
    a, b = np.e * np.sqrt(Tc * nc), nc
    p1 = O.make_params(8, 8, -3.0, 1.0, 0.0, psi_kind=1, psi_p1=Tc, psi_p2=nc)
    p2 = O.make_params(8, 8, -3.0, 1.0, 0.0, psi_kind=2, psi_p1=a, psi_p2=b)
    for r in (0.2, 0.7, 1.1, 2.3):
        v1 = O.lib().or_psi(p1, r)
        v2 = O.lib().or_psi(p2, r)
        assert abs(v2 / v1 - 1.0) < 1e-14
    runs = []
    for kind, q1, q2 in [(1, Tc, nc), (2, a, b)]:
        o = O.OracleLattice(32, 24, G=-3.0, tau=0.9, kT=1e-5, stencil=4,
                            psi_kind=kind, psi_p1=q1, psi_p2=q2)
        o.init(1.3, seed=3, init_amp=0.02)
        o.step(40)
        runs.append(o.populations())
    assert np.max(np.abs(runs[1] - runs[0]) / np.abs(runs[0])) < 1e-12
    assert np.max(np.abs(runs[0] - runs[0][:, :1, :1])) > 1e-4   # the state is not flat


def test_flat_equilibrium_stays_flat():
    nx, ny = 20, 16
    o = O.OracleLattice(nx, ny, G=-3.6, tau=0.7, kT=0.0, stencil=8)
    o.init(LN2)
    o.step(100)
    f = o.populations()
    _, _, w, _ = O.lattice_constants()
    for i in range(9):
        assert np.all(f[i] == f[i][0, 0])
        assert abs(f[i][0, 0] - w[i] * LN2) < 1e-15


@pytest.mark.parametrize("stencil", [4, 8])
def test_conservation_with_noise(stencil):
    nx, ny = 36, 20
    o = O.OracleLattice(nx, ny, G=-3.6, tau=0.8, kT=1e-4, stencil=stencil)
    o.init(LN2, seed=9, init_amp=0.01)
    c0 = o.conserved()
    o.step(300)
    c1 = o.conserved()
    assert abs(c1[0] - c0[0]) / c0[0] < 1e-13
    assert abs(c1[1] - c0[1]) < 1e-12 and abs(c1[2] - c0[2]) < 1e-12
    assert abs(c0[1]) < 1e-13 and abs(c0[2]) < 1e-13


@pytest.mark.parametrize("tau", [1.0, 0.75])
def test_noise_variance_is_fdt_amplitude(tau):
    """One step from the flat state: every non-conserved Hermite moment equals
    its noise N_k, whose variance is mu rho0 b_k (1 - gamma^2); conserved
    moments carry no noise.  This is the fluctuation-dissipation reading of
    the noise paragraph after Eq. (16)."""
    nx = ny = 128
    rho0, kT = 1.3, 1e-4
    o = O.OracleLattice(nx, ny, G=0.0, tau=tau, kT=kT)
    o.init(rho0, seed=11)
    o.step(1)
    f = o.populations()
    M, b = O.moment_basis()
    m = np.tensordot(M, f, 1).reshape(9, -1)
    gam = 1.0 - 1.0 / tau
    mu = kT * 3.0
    assert np.abs(m[0] - rho0).max() < 1e-14
    assert np.abs(m[1]).max() < 1e-15 and np.abs(m[2]).max() < 1e-15
    var = m[3:].var(axis=1)
    expect = mu * rho0 * b[3:] * (1 - gam * gam)
    assert np.all(np.abs(var / expect - 1.0) < 0.05)
    cc = np.corrcoef(m[3:])
    assert np.abs(cc - np.eye(6)).max() < 0.04


def test_structure_factor_sum_matches_numpy_fft():
    nx, ny = 16, 8
    o = O.OracleLattice(nx, ny, G=0.0, tau=1.0, kT=0.0)
    o.init(1.0)
    rho = inputs.perturbed_density(nx, ny, 1.0, 0.1, seed=6)
    o.set_density(rho)
    o.sk_reset()
    o.sk_sample_now()
    S, n = o.structure_factor()
    assert n == 1
    d = o.density()
    X = np.fft.rfft2(d - d.mean())
    ref = np.abs(X) ** 2 / (nx * ny)
    ref[0, 0] = 0.0
    assert np.abs(S - ref).max() < 1e-13 * ref.max()


def test_step_sites_equals_lattice_step():
    """The on-demand single-site evaluation used for large-lattice checks gives
    the same numbers as the whole-lattice step."""
    nx, ny = 20, 12
    o = O.OracleLattice(nx, ny, G=-4.5, tau=0.9, kT=1e-4, stencil=6)
    o.init(LN2, seed=3, init_amp=0.02)
    o.step(3)
    f_in = o.populations()
    p = O.make_params(nx, ny, -4.5, 0.9, 1e-4, stencil=6, rho0=LN2, seed=3)
    xs = np.array([0, 5, 19, 0, 19, 7], np.int32)
    ys = np.array([0, 6, 11, 11, 0, 3], np.int32)
    out = O.step_sites(p, 3, f_in, xs, ys)
    o.step(1)
    f1 = o.populations()
    for s in range(len(xs)):
        assert np.array_equal(out[s], f1[:, ys[s], xs[s]])


# --------------------------------------------------------------------------
# Radial read-out of S(k) and its first moments
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 6), (6, 10)])
def test_full_plane_rebuild_matches_numpy_fft(nx, ny):
    """The half plane of |FFT|^2 of a real field, rebuilt by full_plane, equals
    numpy's full |FFT|^2 (S(-k) = S(k) for a real density)."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((ny, nx))
    P = np.abs(np.fft.fft2(x)) ** 2
    assert np.allclose(O.full_plane(P[:, : nx // 2 + 1], nx, ny), P, rtol=1e-13)


@pytest.mark.parametrize("nx,ny", [(16, 16), (32, 8), (8, 24)])
def test_radial_bins_on_a_known_plane(nx, ny):
    """radial_bins of S = |q|^2 + 1 gives in every bin the mean of that value
    over the integer wave vectors with round(|q|) = b, enumerated here from
    numpy's fftfreq; the counts over all bins add up to nx ny - 1 (every mode
    but k = 0)."""
    Lm = max(nx, ny)
    fy = np.fft.fftfreq(ny) * ny * (Lm / ny)
    fx = np.fft.fftfreq(nx) * nx * (Lm / nx)
    if nx % 2 == 0:
        fx[nx // 2] = abs(fx[nx // 2])
    QY, QX = np.meshgrid(fy, fx, indexing="ij")
    val = QX ** 2 + QY ** 2 + 1.0
    half = val[:, : nx // 2 + 1]
    nb = int(np.ceil(np.hypot(nx, ny))) + 2
    means, counts = O.radial_bins(half, nx, ny, nb)
    assert counts.sum() == nx * ny - 1
    expected = {}
    for qy, qx, v in zip(QY.ravel(), QX.ravel(), val.ravel()):
        if qx == 0 and qy == 0:
            continue
        expected.setdefault(int(np.rint(np.hypot(qx, qy))), []).append(v)
    for b in range(nb):
        if b in expected:
            assert counts[b] == len(expected[b])
            assert abs(means[b] - np.mean(expected[b])) < 1e-12 * means[b]
        else:
            assert counts[b] == 0 and np.isnan(means[b])
    # bins past nbins are dropped, the rest unchanged
    m2, c2 = O.radial_bins(half, nx, ny, 3)
    assert np.array_equal(c2, counts[:3])


def test_first_moments_of_a_single_wave():
    """A density cos(2 pi (3x/nx + 2y/ny)) has S(k) only at k = +-(3, 2), so
    the first moments give L = 2 pi sum S / sum |k| S = 1 / |(3/nx, 2/ny)|,
    and sum S = N/2 (Parseval with the N^{-1/2} transform)."""
    nx, ny = 32, 16
    y, x = np.mgrid[0:ny, 0:nx]
    rho = np.cos(2 * np.pi * (3 * x / nx + 2 * y / ny))
    S = np.abs(np.fft.rfft2(rho)) ** 2 / (nx * ny)
    s0, s1 = O.sk_first_moments(S, nx, ny)
    assert abs(s0 - nx * ny / 2) < 1e-9
    L = 2 * np.pi * s0 / s1
    assert abs(L - 1.0 / np.hypot(3 / nx, 2 / ny)) < 1e-12
