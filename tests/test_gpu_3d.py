"""The D3Q19 step on the GPU against the FP64 oracle: FP64 to 1e-12 and FP32
to 1e-4 per site, with noise, force and ragged z strips; exact flat
equilibrium; conservation; the axis S(k) against the oracle's on the same
noise; and an FP32 ensemble of replicas against Eq. (16) on the axes."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import theory as T
from pairs import LN2, max_rel

pytestmark = pytest.mark.gpu


def _pair(nx, ny, nz, G, tau, kT, precision, rho0, seed, amp, replica=0, strip=None, kind=0,
          p1=0.0, p2=0.0):
    from paper_2212_07848_gb300.lattice3 import Lattice3
    g = Lattice3(nx, ny, nz, G, tau, kT, precision=precision, psi_kind=kind, psi_p1=p1,
                 psi_p2=p2)
    if strip:
        g.set_strip(strip)
    g.set_replica(replica)
    g.init(rho0, seed, amp)
    o = O.OracleLattice3(nx, ny, nz, G, tau, kT, replica=replica, psi_kind=kind, psi_p1=p1,
                         psi_p2=p2)
    o.init(rho0, seed, amp)
    return g, o


@pytest.mark.parametrize("nx,ny,nz,G,tau,kT,rho0,amp,strip,steps", [
    (32, 8, 6, -3.6, 1.0, 1e-4, LN2, 0.01, None, 200),
    (64, 16, 12, -4.5, 0.8, 1e-5, 0.33, 0.005, 5, 100),     # several tiles, ragged strips
    (32, 16, 7, -4.0, 1.3, 0.0, 0.7, 0.02, 3, 100),          # no noise, odd nz
])
def test_fp64_matches_oracle(nx, ny, nz, G, tau, kT, rho0, amp, strip, steps):
    g, o = _pair(nx, ny, nz, G, tau, kT, "fp64", rho0, 17, amp, replica=2, strip=strip)
    g.step(steps)
    o.step(steps)
    assert max_rel(g.populations(), o.populations()) < 1e-12
    assert max_rel(g.density(), o.density()) < 1e-12


@pytest.mark.parametrize("kind,p1,p2,rho0", [(1, 5.0 / 12.0, 1.0, 0.5), (2, 1.3, 0.8, 0.9)])
def test_pseudopotential_kinds_match_oracle(kind, p1, p2, rho0):
    """Eq. (5) (kind 1, T_hat = 0.8 at G = -3, a stable gas) and a exp(-b/rho)
    (kind 2), both on stable homogeneous states."""
    for prec, tol, steps in (("fp64", 1e-12, 150), ("fp32", 1e-4, 100)):
        g, o = _pair(32, 8, 8, -3.0, 1.0, 1e-5, prec, rho0, 9, 0.01, kind=kind, p1=p1, p2=p2)
        g.step(steps)
        o.step(steps)
        assert max_rel(g.populations(), o.populations()) < tol, prec
        assert max_rel(g.density(), o.density()) < tol, prec


# FP32 tiles are 32 x 8 when ny is a multiple of 8, else 32 x 4; tau = 1
# takes the unit-relaxation path
@pytest.mark.parametrize("nx,ny,nz,tau", [(32, 16, 8, 1.0), (32, 12, 8, 1.0), (64, 20, 6, 0.8),
                                          (32, 24, 7, 0.9)])
def test_fp32_matches_oracle(nx, ny, nz, tau):
    g, o = _pair(nx, ny, nz, -4.2, tau, 1e-5, "fp32", 0.6, 4, 0.005)
    g.step(100)
    o.step(100)
    assert max_rel(g.populations(), o.populations()) < 1e-4
    assert max_rel(g.density(), o.density()) < 1e-4


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_flat_equilibrium_exact_and_conservation(precision):
    from paper_2212_07848_gb300.lattice3 import Lattice3
    g = Lattice3(32, 8, 8, -4.5, 0.9, 0.0, precision=precision)
    g.init(0.4)
    f0 = g.populations()
    g.step(20)
    assert np.array_equal(g.populations(), f0)
    g = Lattice3(32, 16, 8, -3.8, 0.9, 1e-4, precision=precision)
    g.init(LN2, 3, 0.02)
    c0 = g.conserved()
    g.step(300)
    c1 = g.conserved()
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert abs(c1[0] - c0[0]) < tol * c0[0]
    assert np.abs(c1[1:] - c0[1:]).max() < tol * c0[0]


def test_axis_structure_factor_matches_oracle():
    g, o = _pair(32, 8, 8, -3.6, 1.0, 1e-4, "fp64", LN2, 5, 0.0)
    g.sk_config(1, 50)
    o.sk_config(1, 50)
    g.step(120)
    o.step(120)
    Sg, ng = g.structure_factor_axes()
    So, no = o.structure_factor_axes()
    assert ng == no == 71
    assert np.abs(Sg - So).max() < 1e-9 * np.abs(So).max()


def test_fp32_replicas_match_eq16_on_axes():
    """Eight replicas of 32^3 (supercritical C1 state): axis modes agree with
    Eq. (16) within 3% or 4 standard errors."""
    from paper_2212_07848_gb300.lattice3 import Lattice3
    L, G, kT, steps, start = 32, -3.6, 1e-5, 4000, 1001
    vals = []
    for r in range(8):
        g = Lattice3(L, L, L, G, 1.0, kT)
        g.set_replica(r)
        g.init(LN2, 31, 0.0)
        g.sk_config(1, start)
        g.step(steps)
        S, n = g.structure_factor_axes()
        assert n == steps - start + 1
        vals += [S[a * (L // 2):(a + 1) * (L // 2)] for a in range(3)]
        g.close()
    v = np.array(vals)
    m = np.arange(1, L // 2 + 1)
    th = T.sk_axis(2 * np.pi * m / L, LN2, G, kT)
    mean, sem = v.mean(axis=0), v.std(axis=0, ddof=1) / np.sqrt(len(v))
    sel = m >= 2
    dev = np.abs(mean - th)
    assert ((dev <= 0.03 * th) | (dev <= 4 * sem))[sel].all(), np.round(mean / th - 1, 3)


def test_full_structure_factor_matches_oracle():
    """The full 3D S(k) (FFTs along x, y, z on the device) in FP64 against the
    oracle's separable DFT on the same noise: radial shells and the first
    moments behind L = 2 pi sum S / sum |k| S."""
    nx, ny, nz = 32, 8, 8
    g, o = _pair(nx, ny, nz, -3.6, 1.0, 1e-4, "fp64", LN2, 5, 0.0)
    g.sk_config(1, 20)
    g.sk_full()
    o.sk_config(1, 20)
    o.sk_full()
    g.step(60)
    o.step(60)
    So, no = o.structure_factor_full()
    ref = O.radial_bins3(So)
    got, ng = g.structure_factor(len(ref))
    assert ng == no == 41
    assert np.abs(got - ref).max() < 1e-9 * ref.max()
    fold = lambda n: np.where(np.arange(n) <= n // 2, np.arange(n), np.arange(n) - n)
    kz, ky, kx = np.meshgrid(fold(nz) / nz, fold(ny) / ny, fold(nx) / nx, indexing="ij")
    kabs = 2 * np.pi * np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    m = g.sk_moments()
    assert abs(m[0] - So.sum()) < 1e-9 * So.sum()
    assert abs(m[1] - (kabs * So).sum()) < 1e-9 * (kabs * So).sum()


def test_full_structure_factor_fp32_one_sample_matches_fft():
    """FP32, 64^3: one sample of the device S(k) against numpy's FFT of the
    lattice's own density at that step (radial shells, domain size)."""
    from paper_2212_07848_gb300.lattice3 import Lattice3
    n, T = 64, 200
    g = Lattice3(n, n, n, -3.6, 1.0, 1e-5)
    g.init(LN2, 11, 0.01)
    g.sk_config(1, T)
    g.sk_full()
    g.step(T)
    rho = g.density()
    S = np.abs(np.fft.fftn(rho - rho.mean())) ** 2 / rho.size
    ref = O.radial_bins3(S)
    got, ns = g.structure_factor(len(ref))
    assert ns == 1
    rel = np.abs(got[1:] - ref[1:]) / ref[1:]
    assert rel.max() < 1e-3, rel.max()
    fold = np.where(np.arange(n) <= n // 2, np.arange(n), np.arange(n) - n) / n
    kz, ky, kx = np.meshgrid(fold, fold, fold, indexing="ij")
    kabs = 2 * np.pi * np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    L_ref = 2 * np.pi * S.sum() / (kabs * S).sum()
    assert abs(g.domain_size() / L_ref - 1.0) < 1e-4
    g.close()
