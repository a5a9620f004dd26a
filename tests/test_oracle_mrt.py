"""Pins of the oracle's multiple-relaxation-time collision (the variant of
the BGK collision with separate bulk, shear and ghost rates)."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import theory as T

LN2 = float(np.log(2.0))


def test_moment_path_with_one_rate_is_bgk():
    a = O.OracleLattice(36, 20, -3.6, 0.8, 1e-4, stencil=6)
    b = O.OracleLattice(36, 20, -3.6, 0.8, 1e-4, stencil=6, force_mrt=1)
    for o in (a, b):
        o.init(LN2, 4, 0.01)
        o.step(100)
    fa, fb = a.populations(), b.populations()
    assert np.max(np.abs(fa - fb) / np.abs(fa)) < 1e-13


@pytest.mark.parametrize("tau_b,tau_g", [(1.4, 1.1), (0.6, 1.9)])
def test_shear_wave_decays_at_the_shear_viscosity(tau_b, tau_g):
    """A transverse momentum wave j_x ~ sin(k y) decays as exp(-nu k^2 t),
    nu = c_s^2 (tau - 1/2), whatever the bulk and ghost rates."""
    nx, ny, tau, rho0 = 4, 128, 0.8, 1.0
    o = O.OracleLattice(nx, ny, 0.0, tau, 0.0, tau_bulk=tau_b, tau_ghost=tau_g)
    o.init(rho0)
    cx, cy, w, _ = O.lattice_constants()
    y = np.arange(ny)
    k = 2 * np.pi / ny
    jx = 1e-4 * np.sin(k * y)
    f = np.array([w[i] * (rho0 + 3.0 * cx[i] * jx[:, None] * np.ones((1, nx))) for i in range(9)])
    o.set_populations(f)

    def amp():
        fp = o.populations()
        j = np.tensordot(cx.astype(float), fp, 1)[:, 0]
        return (j * np.sin(k * y)).sum()

    o.step(200)                       # let the non-hydrodynamic modes die out
    a1 = amp()
    o.step(2000)
    a2 = amp()
    rate = np.log(a1 / a2) / 2000
    nu = (tau - 0.5) / 3.0
    assert abs(rate / (nu * k * k) - 1.0) < 5e-3


def test_mrt_ideal_gas_structure_factor_is_flat():
    L, rho0, kT = 32, LN2, 1e-4
    o = O.OracleLattice(L, L, 0.0, 0.8, kT, tau_bulk=1.5, tau_ghost=0.7)
    o.init(rho0, seed=7)
    o.step(500)
    o.sk_config(2, o.t + 2)
    o.step(6000)
    S, n = o.structure_factor()
    S = S / (rho0 * kT * 3.0)
    S[0, 0] = np.nan
    assert abs(np.nanmean(S) - 1.0) < 0.015


def test_mrt_structure_factor_matches_exact_theory_on_axes():
    """Eq. (16) on lattice axes holds for any set of relaxation rates."""
    L, nb, G, rho0, kT = 32, 10, -3.6, LN2, 1e-5
    o = O.OracleLattice(L, L, G, 0.8, kT, tau_bulk=1.3, tau_ghost=1.1)
    o.init(rho0, seed=11)
    o.step(2000)
    B = []
    for _ in range(nb):
        o.sk_reset()
        o.sk_config(5, o.t + 5)
        o.step(3000)
        B.append(o.structure_factor()[0])
    B = np.array(B)
    ratios, z = [], []
    for m in range(2, L // 2 + 1):
        vals = (B[:, 0, m] + B[:, m, 0]) / 2
        th = T.sk_axis(2 * np.pi * m / L, rho0, G, kT)
        ratios.append(vals.mean() / th)
        z.append((vals.mean() - th) / (vals.std(ddof=1) / np.sqrt(nb)))
    assert np.all(np.abs(z) < 5.0) and abs(np.mean(ratios) - 1.0) < 0.01
