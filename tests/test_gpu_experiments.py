"""The structure-factor experiments of the paper's Figs. 2 and 3 on FP32
ensembles (32 replicas of 128^2 per state, 30000 steps, S(k) sampled over
the last 20000): S(k -> 0) from the axis modes against the exact long-
wavelength theory, and its scaling exponents against the theory's on the
same state points, approaching the spinodal along the G = -4.5 isotherm
(both metastable branches, Fig. 2 top and Fig. 3), approaching the critical
point on the critical isochore rho_c = ln 2 from above (T_hat -> 1+,
exponent -1), and along the binodal from below (Fig. 2 bottom)."""
import numpy as np
import pytest

from oracle import theory as T
from pairs import LN2

pytestmark = pytest.mark.gpu
KT = 1e-6


def _s0_theory(rho, G):
    return float(T.sk_axis(np.array([1e-9]), rho, G, KT)[0])


@pytest.fixture(scope="module")
def runs():
    from paper_2212_07848_gb300 import experiments as X
    G = -4.5
    rs_g, rs_l = T.spinodal(G)
    rc_g, rc_l = T.coexistence(G, eps=0.0)
    fr = [0.2, 0.4, 0.6, 0.75, 0.85]
    spin = [(G, rc_g + f * (rs_g - rc_g)) for f in fr] + [(G, rc_l - f * (rc_l - rs_l)) for f in fr]
    iso = [(g, LN2) for g in (-3.2, -3.5, -3.7, -3.8, -3.9)]
    bino = [(g, T.coexistence(g, eps=0.0)[0]) for g in (-4.8, -4.6, -4.4, -4.3, -4.2)]
    states = spin + iso + bino
    k, mean, sem = X.axis_structure_factor(states, L=128, steps=30000, start=10000,
                                           seeds_per_state=32, kT=KT, seed=21)
    s0 = [X.s0_from_axis(k, mu, slice(0, 8), se)[0] for mu, se in zip(mean, sem)]
    return X, G, (rs_g, rs_l), states, np.array(s0), len(spin), len(iso)


def test_s0_matches_theory_at_every_state(runs):
    X, G, _, states, s0, _, _ = runs
    th = np.array([_s0_theory(r, g) for g, r in states])
    rel = s0 / th - 1
    assert np.abs(rel).max() < 0.03, list(zip(states, np.round(rel, 4)))


def test_spinodal_exponents(runs):
    """S(0) against the pressure distance to the spinodal on each branch:
    the fitted exponent matches the theory's over the same points (the
    asymptotic value is -1/2, approached as the last points near the spinodal)."""
    X, G, (rs_g, rs_l), states, s0, nspin, _ = runs
    for branch, rs in ((slice(0, 5), rs_g), (slice(5, 10), rs_l)):
        rho = np.array([r for _, r in states[branch]])
        dp = np.abs(T.pressure(rho, G) - T.pressure(rs, G))
        p_meas = X.power_law(dp, s0[branch])[0]
        p_th = X.power_law(dp, [_s0_theory(r, G) for r in rho])[0]
        assert abs(p_meas - p_th) < 0.03, (p_meas, p_th)
        assert -0.75 < p_meas < -0.35


def test_critical_isochore_exponent(runs):
    """S(0) on rho_c = ln 2 against T_hat - 1 = -4/G - 1: exponent -1 (mean
    field, Eq. (8) with n_hat = 1)."""
    X, _, _, states, s0, nspin, niso = runs
    iso = slice(nspin, nspin + niso)
    t = np.array([-4.0 / g - 1.0 for g, _ in states[iso]])
    p_meas = X.power_law(t, s0[iso])[0]
    p_th = X.power_law(t, [_s0_theory(r, g) for g, r in states[iso]])[0]
    assert abs(p_meas - p_th) < 0.05, (p_meas, p_th)
    assert abs(p_meas + 1.0) < 0.15, p_meas
