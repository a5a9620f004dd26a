"""3D unstable-branch quenches on the Eq. (5) isotherm T_hat = 0.8 (Fig. 1,
upper panels) at 64^3: the low-density side ends as a droplet, the middle as
a flat slab, the side next to the upper spinodal on the bubble side; the
liquid fraction follows the lever rule of the measured coexisting densities
and mass is conserved."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_hat,allowed", [
    (0.67, {"droplet"}),
    (1.3, {"flat"}),
    (1.64, {"bubble", "bubble-cylinder"}),
])
def test_quench_topology(n_hat, allowed):
    import numpy as np
    from paper_2212_07848_gb300 import quench3 as Q
    r = Q.run_quench3(64, Q.EQ5_G, n_hat, kT=1e-6, steps=10000, seed=1, psi_kind=1,
                      psi_p1=Q.EQ5_TC, psi_p2=Q.EQ5_NC)
    assert r["topology"] in allowed, r["topology"]
    lo, hi = np.percentile(r["density"], [1.0, 99.0])
    assert 0.40 < lo < 0.48 and 2.3 < hi < 2.5          # coexistence near 0.43 / 2.4
    lever = (n_hat - lo) / (hi - lo)
    assert abs(r["liquid_fraction"] - lever) < 0.02
    assert r["mass_drift"] < 1e-5


def test_quench_domain_size_grows():
    """S(k, t) of a 64^3 quench from the full 3D S(k): L(t) grows with t and
    power moves into the longest-wavelength shell."""
    from paper_2212_07848_gb300 import quench3 as Q
    r = Q.run_quench3(64, Q.EQ5_G, 1.3, kT=1e-6, steps=3000, seed=1, psi_kind=1,
                      psi_p1=Q.EQ5_TC, psi_p2=Q.EQ5_NC, every=500)
    L = r["L"]
    assert len(L) == 6 and all(x > 0 for x in L)
    assert L[-1] > 1.5 * L[0]
    assert r["S"][-1, 1] > 2.0 * r["S"][0, 1]
