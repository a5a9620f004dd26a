"""Unstable-branch quench at G = -5.0 (T_hat = 0.8): spinodal decomposition
coarsens (L(t) grows) into isolated droplets for a gas-rich density, while a
near-symmetric density gives a minority phase that percolates across the
periodic box (a slab, or a bicontinuous network on its way to one) whose
domain size reaches the box scale; mass is conserved throughout."""
import numpy as np
import pytest

from oracle import theory as T

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,steps,every,rho0,expect", [(128, 8000, 500, 0.45, ("droplet",)),
                                                         (64, 20000, 1250, 0.95, ("stripe", "mixed"))])
def test_quench_topology_and_coarsening(n, steps, every, rho0, expect):
    from paper_2212_07848_gb300.quench import run_quench
    sg, sl = T.spinodal(-5.0)
    assert sg < rho0 < sl                                  # inside the unstable region
    res = run_quench(n, n, -5.0, rho0, kT=1e-5, steps=steps, every=every, seed=3)
    assert res["topology"] in expect, (res["topology"], res["liquid_fraction"])
    L = res["L"]
    assert np.all(np.isfinite(L))
    if expect == ("droplet",):
        assert L[-1] > 1.5 * L[1]          # droplets coarsen
    else:
        assert L[-1] > 0.5 * n             # the percolating phase spans the box
    assert abs(res["density"].mean() - rho0) < 1e-4
