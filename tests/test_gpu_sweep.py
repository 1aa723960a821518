"""The battery-cost sweep of Section 3.3 on a small synthetic case: as the battery capital
cost rises, the planned battery expansion does not grow (within SGD noise) and ends far
below where it started, while transmission expansion stays within a band."""
import numpy as np
import pytest

from paper_2410_13055_gb300 import study

pytestmark = pytest.mark.gpu


def test_battery_build_falls_with_cost_other_assets_stable():
    costs = [40.0, 200.0, 400.0, 600.0, 800.0]
    rep = study.battery_cost_sweep(costs=costs, iters=60, batch=2, eval_every=20, S=4, T=24)
    bat = np.array([r["expansion_mw"]["batteries"] for r in rep["rows"]])
    lines = np.array([r["expansion_mw"]["lines"] for r in rep["rows"]])
    assert bat[0] > 0, bat
    # non-increasing up to 5 % of the cheapest cost's build (stochastic gradient noise)
    assert np.all(np.diff(bat) <= 0.05 * bat[0]), bat
    assert bat[-1] <= 0.5 * bat[0], bat
    # transmission: within 25 % of its mean across the sweep
    m = float(np.mean(lines))
    assert m > 0 and np.all(np.abs(lines - m) <= 0.25 * m), lines
