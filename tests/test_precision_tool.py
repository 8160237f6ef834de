"""Host-side statistics of the precision comparison tool."""

import numpy as np

from paper_0812_2801_gb300 import precision


def test_drift_statistics():
    steps = np.arange(0, 1001, 10)
    E = -100.0 + 2e-6 * steps / 1000.0 + 1e-7 * np.sin(steps / 30.0)
    d = precision._drift(E, steps)
    assert abs(d["drift_rel"] - abs(E[-1] - E[0]) / 100.0) < 1e-15
    assert abs(d["slope_rel_1000"] - 2e-8) < 2e-9          # the linear part
    assert d["max_dev_rel"] >= d["drift_rel"]


def test_relative_force_error_uses_the_largest_force():
    F = np.array([[0.0, 0.0, 2.0], [0.0, 1.0, 0.0]])
    G = F + np.array([[0.0, 0.0, 1e-3], [0.0, 0.0, 0.0]])
    assert abs(precision._rel_force_err(G, F) - 5e-4) < 1e-15
