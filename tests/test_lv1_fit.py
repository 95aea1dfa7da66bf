"""The LV1 cut fit (host logic): every segment marked to keep survives the
fitted cut, and the cut removes what it reports."""
import numpy as np

from paper_2405_04229_gb300 import lv1


def test_fit_keeps_every_marked_segment():
    rng = np.random.default_rng(3)
    x = rng.uniform(0.01, 60.0, 20000)
    y = rng.uniform(10.0, 20000.0, 20000)
    keep = y * x ** 1.3 < 4.0e4          # the "contributing" region: a power-law boundary
    cut = lv1.fit_cut(x, y, keep, margin=1.05)
    dropped = y >= cut["a"] * x ** cut["b"]
    assert not (dropped & keep).any()
    assert abs(dropped.mean() - cut["removed"]) < 1e-12
    assert cut["removed"] > 0.8 * (~keep).mean()       # close to the best possible
    assert -1.5 < cut["b"] < -1.1                       # the boundary's slope


def test_fit_with_nothing_to_keep_removes_everything():
    x = np.linspace(0.1, 10, 100)
    y = np.linspace(10, 1000, 100)
    cut = lv1.fit_cut(x, y, np.zeros(100, bool))
    assert cut["removed"] == 1.0
