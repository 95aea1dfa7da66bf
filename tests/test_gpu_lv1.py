"""The LV1 particle filter on the GPU: parity with the oracle for the three
metrics, and a cut fitted on one run's labels drops segments without
changing a single telescope count."""
import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import binding as B
from paper_2405_04229_gb300 import lv1 as L
from paper_2405_04229_gb300 import synth
from tests import parity_util as PU

pytestmark = pytest.mark.gpu

ORC_ATM = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
HIST = synth.histogram_400()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _segs():
    return synth.shower_segments(1500, 30.0, 20.0, 1e12, seed=5, core=(300.0, -200.0))


@pytest.mark.parametrize("metric", [B.CS_LV1_ARRAY_CENTRE, B.CS_LV1_ARRAY_DISC, B.CS_LV1_TELESCOPES])
def test_filter_parity_with_oracle(metric):
    segs = _segs()
    tel = synth.grid_telescopes(nx=4, ny=4, pitch=150.0)
    # a cut through the middle of the segments' (x, y) cloud: about 40 % dropped
    x, y = L.cut_parameters(segs, metric, centre=(0.0, 0.0, 2000.0), radius=350.0, tel=tel)
    b = -0.6
    a = float(np.quantile(y / x ** b, 0.6))
    cfg = dict(metric=metric, a=a, b=b, centre=(0.0, 0.0, 2000.0), radius=350.0)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    det = B.Detector(hist=HIST, tel=tel)
    g = B.propagate_host(segs, atm, det, seed=3, bunch=2, records=True, lv1=cfg)
    o = oracle.propagate(segs, ORC_ATM, hist=HIST, tel=tel, bunch=2, refraction=True, transmission=True, seed=3,
                         lv1=dict(cfg, band=1e-4))
    assert 0 < g["lv1_dropped"] < len(segs["z0"])
    near = len({int(s) for s in o["records"]["seg"][(o["records"]["flags"] & oracle.FL_LV1) != 0]})
    assert abs(g["lv1_dropped"] - o["lv1_dropped"]) <= near
    assert abs(g["lv1_dropped"] / len(segs["z0"]) - 0.4) < 0.05
    st = PU.compare(g, o, bunch=2)
    assert st["matched"] > 3000


def test_fitted_cut_keeps_every_telescope_count():
    segs = _segs()
    tel = synth.grid_telescopes(nx=4, ny=4, pitch=150.0)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    det = B.Detector(hist=HIST, tel=tel)
    full = B.propagate_host(segs, atm, det, seed=8, bunch=2, records=True)
    keep = L.contributing(full["records"], len(segs["z0"]))
    assert keep.any()
    for metric in (B.CS_LV1_ARRAY_DISC, B.CS_LV1_TELESCOPES):
        x, y = L.cut_parameters(segs, metric, centre=(0.0, 0.0, 2000.0), radius=350.0, tel=tel)
        cut = L.fit_cut(x, y, keep, margin=1.1)
        assert cut["removed"] > 0.05
        cfg = dict(metric=metric, a=cut["a"], b=cut["b"], centre=(0.0, 0.0, 2000.0), radius=350.0)
        f = B.propagate_host(segs, atm, det, seed=8, bunch=2, lv1=cfg)
        assert f["lv1_dropped"] > 0
        assert np.array_equal(f["tel_counts"], full["tel_counts"])
        np.testing.assert_allclose(f["tel_time"], full["tel_time"], rtol=1e-12)
        assert int(f["counters"][0]) < int(full["counters"][0])
