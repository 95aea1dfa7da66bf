"""Parity of the LV3 photon pre-filter (Sec. 4.3.4, 6.2.2) with the FP64 oracle,
photon by photon on the planar and the spherical path, and its promise: with
a disc that holds the detectors and a margin that covers the refraction
correction, the detector counts do not change."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import binding as B
from paper_2405_04229_gb300 import synth
from tests import parity_util as PU

pytestmark = pytest.mark.gpu

ORC_ATM = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
HIST = dict(nx=100, ny=100, x0=-50.0, y0=-50.0, dx=1.0, dy=1.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _tel():
    return synth.grid_telescopes(nx=3, ny=3, pitch=60.0)


@pytest.mark.parametrize("refr", [True, False])
def test_planar_lv3_parity(refr):
    segs = synth.shower_segments(2000, 20.0, 30.0, 1e12, seed=2)
    lv3 = dict(centre=(15.0, -10.0, 2000.0), radius=300.0, margin=5.0)
    tel = _tel()
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=refr, transmission=refr)
    det = B.Detector(hist=HIST, tel=tel)
    g = B.propagate_host(segs, atm, det, seed=3, bunch=2, records=True, lv3=lv3)
    o = oracle.propagate(segs, ORC_ATM, hist=HIST, tel=tel, bunch=2, refraction=refr, transmission=refr,
                         seed=3, lv3=lv3)
    st = PU.compare(g, o, bunch=2)
    assert st["matched"] > 10000
    n_lv3 = int((g["records"]["status"] == B.CS_ST_LV3).sum())
    assert n_lv3 > 2000 and n_lv3 < 0.9 * len(g["records"])
    PU.check_conservation(g["counters"])


def test_spherical_lv3_parity():
    segs = synth.shower_segments(1500, 60.0, 10.0, 1e13, seed=4)
    lv3 = dict(centre=(0.0, 0.0, 2000.0), radius=900.0, margin=20.0)
    tel = _tel()
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True, spherical=True)
    det = B.Detector(hist=HIST, tel=tel, spherical=True)
    g = B.propagate_host(segs, atm, det, seed=4, bunch=2, records=True, lv3=lv3)
    o = oracle.propagate(segs, ORC_ATM, hist=HIST, tel=tel, bunch=2, refraction=True, transmission=True, seed=4,
                         spherical=True, lv3=lv3, bands=dict(band_pos=0.03))
    st = PU.compare(g, o, bunch=2)
    assert st["matched"] > 10000
    assert int((g["records"]["status"] == B.CS_ST_LV3).sum()) > 2000
    PU.check_conservation(g["counters"])


@pytest.mark.parametrize("spherical", [False, True])
def test_covering_disc_keeps_the_detector_counts(spherical):
    zen = 60.0 if spherical else 20.0
    segs = synth.shower_segments(20000, zen, 30.0, 1e13, seed=6)
    tel = _tel()
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True, spherical=spherical)
    det = B.Detector(hist=HIST, tel=tel, spherical=spherical)
    full = B.propagate_host(segs, atm, det, seed=5, bunch=3)
    # the histogram's corners lie 71 m from the centre; a photon that hits a sphere
    # (centre 85 m out, radius 6 m) lands within 6 m / cos(60 deg) of it; the correction
    # moves these showers' ground points by under 1 m (20 deg) and 30 m (60 deg)
    lv3 = dict(centre=(0.0, 0.0, 2000.0), radius=math.hypot(60.0, 60.0) + 12.0, margin=80.0 if spherical else 10.0)
    filt = B.propagate_host(segs, atm, det, seed=5, bunch=3, lv3=lv3)
    assert np.array_equal(filt["hist"], full["hist"])
    assert np.array_equal(filt["tel_counts"], full["tel_counts"])
    assert filt["counters"][B.CS_CNT_ABSORBED] < full["counters"][B.CS_CNT_ABSORBED]
    PU.check_conservation(filt["counters"])


def test_lv3_with_the_surrogate_and_invalid_arguments():
    segs = synth.shower_segments(500, 20.0, 30.0, 1e12, seed=8)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    det = B.Detector(hist=HIST, tel=_tel())
    lv3 = dict(centre=(0.0, 0.0, 2000.0), radius=60.0, margin=2.0)
    exact = B.propagate_host(segs, atm, det, seed=1, bunch=2, records=True, lv3=lv3)
    sur = B.Surrogate(atm, epochs=2, n_train=1 << 16, n_heldout=1 << 12)
    s = B.propagate_host(segs, atm, det, seed=1, bunch=2, records=True, lv3=lv3, surrogate=sur)
    sur.close()
    # the filter decides on the straight line, before the network or the tables
    ke = np.sort(exact["records"][exact["records"]["status"] == B.CS_ST_LV3]["seg"])
    ks = np.sort(s["records"][s["records"]["status"] == B.CS_ST_LV3]["seg"])
    assert len(ke) > 0 and np.array_equal(ke, ks)
    with pytest.raises(RuntimeError):
        B.propagate_host(segs, atm, det, seed=1, bunch=2, lv3=dict(centre=(0, 0, 2000.0), radius=-1.0))
