"""Pins of the oracle's LV3 photon pre-filter (Sec. 4.3.4, 6.2.2): a photon is
dropped before the refraction correction when its vacuum straight line lands
farther than radius + margin from the array centre.

The straight line's landing point is fixed independently of the filter: the
same photons (draws keyed by segment, sub-step and bunch) propagated with
refraction off land exactly there.  So the dropped set is checked by brute
force against that run, and the filter's promise -- unchanged detector counts
when the margin covers the correction -- against the unfiltered run."""
import math

import numpy as np

import oracle
from paper_2405_04229_gb300 import synth
from tests import parity_util as PU

ATM = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
HIST = dict(nx=100, ny=100, x0=-50.0, y0=-50.0, dx=1.0, dy=1.0)
TEL = synth.grid_telescopes(nx=3, ny=3, pitch=60.0)


def _key(r):
    return (r["seg"].astype(np.int64) << 24) | (r["k"].astype(np.int64) << 12) | r["i"].astype(np.int64)


def _real(r):
    return r[r["status"] != oracle.ST_SUBSTEP_FLAG]


def _run(segs, refr, lv3=None, spherical=False, **kw):
    return oracle.propagate(segs, ATM, hist=HIST, tel=TEL, bunch=2, refraction=refr, transmission=refr,
                            seed=3, lv3=lv3, spherical=spherical, **kw)


def _paired(a, b):
    ra, rb = _real(a["records"]), _real(b["records"])
    ka, kb = _key(ra), _key(rb)
    assert len(np.unique(ka)) == len(ka)
    assert np.array_equal(np.sort(ka), np.sort(kb))   # the same photons on both runs
    return ra[np.argsort(ka)], rb[np.argsort(kb)]


def test_dropped_set_is_the_straight_line_beyond_the_disc():
    segs = synth.shower_segments(600, 20.0, 30.0, 1e12, seed=2)
    lv3 = dict(centre=(15.0, -10.0, 2000.0), radius=80.0, margin=5.0)
    line = _run(segs, False)
    filt = _run(segs, True, lv3)
    s, f = _paired(line, filt)
    landed = s["status"] == oracle.ST_LANDED
    dist = np.hypot(s["x"] - 15.0, s["y"] + 10.0)
    want = landed & (dist > 85.0)
    got = f["status"] == oracle.ST_LV3
    ok = (f["flags"] & oracle.FL_LV3) == 0
    assert np.array_equal(want[ok], got[ok])
    assert got.sum() > 1000 and (~got & landed).sum() > 1000
    # photons that do not land on the straight line are never the filter's
    assert not (got & ~landed).any()
    PU.check_conservation(filt["counters"])


def test_margin_covering_the_correction_keeps_the_detector_counts():
    segs = synth.shower_segments(600, 20.0, 30.0, 1e12, seed=5)
    line = _run(segs, False)
    full = _run(segs, True)
    s, r = _paired(line, full)
    both = (s["status"] == oracle.ST_LANDED) & np.isin(r["status"], [oracle.ST_LANDED, oracle.ST_ABSORBED])
    shift = float(np.hypot(r["x"] - s["x"], r["y"] - s["y"])[both].max())
    assert 0.0 < shift < 5.0   # the correction moves ground points by less than the margin below
    # a disc holding the histogram and the telescopes' spheres, plus the margin
    radius = max(50.0 * math.sqrt(2.0), float(np.hypot(TEL[:, 0], TEL[:, 1]).max() + TEL[:, 3].max()))
    filt = _run(segs, True, dict(centre=(0.0, 0.0, 2000.0), radius=radius, margin=2.0 * shift + 1.0))
    assert int(np.sum(_real(filt["records"])["status"] == oracle.ST_LV3)) > 0
    assert np.array_equal(filt["hist"], full["hist"])
    assert np.array_equal(filt["tel_counts"], full["tel_counts"])
    cf, cu = filt["counters"], full["counters"]
    assert cf[0] == cu[0] and cf[2] == cu[2] and cf[3] == cu[3]   # emitted, histogram, telescopes
    assert cf[1] <= cu[1]                                         # fewer photons reach the absorption test
    PU.check_conservation(cf)


def test_dropped_sets_shrink_as_the_margin_grows():
    segs = synth.shower_segments(300, 20.0, 30.0, 1e12, seed=7)
    drops = []
    for m in (0.0, 10.0, 40.0):
        r = _real(_run(segs, True, dict(centre=(0.0, 0.0, 2000.0), radius=60.0, margin=m))["records"])
        drops.append(set(_key(r[r["status"] == oracle.ST_LV3]).tolist()))
    assert drops[0] > drops[1] > drops[2]


def test_spherical_dropped_set_is_the_straight_line_chord_beyond_the_disc():
    """On the sphere the landing point is the first crossing of the ground
    sphere; the straight run's azimuthal-equidistant (x, y) map back to it."""
    segs = synth.shower_segments(400, 60.0, 10.0, 1e13, seed=4)
    R, h_obs = oracle.EARTH_RADIUS, 2000.0
    rg = R + h_obs
    lv3 = dict(centre=(0.0, 0.0, h_obs), radius=900.0, margin=0.0)
    line = _run(segs, False, spherical=True, bands=dict(band_pos=0.03))
    filt = _run(segs, True, lv3, spherical=True, bands=dict(band_pos=0.03))
    s, f = _paired(line, filt)
    landed = s["status"] == oracle.ST_LANDED
    rho = np.hypot(s["x"], s["y"])
    a = rho / rg
    sa = np.where(rho > 0, np.sin(a) / np.maximum(rho, 1e-300), 1.0 / rg)
    G = np.stack([rg * sa * s["x"], rg * sa * s["y"], rg * np.cos(a) - R], axis=1)
    dist = np.linalg.norm(G - np.array(lv3["centre"]), axis=1)
    want = landed & (dist > 900.0)
    got = f["status"] == oracle.ST_LV3
    ok = (f["flags"] & oracle.FL_LV3) == 0
    assert np.array_equal(want[ok], got[ok])
    assert got.sum() > 1000 and (~got & landed).sum() > 100
