"""Pins of the oracle's LV1 particle filter (Sec. 4.3.2; the cut y / x^b < a
of Sec. 6.2.1): the dropped set equals a numpy evaluation of the angles and
the cut, and the photons of the kept segments are exactly those of the
unfiltered run."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import synth

ATM = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
H_OBS = 2000.0


def _angles(segs, centres, radii):
    """x [deg]: smallest angle between each segment's direction and the
    spheres (centre, radius), less their angular radius (numpy, FP64)."""
    S = np.stack([segs["x0"], segs["y0"], segs["z0"]], 1)
    P = np.stack([segs["ux"], segs["uy"], segs["uz"]], 1).astype(np.float64)
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    best = np.full(len(S), 180.0)
    for C, r in zip(centres, radii):
        d = np.asarray(C)[None, :] - S
        dn = np.linalg.norm(d, axis=1)
        a = np.degrees(np.arccos(np.clip(np.sum(P * d, 1) / dn, -1, 1)) - np.arcsin(np.minimum(r / dn, 1.0)))
        best = np.minimum(best, np.where(dn > r, np.maximum(a, 0.0), 0.0))
    return best


def test_angle_geometry_special_cases():
    s = synth._empty(3)
    s["x0"][:] = [0.0, 1000.0, 1000.0]
    s["z0"][:] = [10000.0, 3000.0, 3000.0]
    s["uz"][:] = -1.0
    s["length"][:] = 1.0
    s["inv_gamma2"][:] = np.float32(1e-8)
    x = _angles(s, [(0.0, 0.0, H_OBS)], [0.0])
    assert x[0] == pytest.approx(0.0, abs=1e-9) and x[1] == pytest.approx(45.0, abs=1e-9)
    x = _angles(s, [(0.0, 0.0, H_OBS)], [500.0])
    assert x[1] == pytest.approx(45.0 - math.degrees(math.asin(500.0 / math.hypot(1000.0, 1000.0))), abs=1e-9)


@pytest.mark.parametrize("metric", [oracle.LV1_ARRAY_CENTRE, oracle.LV1_ARRAY_DISC, oracle.LV1_TELESCOPES])
def test_dropped_set_and_kept_photons(metric):
    segs = synth.shower_segments(400, 30.0, 20.0, 1e12, seed=5, core=(300.0, -200.0))
    tel = synth.grid_telescopes(nx=4, ny=4, pitch=150.0)
    centre, radius = (0.0, 0.0, H_OBS), 350.0
    a, b = 2500.0, -0.6
    lv1 = dict(metric=metric, a=a, b=b, centre=centre, radius=radius, band=0.0)
    kw = dict(hist=synth.histogram_400(), tel=tel, bunch=2, refraction=True, transmission=True, seed=3)
    full = oracle.propagate(segs, ATM, **kw)
    cut = oracle.propagate(segs, ATM, lv1=lv1, **kw)
    if metric == oracle.LV1_TELESCOPES:
        x = _angles(segs, [t[:3] for t in tel], [t[3] for t in tel])
    else:
        x = _angles(segs, [centre], [radius if metric == oracle.LV1_ARRAY_DISC else 0.0])
    y = segs["z0"] - H_OBS
    drop = y >= a * np.maximum(x, 1e-3) ** b
    assert 0 < drop.sum() < len(drop)
    assert cut["lv1_dropped"] == int(drop.sum())
    kept = np.flatnonzero(~drop)
    fr, cr = full["records"], cut["records"]
    sel = np.isin(fr["seg"], kept)
    assert len(cr) == int(sel.sum())
    for f in ("seg", "k", "i", "status", "tel", "bin"):
        assert np.array_equal(cr[f], fr[f][sel]), f
    np.testing.assert_array_equal(cr["x"], fr["x"][sel])
    real = sel & (fr["status"] != oracle.ST_SUBSTEP_FLAG)
    assert int(cut["counters"][0]) == int(real.sum()) * 2   # emitted photons of the kept segments
