"""Parity of the cylindrical atmosphere (Sec. 3.3.3) on the GPU with the FP64
oracle, photon by photon: the kernel traces every photon with the Snell
stepper through the coaxial cylinders of its own axis (scalar invariant form)
and lays its ground point on the unrolled ground cylinder; the oracle runs
the same stepper in three-dimensional vector form, and the exact quadrature
for straight lines.  Showers from 20 to 70 degrees with cores up to 15 km
from the array centre, so that the axes turn from photon to photon.

Edge band: as on the sphere, ground points of long slant paths carry FP32
ulps of a few mm, so bin and sphere edges are flagged within 0.03 m."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import binding as B
from paper_2405_04229_gb300 import synth
from tests import parity_util as PU

pytestmark = pytest.mark.gpu

ORC_ATM = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
HIST = synth.histogram_400()
BANDS = dict(band_pos=0.03)
DH = 10.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _showers(n_each, seed):
    parts = []
    for i, (zen, az, core) in enumerate([(20.0, 30.0, (0.0, 0.0)), (45.0, 200.0, (12000.0, -5000.0)),
                                         (60.0, 110.0, (-8000.0, 9000.0)), (70.0, 300.0, (3000.0, 15000.0))]):
        parts.append(synth.shower_segments(n_each, zen, az, 1e12, seed, shower_id=i, core=core))
    return synth.concat(parts)


def _tel():
    return synth.poisson_disk_telescopes(n=300, half=3000.0, min_sep=40.0, radius=6.0, seed=2)


def _run(segs, refr, trans, bunch, seed, fluorescence=None, hist=HIST):
    tel = _tel()
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=refr, transmission=trans, cylindrical=True)
    det = B.Detector(hist=hist, tel=tel, cylindrical=True)
    g = B.propagate_host(segs, atm, det, seed=seed, bunch=bunch, records=True, snell_dh=DH,
                         fluorescence=fluorescence)
    o = oracle.propagate(segs, ORC_ATM, hist=hist, tel=tel, bunch=bunch, refraction=refr, transmission=trans,
                         seed=seed, cylindrical=True, snell_dh=DH, bands=BANDS, fluorescence=fluorescence)
    return g, o


@pytest.mark.parametrize("refr,trans", [(True, True), (True, False), (False, True)])
def test_cylinder_parity(refr, trans):
    segs = _showers(1500, seed=11)
    g, o = _run(segs, refr, trans, bunch=2, seed=5)
    st = PU.compare(g, o, bunch=2)
    assert st["matched"] > 30_000, st
    assert int(g["counters"][3]) > 0 and int(g["counters"][2]) > 0
    PU.check_conservation(g["counters"])
    np.testing.assert_array_equal(g["counters"][[0, 6, 7]], o["counters"][[0, 6, 7]])


def test_axial_drift_reaches_the_ground_points():
    """The unrolled ground point differs from the sphere's by the axial drift's
    effect: for the 70-degree shower the cylinder and the shell disagree by more
    than the parity bar, and the cylinder's points are the oracle's."""
    segs = _showers(1500, seed=12)
    g, o = _run(segs, True, False, bunch=1, seed=6)
    PU.compare(g, o, bunch=1)
    atm_s = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=False, spherical=True)
    det_s = B.Detector(hist=HIST, tel=_tel(), spherical=True)
    s = B.propagate_host(segs, atm_s, det_s, seed=6, bunch=1, records=True, snell_dh=DH)
    gr, sr = g["records"], s["records"]
    key = lambda r: (r["seg"].astype(np.int64) << 32) | (r["k"].astype(np.int64) << 16) | r["i"].astype(np.int64)
    common, ia, ib = np.intersect1d(key(gr), key(sr), return_indices=True)
    a, b = gr[ia], sr[ib]
    m = (a["status"] == B.CS_ST_LANDED) & (b["status"] == B.CS_ST_LANDED)
    gx, gy = PU.position(a[m])
    sx, sy = PU.position(b[m])
    assert np.hypot(gx - sx, gy - sy).max() > 0.01   # the models differ away from the plane of the centre


def test_fluorescence_on_the_cylinder():
    segs = _showers(1200, seed=13)
    fl = dict(synth.FLUORESCENCE, half=True)
    g, o = _run(segs, True, True, bunch=1, seed=7, fluorescence=fl)
    st = PU.compare(g, o, bunch=1)
    assert st["matched"] > 2_000, st


def test_invalid_combinations_are_rejected():
    torch = pytest.importorskip("torch")
    tel = _tel()
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=False, cylindrical=True)
    segs = synth.shower_segments(50, 30.0, 0.0, 1e12, 0)
    with pytest.raises(RuntimeError):   # the tables serve the plane and the sphere only
        B.propagate_host(segs, atm, B.Detector(hist=HIST, tel=tel, cylindrical=True), bunch=1)
    with pytest.raises(RuntimeError):   # the detector's geometry must match
        B.propagate_host(segs, atm, B.Detector(hist=HIST, tel=tel, spherical=True), bunch=1, snell_dh=DH)
    with pytest.raises(RuntimeError):
        B.propagate_host(segs, atm, B.Detector(hist=HIST, tel=tel), bunch=1, snell_dh=DH)
    with pytest.raises(RuntimeError):   # no LV3 pre-filter on the cylinders
        B.propagate_host(segs, atm, B.Detector(hist=HIST, tel=tel, cylindrical=True), bunch=1, snell_dh=DH,
                         lv3=dict(centre=(0.0, 0.0, 2000.0), radius=1000.0))
