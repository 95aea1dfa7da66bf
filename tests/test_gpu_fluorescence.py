"""Parity of fluorescence emission (Eq. 2.6, Sec. 4.2.2) with the oracle,
photon by photon: isotropic and half-sphere emission, the synthetic line list,
refraction, transmission, histogram and telescopes, planar and spherical;
and its argument checks."""
import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import binding as B
from paper_2405_04229_gb300 import synth
from tests import parity_util as PU

pytestmark = pytest.mark.gpu

ORC_ATM = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
HIST = synth.histogram_400()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("half", [False, True])
def test_planar_fluorescence_parity(half):
    segs = synth.shower_segments(6000, 20.0, 30.0, 1e12, seed=21)
    tel = synth.grid_telescopes()
    fl = dict(synth.FLUORESCENCE, half=half)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    det = B.Detector(hist=HIST, tel=tel)
    g = B.propagate_host(segs, atm, det, seed=8, bunch=1, records=True, fluorescence=fl)
    o = oracle.propagate(segs, ORC_ATM, hist=HIST, tel=tel, bunch=1, refraction=True, transmission=True, seed=8,
                         fluorescence=fl)
    st = PU.compare(g, o, bunch=1)
    assert st["matched"] > 10000
    r = g["records"]
    assert (r["status"] == B.CS_ST_UPWARD).any() != half
    lam = np.round(r["lambda_nm"].astype(np.float64), 2)
    assert set(lam.tolist()) <= set(synth.FLUORESCENCE["lines_nm"])
    PU.check_conservation(g["counters"])


def test_spherical_fluorescence_parity():
    """Isotropic photons fall close to their emission points, tens of km out
    in the frame: the ground point is carried as float-float relative to the
    segment's start, so positions agree to 1e-5 of the displacement like every
    other photon's."""
    segs = synth.shower_segments(8000, 60.0, 10.0, 1e13, seed=22)
    fl = dict(synth.FLUORESCENCE, half=True)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True, spherical=True)
    det = B.Detector(hist=HIST, tel=synth.grid_telescopes(), spherical=True)
    g = B.propagate_host(segs, atm, det, seed=9, bunch=1, records=True, fluorescence=fl)
    o = oracle.propagate(segs, ORC_ATM, hist=HIST, tel=synth.grid_telescopes(), bunch=1, refraction=True,
                         transmission=True, seed=9, spherical=True, fluorescence=fl, bands=dict(band_pos=0.03))
    st = PU.compare(g, o, bunch=1)
    assert st["matched"] > 10000
    PU.check_conservation(g["counters"])


def test_fluorescence_arguments():
    segs = synth.shower_segments(50, 20.0, 0.0, 1e12, seed=1)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=False)
    det = B.Detector(hist=HIST)
    bad = [dict(synth.FLUORESCENCE, yield_per_mev=[0.0] * 5), dict(synth.FLUORESCENCE, lines_nm=[0.0] * 5),
           dict(lines_nm=[337.0] * 9, yield_per_mev=[1.0] * 9, dedx=2.2)]
    for fl in bad:
        with pytest.raises(RuntimeError):
            B.propagate_host(segs, atm, det, seed=1, fluorescence=fl)
    with pytest.raises(RuntimeError):   # isotropic light is not filtered by direction
        B.propagate_host(segs, atm, det, seed=1, fluorescence=synth.FLUORESCENCE,
                         lv1=dict(metric=B.CS_LV1_ARRAY_CENTRE, a=1.0, b=1.0))
    # a homogeneous medium has no density: no fluorescence photons
    hom = B.Atmosphere(kind=B.CS_ATM_HOMOGENEOUS, hom_delta=2e-4, refraction=False, transmission=False)
    r = B.propagate_host(segs, hom, det, seed=1, fluorescence=synth.FLUORESCENCE)
    assert r["counters"][B.CS_CNT_EMITTED] == 0
