"""Parity of the Snell vector stepper (Sec. 3.4.2, Eq. 3.15), the per-photon
general-atmosphere tracer, with the oracle's FP64 stepper over the same slabs:
photon by photon for the layered fit and a user's n(h) table, with
refraction and transmission; against the kernel's own table tracer (the two
methods agree up to the stepper's discretisation); and its argument checks."""
import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import binding as B
from paper_2405_04229_gb300 import synth
from tests import parity_util as PU

pytestmark = pytest.mark.gpu

HIST = synth.histogram_400()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("kind,dh", [("layered", 10.0), ("layered", 3.0), ("table", 10.0)])
def test_stepper_parity(kind, dh):
    segs = synth.shower_segments(600, 30.0, 20.0, 1e12, seed=11)
    tel = synth.grid_telescopes()
    if kind == "layered":
        atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
        orc = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
    else:
        t = synth.TABLE_PROFILE
        atm = B.Atmosphere(kind=B.CS_ATM_TABLE, table=t, refraction=True, transmission=True)
        orc = oracle.make_atm(oracle.ATM_TABLE, table=t)
    det = B.Detector(hist=HIST, tel=tel)
    g = B.propagate_host(segs, atm, det, seed=6, bunch=2, records=True, snell_dh=dh)
    o = oracle.propagate(segs, orc, hist=HIST, tel=tel, bunch=2, refraction=True, transmission=True, seed=6,
                         snell_dh=dh)
    st = PU.compare(g, o, bunch=2)
    assert st["matched"] > 10000
    PU.check_conservation(g["counters"])
    assert g["counters"][B.CS_CNT_ABSORBED] > 0


def test_shell_stepper_parity():
    """The spherical shell: the kernel's invariant form of Eq. 3.15 against the
    oracle's vector steps about the radial normal, over the same shells."""
    segs = synth.shower_segments(1200, 60.0, 10.0, 1e13, seed=13)
    tel = synth.poisson_disk_telescopes(n=300, half=250.0, seed=1)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True, spherical=True)
    det = B.Detector(hist=HIST, tel=tel, spherical=True)
    orc = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
    g = B.propagate_host(segs, atm, det, seed=3, bunch=3, records=True, snell_dh=10.0)
    o = oracle.propagate(segs, orc, hist=HIST, tel=tel, bunch=3, refraction=True, transmission=True, seed=3,
                         spherical=True, snell_dh=10.0, bands=dict(band_pos=0.03))
    st = PU.compare(g, o, bunch=3)
    assert st["matched"] > 5000
    PU.check_conservation(g["counters"])


def test_stepper_and_tables_agree_up_to_the_discretisation():
    segs = synth.shower_segments(2000, 35.0, 50.0, 1e12, seed=12)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=False)
    line = B.Atmosphere(layered=synth.US_STANDARD, refraction=False, transmission=False)
    det = B.Detector(hist=HIST)
    kw = dict(seed=7, bunch=2, records=True)
    tab = B.propagate_host(segs, atm, det, **kw)["records"]
    stp = B.propagate_host(segs, atm, det, snell_dh=1.0, **kw)["records"]
    st0 = B.propagate_host(segs, line, det, **kw)["records"]
    key = lambda r: (r["seg"].astype(np.int64) << 24) | (r["k"].astype(np.int64) << 12) | r["i"]
    for r in (tab, stp, st0):
        r.sort(order=["seg", "k", "i"])
    assert np.array_equal(key(tab), key(stp)) and np.array_equal(key(tab), key(st0))
    m = (tab["status"] == B.CS_ST_LANDED) & (stp["status"] == B.CS_ST_LANDED) & (st0["status"] == B.CS_ST_LANDED)
    assert m.sum() > 20000
    shift = np.hypot(tab["x"].astype(np.float64) - st0["x"], tab["y"].astype(np.float64) - st0["y"])[m]
    err = np.hypot(tab["x"].astype(np.float64) - stp["x"], tab["y"].astype(np.float64) - stp["y"])[m]
    assert shift.max() > 0.1
    assert (err <= 3e-3 * shift + 2e-3).all(), float(err.max())
    dt = np.abs(tab["dt_ns"].astype(np.float64) - stp["dt_ns"])[m] / tab["dt_ns"][m]
    assert dt.max() < 5e-6


def test_stepper_rejects_what_it_does_not_cover():
    segs = synth.shower_segments(50, 30.0, 0.0, 1e12, seed=1)
    det = B.Detector(hist=HIST)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=False)
    with pytest.raises(RuntimeError):
        B.propagate_host(segs, atm, det, seed=1, snell_dh=1e-4)      # slabs thinner than 1 cm
    sur = B.Surrogate(atm, epochs=1, n_train=1 << 16, n_heldout=1 << 12)
    with pytest.raises(RuntimeError):
        B.propagate_host(segs, atm, det, seed=1, snell_dh=10.0, surrogate=sur)
    sur.close()
    # with refraction off the option changes nothing: straight lines either way
    line = B.Atmosphere(layered=synth.US_STANDARD, refraction=False, transmission=True)
    a = B.propagate_host(segs, line, det, seed=1, bunch=2)
    b = B.propagate_host(segs, line, det, seed=1, bunch=2, snell_dh=10.0)
    assert np.array_equal(a["hist"], b["hist"]) and np.array_equal(a["counters"], b["counters"])
