"""The photon kernel's fixed-configuration instances (the standard
configuration -- refraction, transmission and tables on; histogram, telescopes
and time sums on; no camera optics -- with those tests as
compile-time constants) give the outputs of the general instances: the counts
and every record's integer fields bit for bit, its times and ground points to a
few ulps (the separately compiled instances may contract a product into an FMA
differently).
The general instance is reached by the same call with camera optics on the
telescopes (no absorption: the optics only add camera images), which no
longer matches the standard configuration."""
import numpy as np
import pytest

from paper_2405_04229_gb300 import binding as B
from paper_2405_04229_gb300 import synth

pytestmark = pytest.mark.gpu

HIST = synth.histogram_400()
OPT = dict(mirror_d=7.0, focal_f=8.0, camera_r=0.5, point_zenith=0.35, point_azimuth=0.5, cam_n=9)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _sorted_records(r):
    rec = r["records"][: r["n_records"]]
    return np.sort(rec, order=["seg", "k", "i"])


def _compare(atm, det, det_optics, segs, bunch):
    for records in (True, False):
        f = B.propagate_host(segs, atm, det, seed=3, bunch=bunch, records=records)
        g = B.propagate_host(segs, atm, det_optics, seed=3, bunch=bunch, records=records)
        assert int(f["counters"][0]) > 0
        for k in ("hist", "tel_counts", "counters"):
            assert np.array_equal(f[k], g[k]), k
        np.testing.assert_allclose(f["tel_time"], g["tel_time"], rtol=1e-12)   # FP64 sums, order of the atomics
        if records:
            assert f["n_records"] == g["n_records"] > 0
            a, c = _sorted_records(f), _sorted_records(g)
            for k in ("seg", "k", "i", "tel", "bin", "status", "lambda_nm"):
                assert np.array_equal(a[k], c[k]), k
            # the two instances are compiled separately: a contraction into FMA may differ, which
            # moves the float-float ground point's low part by a few ulps of the high one
            for hi, lo in (("x", "x_lo"), ("y", "y_lo")):
                pa = a[hi].astype(np.float64) + a[lo]
                pc = c[hi].astype(np.float64) + c[lo]
                assert np.all(np.abs(pa - pc) <= 1e-7 * np.abs(pa) + 1e-6), hi
            assert np.allclose(a["dt_ns"], c["dt_ns"], rtol=1e-6, atol=1e-6)


def test_planar_fixed_instance_equals_general():
    segs = synth.refraction_showers(n_showers=2, per_shower=3000, seed=11)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    tel = synth.grid_telescopes()
    _compare(atm, B.Detector(n_showers=2, hist=HIST, tel=tel), B.Detector(n_showers=2, hist=HIST, tel=tel, optics=OPT),
             segs, 5)


def test_spherical_fixed_instance_equals_general():
    segs = synth.shower_segments(1500, 60.0, 30.0, 1e13, seed=5)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True, spherical=True)
    tel = synth.poisson_disk_telescopes(n=300, half=250.0, seed=1)
    _compare(atm, B.Detector(hist=HIST, tel=tel, spherical=True), B.Detector(hist=HIST, tel=tel, spherical=True, optics=OPT),
             segs, 10)
