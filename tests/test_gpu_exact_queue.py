"""Bunches beyond the correction tables reach the exact pass through the
photon kernel's queue or -- when the queue is full or switched off -- through
the tile map, whose tiles the pass regenerates whole (skipping their queued
entries).  Isotropic fluorescence puts a quarter of its bunches beyond the
tables' 75 deg, so a one-entry-per-tile queue overflows in mid-run: the default
queue, the overflowing one and no queue must give the same counts and the same
records (integer fields bit for bit, times and ground points to a few ulps)."""
import numpy as np
import pytest

from paper_2405_04229_gb300 import binding as B
from paper_2405_04229_gb300 import synth

pytestmark = pytest.mark.gpu

HIST = synth.histogram_400()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _sorted(r):
    return np.sort(r["records"][: r["n_records"]], order=["seg", "k", "i"])


def test_queue_overflow_and_tile_map_agree():
    segs = synth.shower_segments(60000, 20.0, 30.0, 1e12, seed=31)
    fl = dict(synth.FLUORESCENCE, half=False)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    det = B.Detector(hist=HIST, tel=synth.grid_telescopes())
    runs = [B.propagate_host(segs, atm, det, seed=4, bunch=1, records=True, fluorescence=fl, exact_queue=q)
            for q in (0, 1, -1)]
    ref = runs[0]
    assert int(ref["counters"][0]) > 20000   # emitted bunches: several thousand beyond the tables
    for r in runs[1:]:
        for k in ("hist", "tel_counts", "counters"):
            assert np.array_equal(r[k], ref[k]), k
        np.testing.assert_allclose(r["tel_time"], ref["tel_time"], rtol=1e-12)
        a, c = _sorted(ref), _sorted(r)
        assert len(a) == len(c) == ref["n_records"]
        for k in ("seg", "k", "i", "tel", "bin", "status", "pix", "lambda_nm"):
            assert np.array_equal(a[k], c[k]), k
        for hi, lo in (("x", "x_lo"), ("y", "y_lo")):
            pa = a[hi].astype(np.float64) + a[lo]
            pc = c[hi].astype(np.float64) + c[lo]
            assert np.all(np.abs(pa - pc) <= 1e-7 * np.abs(pa) + 1e-6), hi
        assert np.allclose(a["dt_ns"], c["dt_ns"], rtol=1e-6, atol=1e-6)
