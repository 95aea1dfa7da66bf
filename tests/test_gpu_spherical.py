"""Parity of the spherical-shell path (Sec. 3.3.4) with the FP64 oracle:
the FP64 table builder against the oracle's Bouguer quadrature, and photon
by photon for inclined showers with straight lines, refraction,
transmission, a ground histogram and an irregular telescope layout.

Edge band on the sphere: ground points of ~50 km slant paths carry a few
FP32 ulps of ~4 mm, so bin and sphere edges are flagged within
8 ulp(5e4 m) = 0.03 m of the FP64 value (positions and times keep the
relative 1e-5 bar of the planar path)."""
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
BAND_POS = 0.03
C = 299792458.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _atm(refr, trans):
    return B.Atmosphere(layered=synth.US_STANDARD, refraction=refr, transmission=trans, spherical=True)


@pytest.mark.parametrize("refr", [True, False])
def test_spherical_table_builder_matches_oracle_quadrature(refr):
    atm = _atm(refr, True)
    tab, info = atm.table()
    rg = oracle.EARTH_RADIUS + 2000.0
    rng = np.random.default_rng(7)
    for _ in range(60):
        j = int(rng.integers(1, 1500))
        m = int(rng.integers(0, info["nw"]))
        h_e = info["h0"] + j * info["dh"]
        w = max(m * info["dw"], 1e-8)
        th = math.atan(math.sqrt(w))
        c, s = math.cos(th), math.sin(th)
        line = oracle.sph_path(ORC_ATM, 2000.0, h_e, th, refraction=False, rtol=1e-13)
        if refr:
            q = oracle.sph_path(ORC_ATM, 2000.0, h_e, th, refraction=True, rtol=1e-13)
            want = np.array([rg * (q[0] - line[0]) * c**3 / s, (q[1] - line[1]) * C * c, q[2] * c, q[3] * c])
        else:
            want = np.array([0.0, 0.0, line[2] * c, line[3] * c])
        got = tab[j, m, 0].astype(np.float64)
        scale = np.maximum(np.abs(want), [1e-3, 1e-3, 1e-2, 1e-2])
        assert np.all(np.abs(got - want) <= 2e-6 * scale + 1e-9), (j, m, got, want)


def _run_both(segs, refr, trans, bunch, tel=None, seed=0):
    atm = _atm(refr, trans)
    det = B.Detector(hist=HIST, tel=tel, spherical=True)
    g = B.propagate_host(segs, atm, det, seed=seed, bunch=bunch, records=True)
    o = oracle.propagate(segs, ORC_ATM, hist=HIST, tel=tel, bunch=bunch, refraction=refr, transmission=trans,
                         seed=seed, spherical=True, bands=dict(band_pos=BAND_POS))
    return g, o


def _tel():
    return synth.poisson_disk_telescopes(n=300, half=250.0, seed=1)


@pytest.mark.parametrize("zenith", [20.0, 60.0])
def test_spherical_refraction_transmission_parity(zenith):
    segs = synth.shower_segments(1500, zenith, 30.0, 1e13, seed=4)
    tel = _tel()
    g, o = _run_both(segs, True, True, 3, tel=tel, seed=5)
    st = PU.compare(g, o, bunch=3)
    assert st["matched"] > 10000
    PU.check_conservation(g["counters"])
    assert g["counters"][B.CS_CNT_TEL] > 0 and g["counters"][B.CS_CNT_HIST] > 0


def test_spherical_straight_line_parity():
    segs = synth.shower_segments(1500, 60.0, 200.0, 1e13, seed=8)
    g, o = _run_both(segs, False, False, 2, tel=_tel(), seed=1)
    st = PU.compare(g, o, bunch=2)
    assert st["matched"] > 10000
    PU.check_conservation(g["counters"])


def test_spherical_ragged_sizes():
    for n in (1, 255, 257):
        segs = synth.shower_segments(n, 60.0, 0.0, 1e13, seed=n)
        g, o = _run_both(segs, True, False, 1)
        PU.compare(g, o, bunch=1)
        PU.check_conservation(g["counters"])


def test_geometry_mismatch_is_rejected():
    atm = _atm(True, False)
    det = B.Detector(hist=HIST)   # planar
    segs = synth.shower_segments(10, 60.0, 0.0, 1e13, seed=0)
    with pytest.raises(RuntimeError):
        B.propagate_host(segs, atm, det, seed=0, bunch=1)


def test_streamer_equals_one_call():
    """Chunks through two staging buffers on two streams give the integer
    outputs of one call over all segments (draws keyed by global ids)."""
    torch = pytest.importorskip("torch")
    segs = synth.shower_segments(23_000, 60.0, 45.0, 1e13, seed=12)
    arr = B.pack_segments(segs)
    tel = _tel()
    atm = _atm(True, True)
    det = B.Detector(hist=HIST, tel=tel, spherical=True)
    ref = B.propagate_host(segs, atm, det, seed=3, bunch=4)
    pinned = torch.from_numpy(arr.view(np.uint8)).pin_memory()
    outs = B.DeviceOutputs(det)
    st = B.Streamer(5_000)
    for _ in range(2):   # the second run reuses the buffers and re-zeroes the outputs
        st.run(pinned.data_ptr(), len(arr), atm, det, outs.out, seed=3, bunch=4)
        h = outs.host()
        assert np.array_equal(h["counters"], ref["counters"])
        assert np.array_equal(h["hist"], ref["hist"])
        assert np.array_equal(h["tel_counts"], ref["tel_counts"])
        np.testing.assert_allclose(h["tel_time"], ref["tel_time"], rtol=1e-12)
    st.close()


def test_inclined_full_size_streamed_sampled():
    """Two 1e7-segment chunks of the large inclined shower (the benchmark's
    chunk size and launch path) streamed with records on; 150 sampled
    segments checked photon by photon against the oracle, all records
    against the aggregates."""
    torch = pytest.importorskip("torch")
    chunk = 10_000_000
    parts = [synth.inclined_chunk(c, n=chunk) for c in (3, 4)]
    tel = synth.poisson_disk_telescopes(n=2000, half=1000.0, min_sep=13.0, radius=6.0, seed=0)
    atm = _atm(True, True)
    det = B.Detector(hist=HIST, tel=tel, spherical=True)
    pinned = torch.empty(2 * chunk * 64, dtype=torch.uint8).pin_memory()
    hv = pinned.numpy()
    for j, p in enumerate(parts):
        hv[j * chunk * 64:(j + 1) * chunk * 64] = B.pack_segments(p).view(np.uint8)
    cap = 150_000_000
    outs = B.DeviceOutputs(det, record_capacity=cap)
    st = B.Streamer(chunk)
    st.run(pinned.data_ptr(), 2 * chunk, atm, det, outs.out, seed=0, bunch=10, seg_base=3 * chunk)
    torch.cuda.synchronize()
    st.close()
    c = outs.counters.cpu().numpy().astype(np.uint64)
    PU.check_conservation(c)
    nrec = int(outs.record_count.item())
    assert nrec <= cap and int(c[0]) == 10 * nrec
    recs = outs.records[: nrec * B.RECORD_DTYPE.itemsize].view(torch.int64).view(nrec, B.RECORD_DTYPE.itemsize // 8)
    rng = np.random.default_rng(21)
    sample = np.sort(rng.choice(2 * chunk, 150, replace=False))
    gids = torch.from_numpy((sample + 3 * chunk).astype(np.int64)).cuda()
    sel = torch.isin(recs[:, 0], gids)
    g = recs[sel].cpu().numpy().reshape(-1).view(np.uint8).view(B.RECORD_DTYPE)
    # every record's bin agrees with the histogram (records of the whole launch)
    bins = recs.view(torch.int32)[:, 9]
    h = torch.bincount(bins[bins >= 0].long(), minlength=400 * 400) * 10
    assert torch.equal(h.cpu(), outs.hist.view(-1).cpu())
    o_recs = []
    for s in sample:
        part = parts[int(s) // chunk]
        r = oracle.propagate(synth.take(part, slice(int(s) % chunk, int(s) % chunk + 1)), ORC_ATM, hist=HIST,
                             tel=tel, bunch=10, refraction=True, transmission=True, seed=0,
                             seg_base=int(s) + 3 * chunk, spherical=True, bands=dict(band_pos=BAND_POS))
        o_recs.append(r["records"])
    st_ = PU.compare(dict(records=g, n_records=len(g)), dict(records=np.concatenate(o_recs)), bunch=10,
                     check_hist=False)
    assert st_["matched"] > 300


def test_spherical_steep_arrivals_beyond_the_telescope_hash():
    segs = synth.steep_arrival_segments(2000, seed=2)
    g, o = _run_both(segs, False, False, 1, tel=synth.grid_telescopes(), seed=2)
    st = PU.compare(g, o, bunch=1)
    assert st["matched"] > 100000
    assert int(g["counters"][B.CS_CNT_TEL]) > 5000


def test_spherical_surrogate_against_exact_tracer():
    """The network trained on the spherical shell's exact fields (local zenith)
    replaces the tables photon by photon within its stated bars."""
    atm = _atm(True, True)
    sur = B.Surrogate(atm)
    s = sur.stats
    for k, bar in enumerate((0.01, 0.1e-9, 1e-3)):
        assert s["p99"][k] <= bar and s["max"][k] <= bar, s
    segs = synth.shower_segments(1500, 60.0, 30.0, 1e13, seed=21)
    det = B.Detector(hist=HIST, tel=_tel(), spherical=True)
    ex = B.propagate_host(segs, atm, det, seed=2, bunch=5, records=True)
    sg = B.propagate_host(segs, atm, det, seed=2, bunch=5, records=True, surrogate=sur)
    ke = PU._key(ex["records"]["seg"], ex["records"]["k"], ex["records"]["i"])
    ks = PU._key(sg["records"]["seg"], sg["records"]["k"], sg["records"]["i"])
    e, g = ex["records"][np.argsort(ke)], sg["records"][np.argsort(ks)]
    assert np.array_equal(np.sort(ke), np.sort(ks))
    both = (e["status"] == 0) & (g["status"] == 0)
    assert both.sum() > 2000
    ex_, ey_ = PU.position(e[both])
    gx_, gy_ = PU.position(g[both])
    dpos = np.hypot(ex_ - gx_, ey_ - gy_)
    dt = np.abs(e["dt_ns"][both] - g["dt_ns"][both]) * 1e-9
    # the network's bars plus the FP32 resolution of ~50 km paths
    assert dpos.max() <= 0.01 + BAND_POS
    assert dt.max() <= 0.1e-9 + 1e-5 * 2e-4
    assert (e["status"] != g["status"]).sum() <= 0.01 * len(e)
    sur.close()


@pytest.mark.parametrize("refr", [True, False])
def test_spherical_beyond_the_tables_and_past_the_ground(refr):
    """Near-horizontal photons on the spherical shell: beyond the tables'
    zenith they take the exact Bouguer path integrated per photon; those
    whose path passes over the ground sphere are missed on both sides."""
    rng = np.random.default_rng(21)
    n = 500
    s = synth._empty(n)
    th = np.radians(rng.uniform(80.0, 89.6, n))
    az = rng.uniform(0.0, 2 * np.pi, n)
    s["z0"] = rng.uniform(2100.0, 9000.0, n)
    s["x0"] = rng.uniform(-3000.0, 3000.0, n)
    s["y0"] = rng.uniform(-3000.0, 3000.0, n)
    s["ux"] = (np.sin(th) * np.cos(az)).astype(np.float32)
    s["uy"] = (np.sin(th) * np.sin(az)).astype(np.float32)
    s["uz"] = (-np.cos(th)).astype(np.float32)
    s["length"][:] = np.float32(2.0)
    s["inv_gamma2"][:] = np.float32(1e-8)
    s["charge"][:] = 1.0
    g, o = _run_both(s, refr, True, 2, tel=_tel(), seed=8)
    st = PU.compare(g, o, bunch=2)
    rec = o["records"]
    assert (rec["status"] == oracle.ST_NO_GROUND).sum() > 200
    assert ((rec["status"] == oracle.ST_LANDED) & (np.degrees(rec["theta0"]) > 76.0)).sum() > 2000
    assert st["matched"] > 5000
    PU.check_conservation(g["counters"])
