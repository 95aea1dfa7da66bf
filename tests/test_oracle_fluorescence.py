"""Pins of the oracle's fluorescence emission (Eq. 2.6, Sec. 4.2.2): the
mean count per sub-step is the deposited energy times the lines' yields, the
counts round it stochastically, directions are isotropic over the sphere or
the downward half sphere (with half the photons), the lines appear in
proportion to their yields, and the straight line carries each photon from
its emission point to the ground."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import synth

ATM = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
FL = synth.FLUORESCENCE


def _run(segs, half=False, **kw):
    fl = dict(FL, half=half)
    return oracle.propagate(segs, ATM, bunch=kw.pop("bunch", 3), seed=kw.pop("seed", 2), fluorescence=fl, **kw)


def _rho(h):
    """rho = -dT/dh from the column law of the layer holding h (a central
    difference well inside the layer), in g/cm^3."""
    e = 0.05
    return -(oracle.atm_T(ATM, h + e) - oracle.atm_T(ATM, h - e)) / (2 * e) / 100.0


def test_mean_count_is_the_deposited_energy_times_the_yields():
    segs = synth.shower_segments(150, 20.0, 0.0, 1e12, seed=3)
    r = _run(segs, bunch=3)["records"]
    ysum = sum(FL["yield_per_mev"])
    seen = {}
    for rec in r[r["status"] != oracle.ST_SUBSTEP_FLAG]:
        seen[(int(rec["seg"]), int(rec["k"]))] = float(rec["nbar"])
    assert len(seen) > 200
    checked = 0
    for (s, k), nbar in seen.items():
        L = float(segs["length"][s])
        K = max(1, math.ceil(np.float32(L) / np.float32(1.0)))
        P = np.array([segs["ux"][s], segs["uy"][s], segs["uz"][s]], np.float64)
        P /= np.linalg.norm(P)
        h = float(segs["z0"][s]) + (k + 0.5) / K * L * P[2]
        if min(abs(h - b) for b in synth.US_STANDARD["layer_h"][1:]) < 1.0:
            continue
        z = float(segs["charge"][s])
        want = z * z * FL["dedx"] * _rho(h) * 100.0 * ysum * (L / K) / 3
        assert nbar == pytest.approx(want, rel=1e-6)
        checked += 1
    assert checked > 200


def test_counts_round_the_mean():
    segs = synth.shower_segments(100, 20.0, 0.0, 1e12, seed=4)
    r = _run(segs, bunch=2)["records"]
    r = r[r["status"] != oracle.ST_SUBSTEP_FLAG]
    keys, counts = np.unique(r["seg"].astype(np.int64) * 4096 + r["k"], return_counts=True)
    first = {int(kk): i for i, kk in enumerate(r["seg"].astype(np.int64) * 4096 + r["k"])}
    for kk, n in zip(keys, counts):
        nbar = float(r["nbar"][first[int(kk)]])
        assert n in (math.floor(nbar), math.floor(nbar) + 1)
        assert r["i"][r["seg"].astype(np.int64) * 4096 + r["k"] == kk].max() == n - 1


@pytest.mark.parametrize("half", [False, True])
def test_directions_are_isotropic(half):
    segs = synth.shower_segments(5000, 20.0, 0.0, 1e12, seed=5)
    r = _run(segs, half=half, bunch=1)["records"]
    r = r[r["status"] != oracle.ST_SUBSTEP_FLAG]
    uz = np.sort(r["uz"])
    n = len(uz)
    assert n > 10000
    lo = -1.0
    hi = 0.0 if half else 1.0
    cdf = (uz - lo) / (hi - lo)
    ks = np.max(np.abs(cdf - (np.arange(1, n + 1) - 0.5) / n))
    assert ks < 1.63 / math.sqrt(n)                       # 1 % Kolmogorov-Smirnov level
    assert np.allclose(r["ux"] ** 2 + r["uy"] ** 2 + r["uz"] ** 2, 1.0, atol=1e-12)
    phi = np.arctan2(r["uy"], r["ux"])
    hist, _ = np.histogram(phi, bins=16, range=(-math.pi, math.pi))
    assert ((hist - n / 16) ** 2 / (n / 16)).sum() < 37.7  # chi^2, 15 dof, 0.1 %
    if half:
        assert (r["uz"] < 0).all()


def test_half_sphere_emits_half_the_photons():
    segs = synth.shower_segments(2000, 20.0, 0.0, 1e12, seed=6)
    full = _run(segs, bunch=1)["records"]
    half = _run(segs, half=True, bunch=1)["records"]
    kf, i_f = np.unique(full["seg"].astype(np.int64) * 4096 + full["k"], return_index=True)
    kh, i_h = np.unique(half["seg"].astype(np.int64) * 4096 + half["k"], return_index=True)
    _, a, b = np.intersect1d(kf, kh, return_indices=True)
    assert len(a) > 1000
    np.testing.assert_allclose(half["nbar"][i_h[b]], 0.5 * full["nbar"][i_f[a]], rtol=1e-12)
    nf = int((full["status"] != oracle.ST_SUBSTEP_FLAG).sum())
    nh = int((half["status"] != oracle.ST_SUBSTEP_FLAG).sum())
    assert abs(nh - 0.5 * nf) < 4.0 * math.sqrt(nf)


def test_lines_appear_in_proportion_to_their_yields():
    segs = synth.shower_segments(5000, 20.0, 0.0, 1e12, seed=7)
    r = _run(segs, bunch=1)["records"]
    lam = np.round(r["lam"][r["status"] != oracle.ST_SUBSTEP_FLAG] * 1e9, 6)
    n = len(lam)
    y = np.array(FL["yield_per_mev"]) / sum(FL["yield_per_mev"])
    obs = np.array([(lam == l).sum() for l in FL["lines_nm"]])
    assert obs.sum() == n
    assert ((obs - n * y) ** 2 / (n * y)).sum() < 18.5     # chi^2, 4 dof, 0.1 %


def test_straight_line_carries_each_photon_to_the_ground():
    segs = synth.shower_segments(3000, 20.0, 0.0, 1e12, seed=8)
    r = _run(segs, bunch=2, hist=synth.histogram_400())["records"]
    m = r["status"] == oracle.ST_LANDED
    assert m.sum() > 2000
    t = (r["h_e"][m] - 2000.0) / (-r["uz"][m])
    np.testing.assert_allclose(r["x"][m], r["ex"][m] + t * r["ux"][m], rtol=1e-11, atol=1e-7)
    np.testing.assert_allclose(r["y"][m], r["ey"][m] + t * r["uy"][m], rtol=1e-11, atol=1e-7)
