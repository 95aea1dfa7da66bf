"""Pins of the FP64 oracle against facts it does not compute itself: published
known-answer vectors, closed forms derived independently of the quadrature,
textbook constants, the thesis's own numerical tracer and printed bounds,
geometric invariants, distribution laws and brute force on tiny inputs.

A plausible mistake anywhere in the oracle (a dropped term, a wrong sign or
index, a transposed operand, a unit slip) is meant to fail one of these."""
import math
import os

import numpy as np
import pytest
from scipy import optimize, stats

import oracle
from paper_2405_04229_gb300 import synth

C = 299_792_458.0
ATM = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
LIN = oracle.make_atm(oracle.ATM_LINEAR, linear=synth.LINEAR_TEST)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _segs(n, z0, uz=-1.0, ux=0.0, gamma=1e4, length=1.0, charge=1.0, x0=0.0):
    s = synth._empty(n)
    s["x0"][:] = x0
    s["z0"][:] = z0
    d = np.array([ux, 0.0, uz])
    d = d / np.linalg.norm(d)
    s["ux"][:], s["uy"][:], s["uz"][:] = d.astype(np.float32)
    s["length"][:] = length
    s["inv_gamma2"][:] = np.float32(1.0 / gamma**2)
    s["charge"][:] = charge
    return s


# ---------------------------------------------------------------- RNG -----
def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox(v[0:4], v[4:6]) == v[6:10]


def test_keyed_rng_makes_chunking_irrelevant():
    """Counter-based draws keyed by (segment, sub-step, photon): splitting the
    input changes nothing (Sec. 3.1: reproducibility, trivial fast-forward)."""
    segs = synth.tiny_vertical_segments(200, seed=3)
    whole = oracle.propagate(segs, ATM, hist=synth.histogram_400(), seed=11)
    a = oracle.propagate(synth.take(segs, slice(0, 77)), ATM, hist=synth.histogram_400(), seed=11)
    b = oracle.propagate(synth.take(segs, slice(77, 200)), ATM, hist=synth.histogram_400(), seed=11,
                         seg_base=77)
    assert np.array_equal(whole["hist"], a["hist"] + b["hist"])
    assert np.array_equal(whole["counters"], a["counters"] + b["counters"])
    cat = np.concatenate([a["records"], b["records"]])
    assert np.array_equal(whole["records"], cat)


# ---------------------------------------------------------- quadrature -----
@pytest.mark.parametrize("n", [2, 5, 10, 16])
def test_gauss_legendre_rule_matches_library(n):
    x, w = oracle.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    o = np.argsort(x)
    np.testing.assert_allclose(x[o], xr, atol=1e-14)
    np.testing.assert_allclose(w[o], wr, atol=1e-14)
    # exact for polynomials of degree 2n - 1
    for deg in range(2 * n):
        exact = (1.0 - (-1.0) ** (deg + 1)) / (deg + 1)
        assert abs(np.sum(w * x**deg) - exact) < 1e-13


# ---------------------------------------------------------- atmosphere -----
def test_us_standard_column_depth_parameter_set():
    # sea-level column of the US standard atmosphere: about 1033 g/cm^2
    # (1013.25 hPa / g); the Linsley fit gives 1036.1
    assert abs(oracle.atm_T(ATM, 0.0) - 1036.10) < 0.01
    assert abs(oracle.atm_T(ATM, 0.0) - 1033.2) / 1033.2 < 0.005
    # the piecewise fit is continuous at every layer boundary
    for hb in synth.US_STANDARD["layer_h"][1:]:
        assert abs(oracle.atm_T(ATM, hb - 1e-7) - oracle.atm_T(ATM, hb)) < 2e-3
    assert abs(oracle.atm_T(ATM, synth.US_STANDARD["h_top"] - 1e-6)) < 1e-6


@pytest.mark.parametrize("h", [100.0, 2000.0, 5000.0, 12000.0, 45000.0, 105000.0])
def test_density_is_minus_derivative_of_column(h):
    dh = 0.5  # m
    dTdh = (oracle.atm_T(ATM, h + dh) - oracle.atm_T(ATM, h - dh)) / (2 * dh * 100.0)
    assert abs(-dTdh - oracle.atm_rho(ATM, h)) <= 1e-7 * oracle.atm_rho(ATM, h)


def test_refractive_index_and_sea_level_cone_angle():
    assert abs(oracle.atm_delta(ATM, 0.0) - 2.9e-4) < 1e-15
    # the thesis: in air the Cherenkov opening angle is below 1.4 degrees (Sec. 4.3.2)
    theta_max = math.degrees(math.acos(1.0 / (1.0 + oracle.atm_delta(ATM, 0.0))))
    assert 1.3 < theta_max < 1.4
    # the index falls with height and vanishes above the top of the atmosphere
    hs = np.linspace(0, 112000, 300)
    d = np.array([oracle.atm_delta(ATM, h) for h in hs])
    assert np.all(d > 0) and oracle.atm_delta(ATM, 113000.0) == 0.0
    # layers are half-open [h_i, h_i+1): exactly at 10 km the upper law holds
    upper_law = 2.9e-4 * (1305.5948 / 636143.04) * math.exp(-1e6 / 636143.04) / (1222.6562 / 994186.38)
    assert abs(oracle.atm_delta(ATM, 10000.0) - upper_law) < 1e-16


# ---------------------------------------------------------- refraction -----
def test_quadrature_matches_per_layer_closed_forms():
    rng = np.random.default_rng(1)
    for _ in range(40):
        h_e = rng.uniform(2100.0, 60000.0)
        th = math.radians(rng.uniform(0.0, 75.0))
        q = oracle.refract_quad(ATM, 2000.0, h_e, th)
        cf = oracle.refract_closed(ATM, 2000.0, h_e, th)
        np.testing.assert_allclose(q[:3], cf, rtol=1e-9)


def test_linear_profile_analytic_solution():
    """Sec. 3.4.3 / App. A.1: for dn/dh = -c1 the photon path is an arcosh curve
    (Eq. 3.20-3.23, with the integration constant fixed by x(0) = 0)."""
    for h_e in (10000.0, 50000.0, 99000.0):
        for deg in (5.0, 30.0, 60.0, 80.0):
            th = math.radians(deg)
            q = oracle.refract_quad(LIN, 0.0, h_e, th)
            cf = oracle.refract_closed(LIN, 0.0, h_e, th)
            np.testing.assert_allclose(q[:2], cf[:2], rtol=1e-9)
            # Eq. 3.20: along the path sin(nu) = c sin(alpha) / (c - y), i.e. n sin = const
            s = (1.0 + oracle.atm_delta(LIN, h_e)) * math.sin(th)
            assert s < 1.0 + oracle.atm_delta(LIN, 0.0)


@pytest.mark.parametrize("atm,h_obs,h_e", [(LIN, 0.0, 50000.0), (ATM, 2000.0, 12000.0)])
def test_snell_vector_stepper_converges(atm, h_obs, h_e):
    """The thesis's tracer (Eq. 3.15) agrees with the exact path to <= 0.1 %
    (Sec. 6.3.1) and converges to it as the slab thickness shrinks."""
    for deg in (10.0, 40.0, 70.0):
        th = math.radians(deg)
        ref = oracle.refract_quad(atm, h_obs, h_e, th)
        e10 = abs(oracle.snell_stepper(atm, h_obs, h_e, th, 10.0)[0] - ref[0]) / ref[0]
        e1 = abs(oracle.snell_stepper(atm, h_obs, h_e, th, 1.0)[0] - ref[0]) / ref[0]
        assert e10 < 1e-3
        assert e1 < e10 / 4.0 or e1 < 1e-12
        t10 = oracle.snell_stepper(atm, h_obs, h_e, th, 10.0)[1]
        assert abs(t10 - ref[1]) / ref[1] < 1e-3


def test_homogeneous_medium_is_straight():
    for delta in (0.0, 3e-4):
        hom = oracle.make_atm(oracle.ATM_HOMOGENEOUS, hom_delta=delta)
        for deg in (0.0, 20.0, 60.0):
            th = math.radians(deg)
            q = oracle.refract_quad(hom, 0.0, 8000.0, th)
            assert abs(q[0] - 8000.0 * math.tan(th)) < 1e-9
            assert abs(q[1] - (1 + delta) * 8000.0 / math.cos(th) / C) < 1e-18


def test_vertical_columns_match_column_depth():
    for h_e in (3000.0, 9000.0, 25000.0):
        q = oracle.refract_quad(ATM, 2000.0, h_e, 0.0)
        assert q[0] == 0.0
        # integral of rho == the layers' column laws differenced at their ends
        assert abs(q[2] - oracle.column(ATM, 2000.0, h_e)) < 1e-8
        # ... which equals T(h_obs) - T(h_e) up to the fit's boundary mismatch
        assert abs(q[2] - (oracle.atm_T(ATM, 2000.0) - oracle.atm_T(ATM, h_e))) < 3e-3
        assert abs(q[3] - 1200.0 * (math.exp(-2000.0 / 1200.0) - math.exp(-h_e / 1200.0))) < 1e-10


def test_refraction_pulls_photons_toward_vertical_first_order():
    """For small angles the correction to the straight line is
    sin(theta0) * int (n_e / n - 1) dh (first order of Eq. 3.17 in theta0)."""
    h_e = 10000.0
    n_e = 1 + oracle.atm_delta(ATM, h_e)
    hs, w = np.polynomial.legendre.leggauss(200)
    edges = [2000.0, 4000.0, 10000.0]
    first = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
        first += half * sum(wi * (n_e / (1 + oracle.atm_delta(ATM, mid + half * xi)) - 1.0)
                            for xi, wi in zip(hs, w))
    th = 1e-4
    q = oracle.refract_quad(ATM, 2000.0, h_e, th)
    dR = q[0] - 8000.0 * math.tan(th)
    assert abs(dR / math.sin(th) - first) < 1e-6 * abs(first)
    prev = 0.0
    for deg in (5, 15, 30, 50, 70):
        th = math.radians(deg)
        dR = oracle.refract_quad(ATM, 2000.0, h_e, th)[0] - 8000.0 * math.tan(th)
        assert dR < prev
        prev = dR


# -------------------------------------------------------- emission -----
def test_frank_tamm_prefactor_matches_pdg_constant():
    """d2N/dxdE = (alpha z^2 / hbar c) sin^2 = 369.8 sin^2 photons / (eV cm)
    (PDG, Passage of particles through matter); the oracle's sub-step mean
    divided by sin^2 and by the band in eV must reproduce it."""
    segs = _segs(50, 9000.0, gamma=1e6, length=1.0)
    r = oracle.propagate(segs, ATM, hist=None, s_max=1.0, bunch=1)
    nbar = r["records"]["nbar"][r["records"]["status"] != oracle.ST_SUBSTEP_FLAG]
    n = 1 + oracle.atm_delta(ATM, 9000.0 - 0.5)
    beta2 = 1.0 - float(np.float32(1e-12))
    sin2 = 1.0 - 1.0 / (beta2 * n * n)
    hc_eVnm = 1239.841984
    dE = hc_eVnm / 300.0 - hc_eVnm / 600.0
    per_eV_cm = nbar[0] / sin2 / dE / 100.0
    assert abs(per_eV_cm - 369.81) / 369.81 < 2e-4
    assert abs(per_eV_cm - 370.0) / 370.0 < 1e-3


def test_stochastic_rounding_is_unbiased():
    segs = _segs(3000, 9000.0, gamma=1e5, length=1.0)
    r = oracle.propagate(segs, ATM, hist=None, s_max=1.0, bunch=7)
    rec = r["records"][r["records"]["status"] != oracle.ST_SUBSTEP_FLAG]
    nbar = rec["nbar"][0]
    emitted = r["counters"][0] / 7
    mean = emitted / 3000
    frac = nbar - math.floor(nbar)
    sd = math.sqrt(frac * (1 - frac) / 3000)
    assert abs(mean - nbar) < 5 * sd
    assert set(np.bincount(np.unique(rec["seg"], return_counts=True)[1])) <= set(range(0, 10**6))
    counts = np.unique(rec["seg"], return_counts=True)[1]
    assert counts.min() >= math.floor(nbar) and counts.max() <= math.floor(nbar) + 1


def test_cherenkov_threshold():
    """Light only if beta n > 1 (Eq. 2.3 / Fig. 2.7)."""
    h = 10000.0
    n = 1 + oracle.atm_delta(ATM, h - 0.5)
    gamma_th = 1.0 / math.sqrt(1.0 - 1.0 / n**2)
    assert 70.0 < gamma_th < 72.0
    below = oracle.propagate(_segs(200, h, gamma=0.995 * gamma_th), ATM, bunch=1)
    above = oracle.propagate(_segs(200, h, gamma=1.05 * gamma_th), ATM, bunch=1)
    assert below["counters"][0] == 0
    assert above["counters"][0] > 0


def _c1(n=300, seed=0, **kw):
    segs = synth.tiny_vertical_segments(n, seed)
    return segs, oracle.propagate(segs, ATM, hist=synth.histogram_400(), **kw)


def test_cone_angle_rotation_and_direction_norm():
    segs, r = _c1(300)
    rec = r["records"][r["records"]["status"] != oracle.ST_SUBSTEP_FLAG]
    s = rec["seg"].astype(int)
    P = np.stack([segs["ux"][s], segs["uy"][s], segs["uz"][s]], 1).astype(np.float64)
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    u = np.stack([rec["ux"], rec["uy"], rec["uz"]], 1)
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-14)
    L = segs["length"][s].astype(np.float64)
    K = np.maximum(1, np.ceil(L / 1.0))
    h_mid = segs["z0"][s] + (rec["k"] + 0.5) / K * L * P[:, 2]
    n = 1 + np.array([oracle.atm_delta(ATM, h) for h in h_mid])
    beta = np.sqrt(1.0 - segs["inv_gamma2"][s].astype(np.float64))
    np.testing.assert_allclose(np.sum(P * u, 1), 1.0 / (beta * n), rtol=1e-13)
    # azimuth about P is uniform: project u onto a frame perpendicular to P
    e1 = np.cross(P, [0.0, 1.0, 0.0]); e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(P, e1)
    phi = np.arctan2(np.sum(u * e2, 1), np.sum(u * e1, 1))
    assert stats.kstest((phi + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3


def test_wavelength_follows_inverse_square_law():
    segs, r = _c1(300)
    lam = r["records"]["lam"][r["records"]["status"] != oracle.ST_SUBSTEP_FLAG] * 1e9
    cdf = lambda x: (1 / 300.0 - 1 / np.asarray(x)) / (1 / 300.0 - 1 / 600.0)
    assert stats.kstest(lam, cdf).pvalue > 1e-3
    assert lam.min() >= 300.0 and lam.max() < 600.0


def test_emission_point_uniform_along_segment():
    segs, r = _c1(300)
    rec = r["records"][r["records"]["status"] != oracle.ST_SUBSTEP_FLAG]
    s = rec["seg"].astype(int)
    ell = (segs["z0"][s] - rec["h_e"]) / -segs["uz"][s].astype(np.float64)
    frac = ell / segs["length"][s]
    assert frac.min() >= -1e-9 and frac.max() <= 1 + 1e-9
    assert stats.kstest(frac, "uniform").pvalue > 1e-3


def test_straight_line_geometry():
    """Eq. 3.3: the ground point lies on the photon's line at the observation level."""
    segs, r = _c1(300)
    rec = r["records"][r["records"]["status"] == oracle.ST_LANDED]
    dx, dy = rec["x"] - rec["ex"], rec["y"] - rec["ey"]
    t = (2000.0 - rec["h_e"]) / rec["uz"]
    np.testing.assert_allclose(dx, t * rec["ux"], atol=1e-9)
    np.testing.assert_allclose(dy, t * rec["uy"], atol=1e-9)
    np.testing.assert_allclose(rec["dt"] * C, (rec["h_e"] - 2000.0) / -rec["uz"]
                               + (segs["z0"][rec["seg"].astype(int)] - rec["h_e"])
                               / -segs["uz"][rec["seg"].astype(int)].astype(np.float64)
                               / np.sqrt(1 - segs["inv_gamma2"][rec["seg"].astype(int)].astype(np.float64)),
                               rtol=1e-9)


def test_conservation_and_aggregates_match_records():
    segs = synth.refraction_showers(2, 150, seed=4)
    r = oracle.propagate(segs, ATM, hist=synth.histogram_400(), tel=synth.grid_telescopes(), bunch=5,
                         refraction=True, transmission=True, n_showers=2)
    c = r["counters"]
    assert c[0] == c[1] + c[2] + c[4] == c[1] + c[3] + c[5]
    assert r["hist"].sum() == c[2] and r["tel_counts"].sum() == c[3]
    rec = r["records"][r["records"]["status"] != oracle.ST_SUBSTEP_FLAG]
    sh = segs["shower_id"][rec["seg"].astype(int)]
    h = np.zeros_like(r["hist"])
    m = rec["bin"] >= 0
    np.add.at(h.reshape(2, -1), (sh[m], rec["bin"][m]), 5)
    assert np.array_equal(h, r["hist"])
    assert (rec["status"] == oracle.ST_ABSORBED).sum() * 5 == c[1]


def test_histogram_bins_brute_force():
    segs, r = _c1(300)
    rec = r["records"][r["records"]["status"] == oracle.ST_LANDED]
    h = np.zeros((400, 400), np.uint64)
    for x, y in zip(rec["x"], rec["y"]):
        for iy in range(400):
            if -200.0 + iy <= y < -200.0 + iy + 1:
                for ix in range(400):
                    if -200.0 + ix <= x < -200.0 + ix + 1:
                        h[iy, ix] += 1
    assert np.array_equal(h, r["hist"][0])


def test_telescope_hits_brute_force_minimisation():
    """Telescope hit = the photon's line passes within R of the sphere centre;
    checked by numerically minimising the distance along the line."""
    segs = synth.tiny_vertical_segments(150, seed=2)
    tel = synth.grid_telescopes(nx=7, ny=7, pitch=40.0, radius=6.0)
    r = oracle.propagate(segs, ATM, hist=None, tel=tel, bunch=1)
    rec = r["records"][r["records"]["status"] == oracle.ST_LANDED]
    hits = 0
    for p in rec:
        I = np.array([p["x"], p["y"], 2000.0])
        u = np.array([p["ux"], p["uy"], p["uz"]])
        best, best_d = -1, np.inf
        for j, T in enumerate(tel):
            if np.hypot(T[0] - I[0], T[1] - I[1]) > 30.0:
                continue
            f = lambda t: np.sum((I + t * u - T[:3]) ** 2)
            d = math.sqrt(optimize.minimize_scalar(f, bounds=(-100, 100), method="bounded",
                                                   options=dict(xatol=1e-10)).fun)
            if d < T[3] and d < best_d:
                best, best_d = j, d
        if not (p["flags"] & oracle.FL_TEL_EDGE):
            assert best == p["tel"]
        hits += best >= 0
    assert hits >= 10


def test_transmission_vertical_closed_form_and_limits():
    segs = _segs(400, 9000.0, gamma=1e4, length=1.0)
    r = oracle.propagate(segs, ATM, transmission=True, bunch=1, hist=None)
    rec = r["records"][r["records"]["status"] != oracle.ST_SUBSTEP_FLAG]
    lam = rec["lam"]
    X = np.array([oracle.column(ATM, 2000.0, h) for h in rec["h_e"]]) / np.cos(rec["theta0"])
    A = 1200.0 * (np.exp(-2000.0 / 1200.0) - np.exp(-rec["h_e"] / 1200.0)) / np.cos(rec["theta0"])
    T = np.exp(-X / (2974.0 * (lam / 400e-9) ** 4) - 0.05 * (lam / 350e-9) ** -1.3 * A / 1200.0)
    np.testing.assert_allclose(rec["T"], T, rtol=1e-12)
    surv = np.mean(rec["status"] == oracle.ST_LANDED)
    assert abs(surv - T.mean()) < 5 * math.sqrt(T.mean() * (1 - T.mean()) / len(T))
    clear = oracle.propagate(segs, ATM, transmission=True, bunch=1,
                             transmission_params=dict(aer_tau0=0.0, rayl_X0=1e30))
    assert clear["counters"][1] == 0 and clear["counters"][0] == r["counters"][0]


def test_refraction_records_match_direct_quadrature():
    segs = synth.refraction_showers(1, 60, seed=5)
    r = oracle.propagate(segs, ATM, refraction=True, bunch=5, hist=synth.histogram_400())
    rec = r["records"][r["records"]["status"] == oracle.ST_LANDED][:40]
    for p in rec:
        q = oracle.refract_quad(ATM, 2000.0, p["h_e"], p["theta0"])
        uh = math.hypot(p["ux"], p["uy"])
        assert abs(p["x"] - (p["ex"] + q[0] * p["ux"] / uh)) < 1e-6
        assert abs(p["y"] - (p["ey"] + q[0] * p["uy"] / uh)) < 1e-6


def test_status_edge_cases():
    # emission below the observation level
    r = oracle.propagate(_segs(20, 1500.0), ATM, bunch=1)
    rec = r["records"][r["records"]["status"] != oracle.ST_SUBSTEP_FLAG]
    assert np.all(rec["status"] == oracle.ST_BELOW)
    # an upward-going segment: every photon goes up
    r = oracle.propagate(_segs(20, 9000.0, uz=0.9, ux=0.43), ATM, bunch=1)
    rec = r["records"][r["records"]["status"] != oracle.ST_SUBSTEP_FLAG]
    assert len(rec) > 0 and np.all(rec["status"] == oracle.ST_UPWARD)
    assert r["counters"][6] == r["counters"][0]
    # invalid inputs are counted and skipped
    bad = _segs(5, 9000.0)
    bad["length"][0] = 0.0
    bad["inv_gamma2"][1] = 1.5
    bad["uz"][2] = np.nan
    bad["shower_id"][3] = 7
    bad["ux"][4], bad["uy"][4], bad["uz"][4] = 0.0, 0.0, 1.0
    r = oracle.propagate(bad, ATM, bunch=1)
    assert r["counters"][7] == 5 and r["counters"][0] == 0
    # empty input
    r = oracle.propagate(_segs(0, 9000.0), ATM, bunch=1)
    assert r["counters"].sum() == 0
