"""Pins of the oracle's sub-step count and of its treatment of steep photons.

* Sub-stepping (Sec. 4.2.1): K = ceil(L / s_max) in FP64, checked against the
  sub-step indices the records carry; a count that is itself a rounding
  decision flags the whole segment.
* Every descending photon is propagated along the exact path (Sec. 3.4.3,
  Eq. 3.17-3.18): zenith angles beyond any table domain land where an
  independent scipy quadrature of the invariant's integral puts them.
* On the spherical shell (Sec. 3.3.4) a photon whose path never meets the
  ground sphere is not detected: for the straight line the brute-force
  closest approach to the Earth's centre decides, with refraction an
  independent Runge-Kutta ray march shows the ray turning above the ground.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2405_04229_gb300 import synth

C = 299_792_458.0
R_E = oracle.EARTH_RADIUS
H_OBS = 2000.0
ATM = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)


def _real(r):
    return r[r["status"] != oracle.ST_SUBSTEP_FLAG]


def _tilted(n, z0, zenith_deg, seed, length=2.0, gamma=1e4, x_spread=0.0):
    rng = np.random.default_rng(seed)
    s = synth._empty(n)
    th = math.radians(zenith_deg)
    s["z0"][:] = z0
    s["x0"][:] = rng.uniform(-x_spread, x_spread, n) if x_spread else 0.0
    s["ux"][:], s["uz"][:] = np.float32(math.sin(th)), np.float32(-math.cos(th))
    s["length"][:] = length
    s["inv_gamma2"][:] = np.float32(1.0 / gamma**2)
    s["charge"][:] = 1.0
    return s


# ------------------------------------------------------------ sub-steps -----
def test_substep_count_is_the_fp64_ceiling():
    """At 9 km a fast electron emits ~17 photons per metre, so every sub-step
    longer than 0.1 m has a mean count above one and, with stochastic
    rounding, at least one photon: the sub-step indices of a segment's records
    are exactly 0 .. K - 1 with K = ceil(L / s_max)."""
    rng = np.random.default_rng(4)
    s = _tilted(300, 9000.0, 0.0, seed=1)
    s["length"][:] = rng.uniform(0.2, 7.0, 300).astype(np.float32)
    for s_max in (1.0, 0.37, 2.5):
        r = oracle.propagate(s, ATM, s_max=s_max, bunch=1)
        rec = _real(r["records"])
        for i in range(300):
            K = max(1, math.ceil(float(s["length"][i]) / s_max))
            ks = np.unique(rec["k"][rec["seg"] == i])
            assert np.array_equal(ks, np.arange(K)), (i, K, ks)


def test_count_is_the_exact_ceiling_and_near_ties_are_flagged():
    """K is the exact ceiling of L / s_max for the stored numbers.  L = 0.3
    (as FP32, 0.300000012) over s_max = 0.1 is 3.0000001: K = 4.  L = 1 over
    s_max = 1/3 (the double 0.333...3148) is 3.0000000000000002 in exact
    arithmetic, so K = 4 although the FP64 product 3 s_max rounds to 1: a tie
    at the 1e-16 level, flagged.  Whole multiples (12 m over 1 m) are exact
    and not flagged."""
    s = _tilted(3, 9000.0, 0.0, seed=2, length=0.3)
    s["length"][1] = np.float32(1.0)
    s["length"][2] = np.float32(12.0)
    from fractions import Fraction
    for s_max in (0.1, 1.0 / 3.0, 1.0):
        r = oracle.propagate(s, ATM, s_max=s_max, bunch=1)
        allr = r["records"]
        rec = _real(allr)
        flagged = set(allr["seg"][(allr["status"] == oracle.ST_SUBSTEP_FLAG) &
                                  ((allr["flags"] & oracle.FL_SEGMENT) != 0)].tolist())
        for i in range(3):
            L = Fraction(float(s["length"][i]))
            q = L / Fraction(s_max)                     # exact rational quotient
            K = max(1, -((-q.numerator) // q.denominator))
            ks = np.unique(rec["k"][rec["seg"] == i])
            assert ks.max() == K - 1 and len(ks) == K, (s_max, i, K, ks)
            tie = q != round(q) and abs(q - round(q)) < Fraction(1, 10**13) * q
            assert (i in flagged) == tie, (s_max, i)
        if s_max == 1.0 / 3.0:
            assert flagged == {1, 2}   # 12 m is 36 sub-steps up to a tie too


# ------------------------------------------------- steep planar photons -----
def _quad_R(h_e, theta0, h_obs=H_OBS):
    """Horizontal displacement and c t of the exact path by scipy's adaptive
    quadrature, split at the layer boundaries."""
    s = (1.0 + oracle.atm_delta(ATM, h_e)) * math.sin(theta0)
    edges = [h_obs] + [b for b in (4000.0, 10000.0, 40000.0, 100000.0) if h_obs < b < h_e] + [h_e]

    def fr(h):
        n = 1.0 + oracle.atm_delta(ATM, h)
        return s / math.sqrt(n * n - s * s)

    def ft(h):
        n = 1.0 + oracle.atm_delta(ATM, h)
        return n * n / math.sqrt(n * n - s * s)

    R = sum(integrate.quad(fr, a, b, epsabs=0, epsrel=1e-12, limit=400)[0] for a, b in zip(edges, edges[1:]))
    T = sum(integrate.quad(ft, a, b, epsabs=0, epsrel=1e-12, limit=400)[0] for a, b in zip(edges, edges[1:]))
    return R, T


@pytest.mark.parametrize("z0,zen", [(2300.0, 80.0), (5000.0, 84.0), (12000.0, 86.5)])
def test_steep_refracted_photons_land_on_the_exact_path(z0, zen):
    s = _tilted(6, z0, zen, seed=3)
    r = oracle.propagate(s, ATM, refraction=True, transmission=True, bunch=1, hist=synth.histogram_400())
    rec = _real(r["records"])
    land = rec[np.isin(rec["status"], [oracle.ST_LANDED, oracle.ST_ABSORBED])]
    assert len(land) > 20 and len(land) == len(rec)          # every photon descends and reaches the ground
    assert np.degrees(land["theta0"]).max() > 75.0
    for p in land[:12]:
        R, ct = _quad_R(p["h_e"], p["theta0"])
        uh = math.hypot(p["ux"], p["uy"])
        assert abs(p["x"] - (p["ex"] + R * p["ux"] / uh)) <= 1e-9 * R
        assert abs(p["y"] - (p["ey"] + R * p["uy"] / uh)) <= 1e-9 * R
        t_emit = p["dt"] - ct / C
        assert 0.0 <= t_emit < 1e-8   # the rest of the time is the emission delay along a 2 m track


# ------------------------------------------------- the spherical shell -----
def _march(h_e, psi0, ds):
    """RK4 on d/ds (n t) = grad n in the plane of travel; returns the smallest
    radius reached and whether the ray met the ground sphere."""
    rg = R_E + H_OBS

    def n_dn(h):
        e = 0.05
        return 1.0 + oracle.atm_delta(ATM, h), (oracle.atm_delta(ATM, h + e) - oracle.atm_delta(ATM, h - e)) / (2 * e)

    def f(y):
        x, z, px, pz = y
        r = math.hypot(x, z)
        n, dn = n_dn(r - R_E)
        return np.array([px / n, pz / n, dn * x / r, dn * z / r])

    n0, _ = n_dn(h_e)
    y = np.array([0.0, R_E + h_e, n0 * math.sin(psi0), -n0 * math.cos(psi0)])
    rmin = R_E + h_e
    for _ in range(200000):
        k1 = f(y)
        k2 = f(y + 0.5 * ds * k1)
        k3 = f(y + 0.5 * ds * k2)
        k4 = f(y + ds * k3)
        y = y + ds / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        r = math.hypot(y[0], y[1])
        if r <= rg:
            return r, True
        if r > rmin + 1.0:   # climbing again: the ray has turned
            return rmin, False
        rmin = min(rmin, r)
    raise AssertionError("ray march did not end")


def test_straight_lines_that_pass_over_the_ground_sphere():
    """Without refraction a photon reaches the ground iff the line's closest
    approach to the Earth's centre lies inside the ground sphere (brute force
    on a fine grid of points along the line)."""
    s = _tilted(40, 3000.0, 88.8, seed=5, length=3.0, x_spread=20000.0)
    r = oracle.propagate(s, ATM, bunch=1, spherical=True, hist=synth.histogram_400())
    rec = _real(r["records"])
    rec = rec[~np.isin(rec["status"], [oracle.ST_UPWARD, oracle.ST_BELOW])]   # descending photons
    assert len(rec) > 100
    rg = R_E + H_OBS
    n_ng = 0
    for p in rec[::7]:
        # rebuild the emission point in frame coordinates from its altitude and footprint
        E = oracle.ae_inverse(p["ex"], p["ey"], dz=p["h_e"] - H_OBS, h_obs=H_OBS)
        u = np.array([p["ux"], p["uy"], p["uz"]])
        ts = np.linspace(0.0, 4.0e5, 400001)
        pts = E[None, :] + ts[:, None] * u[None, :] - np.array([0.0, 0.0, -R_E])[None, :]
        reach = np.linalg.norm(pts, axis=1).min() < rg
        assert (p["status"] != oracle.ST_NO_GROUND) == reach, p
        n_ng += p["status"] == oracle.ST_NO_GROUND
    assert 5 < n_ng < len(rec[::7]) - 5


def test_refracted_rays_that_turn_above_the_ground():
    """With refraction the oracle's decision (Bouguer's invariant against n r
    at the ground) agrees with a Runge-Kutta ray march for photons whose
    margin is not tiny: the ones it keeps meet the ground sphere, the others
    turn and climb."""
    s = _tilted(60, 2600.0, 89.2, seed=6, length=3.0, x_spread=3000.0)
    r = oracle.propagate(s, ATM, bunch=1, spherical=True, refraction=True, hist=synth.histogram_400())
    rec = _real(r["records"])
    rec = rec[~np.isin(rec["status"], [oracle.ST_UPWARD, oracle.ST_BELOW])]
    rg = R_E + H_OBS
    n_g = 1.0 + oracle.atm_delta(ATM, H_OBS)
    checked = {True: 0, False: 0}
    for p in rec:
        K = (1.0 + oracle.atm_delta(ATM, p["h_e"])) * (R_E + p["h_e"]) * math.sin(p["theta0"])
        margin = (n_g * rg - K) / K
        if abs(margin) < 2e-6 or checked[margin > 0] >= 4:
            continue
        _, reached = _march(p["h_e"], p["theta0"], ds=5.0)
        assert reached == (p["status"] != oracle.ST_NO_GROUND), (margin, p["status"])
        checked[margin > 0] += 1
    assert checked[True] >= 2 and checked[False] >= 2
