"""Pins of the oracle's spherical-shell atmosphere (Sec. 3.3.4) against facts
it does not compute itself: the planar limit of an infinite Earth, the
straight line of a homogeneous medium, a brute-force line/sphere
intersection, slant columns integrated along the line in arc length, an
independent Runge-Kutta ray tracer for the refracted path, and the geometry
of the azimuthal-equidistant ground coordinates."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import synth

C = 299_792_458.0
R_E = oracle.EARTH_RADIUS
H_OBS = 2000.0
ATM = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
# one smooth exponential layer below 150 km (the second layer starts above the top)
SMOOTH = dict(layer_h=[0.0, 200000.0], a=[-186.555305, 0.0], b=[1222.6562, 1.0], c=[994186.38, 1.0e9],
              h_top=150000.0, kappa=2.9e-4)
ATM_SMOOTH = oracle.make_atm(oracle.ATM_LAYERED, layered=SMOOTH)
HOM = oracle.make_atm(oracle.ATM_HOMOGENEOUS, hom_delta=2.5e-4)


def _line_to_sphere(h_e, psi0, R=R_E, h_obs=H_OBS):
    """Brute force: the straight line from altitude h_e (local zenith psi0) to
    the ground sphere, by the quadratic of |E + s u - c| = r_g; returns the
    central angle (via atan2 of the landing point) and the length."""
    E = np.array([0.0, R + h_e])                 # centre at the origin, E on the +z axis
    u = np.array([math.sin(psi0), -math.cos(psi0)])
    rg = R + h_obs
    b = E @ u
    c = E @ E - rg * rg
    s = -b - math.sqrt(b * b - c)
    G = E + s * u
    return math.atan2(G[0], G[1]), s


def _simpson(f, a, b, n):
    n += n % 2
    x = np.linspace(a, b, n + 1)
    y = f(x)
    return (b - a) / (3 * n) * (y[0] + y[-1] + 4 * y[1:-1:2].sum() + 2 * y[2:-1:2].sum())


def _gauss(f, a, b, pieces=64):
    """Composite 16-point Gauss-Legendre (numpy's nodes): interior points only,
    so a jump at an end point is never sampled."""
    x, w = np.polynomial.legendre.leggauss(16)
    edges = np.linspace(a, b, pieces + 1)
    mid, half = 0.5 * (edges[1:] + edges[:-1]), 0.5 * (edges[1:] - edges[:-1])
    pts = (mid[:, None] + half[:, None] * x[None, :]).ravel()
    return float((f(pts).reshape(pieces, 16) * w[None, :] * half[:, None]).sum())


@pytest.mark.parametrize("h_e,deg", [(5000.0, 0.0), (12000.0, 30.0), (25000.0, 60.0), (9000.0, 80.0)])
def test_straight_line_matches_line_sphere_intersection(h_e, deg):
    psi = math.radians(deg)
    out = oracle.sph_path(ATM, H_OBS, h_e, psi, refraction=False)
    phi, length = _line_to_sphere(h_e, psi)
    assert out[0] == pytest.approx(phi, abs=1e-14)
    assert out[1] * C == pytest.approx(length, rel=1e-12)


@pytest.mark.parametrize("h_e,deg", [(12000.0, 30.0), (25000.0, 60.0), (9000.0, 80.0)])
def test_straight_columns_along_arc_length(h_e, deg):
    """X and A integrated along the 3D line in arc length (the oracle
    integrates in altitude with the r / q0 Jacobian)."""
    psi = math.radians(deg)
    out = oracle.sph_path(ATM, H_OBS, h_e, psi, refraction=False)
    _, length = _line_to_sphere(h_e, psi)
    re = R_E + h_e

    def alt(s):
        return np.sqrt(re * re - 2.0 * re * math.cos(psi) * s + s * s) - R_E

    # pieces between the crossings of the layer boundaries, where the density fit has kinks
    cuts = [0.0]
    for hb in sorted(synth.US_STANDARD["layer_h"], reverse=True):
        if H_OBS < hb < h_e:
            rb = R_E + hb
            cuts.append(re * math.cos(psi) - math.sqrt(rb * rb - (re * math.sin(psi)) ** 2))
    cuts.append(length)
    rho = np.vectorize(lambda h: oracle.atm_rho(ATM, h))
    X = sum(_gauss(lambda s: 100.0 * rho(alt(s)), a, b) for a, b in zip(cuts[:-1], cuts[1:]))
    A = sum(_gauss(lambda s: np.exp(-alt(s) / 1200.0), a, b) for a, b in zip(cuts[:-1], cuts[1:]))
    assert out[2] == pytest.approx(X, rel=1e-11)
    assert out[3] == pytest.approx(A, rel=1e-11)


@pytest.mark.parametrize("h_e,deg", [(12000.0, 30.0), (25000.0, 60.0), (9000.0, 80.0)])
def test_homogeneous_medium_is_the_straight_line(h_e, deg):
    """Constant n bends nothing: the refracted central angle is the straight
    line's and the time is n times its length over c."""
    psi = math.radians(deg)
    out = oracle.sph_path(HOM, H_OBS, h_e, psi, refraction=True)
    phi, length = _line_to_sphere(h_e, psi)
    assert out[0] == pytest.approx(phi, rel=1e-10, abs=1e-15)
    assert out[1] * C == pytest.approx((1.0 + 2.5e-4) * length, rel=1e-10)


@pytest.mark.parametrize("h_e,deg", [(12000.0, 30.0), (25000.0, 60.0), (9000.0, 75.0)])
def test_infinite_earth_is_the_planar_atmosphere(h_e, deg):
    """As R_E grows, the arc length on the ground sphere, the time and the
    columns approach the planar refracted path (Eq. 3.17 and 3.18), with the
    curvature terms falling as 1 / R_E."""
    psi = math.radians(deg)
    pla = oracle.refract_quad(ATM, H_OBS, h_e, psi)

    def rel(R):
        sph = oracle.sph_path(ATM, H_OBS, h_e, psi, refraction=True, R=R)
        return np.array([sph[0] * (R + H_OBS), sph[1], sph[2], sph[3]]) / pla - 1.0

    far, farther = rel(1e12), rel(1e14)
    assert np.all(np.abs(farther) < 2e-9)
    np.testing.assert_allclose(far, 100.0 * farther, rtol=1e-2)


def test_vertical_photon():
    out = oracle.sph_path(ATM, H_OBS, 20000.0, 0.0, refraction=True)
    assert out[0] == 0.0
    assert out[2] == pytest.approx(oracle.straight(ATM, H_OBS, 20000.0, 0.0)[2], rel=1e-9)
    # time: integral of n dh / c, by Simpson in altitude
    n = np.vectorize(lambda h: 1.0 + oracle.atm_delta(ATM, h))
    ct = _gauss(n, H_OBS, 4000.0) + _gauss(n, 4000.0, 10000.0) + _gauss(n, 10000.0, 20000.0)
    assert out[1] * C == pytest.approx(ct, rel=1e-12)


def _ray_trace(atm, h_e, psi0, ds, R=R_E, h_obs=H_OBS):
    """Runge-Kutta 4 on the ray equation d/ds (n t) = grad n in the plane of
    travel (centre at the origin), until the ray meets the ground sphere.
    Returns (central angle, c t, arrival zenith)."""
    def n_and_dn(h):
        d = oracle.atm_delta(atm, h)
        e = 0.05
        return 1.0 + d, (oracle.atm_delta(atm, h + e) - oracle.atm_delta(atm, h - e)) / (2 * e)

    def f(y):
        x, z, px, pz, _ = y
        r = math.hypot(x, z)
        n, dn = n_and_dn(r - R)
        return np.array([px / n, pz / n, dn * x / r, dn * z / r, n])

    n0, _ = n_and_dn(h_e)
    y = np.array([0.0, R + h_e, n0 * math.sin(psi0), -n0 * math.cos(psi0), 0.0])
    rg = R + h_obs
    while True:
        k1 = f(y)
        k2 = f(y + 0.5 * ds * k1)
        k3 = f(y + 0.5 * ds * k2)
        k4 = f(y + ds * k3)
        y2 = y + ds / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        if math.hypot(y2[0], y2[1]) <= rg:
            # last partial step: bisect the step length on the ground sphere
            lo, hi = 0.0, ds
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                k1 = f(y)
                k2 = f(y + 0.5 * mid * k1)
                k3 = f(y + 0.5 * mid * k2)
                k4 = f(y + mid * k3)
                ym = y + mid / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
                if math.hypot(ym[0], ym[1]) > rg:
                    lo = mid
                else:
                    hi = mid
            y = ym
            break
        y = y2
    x, z, px, pz, ct = y
    r = math.hypot(x, z)
    cos_g = -(px * x + pz * z) / (r * math.hypot(px, pz))
    return math.atan2(x, z), ct, math.acos(min(1.0, cos_g))


@pytest.mark.parametrize("h_e,deg", [(8000.0, 30.0), (15000.0, 60.0), (6000.0, 78.0)])
def test_refracted_path_matches_ray_tracer(h_e, deg):
    psi = math.radians(deg)
    phi_rk, ct_rk, zen_rk = _ray_trace(ATM_SMOOTH, h_e, psi, ds=10.0)
    out = oracle.sph_path(ATM_SMOOTH, H_OBS, h_e, psi, refraction=True)
    rg = R_E + H_OBS
    assert out[0] * rg == pytest.approx(phi_rk * rg, abs=2e-3)
    assert out[1] * C == pytest.approx(ct_rk, abs=2e-3)
    # refraction is resolved: the bending differs from the straight line by far more than the tolerance
    phi_line, _ = _line_to_sphere(h_e, psi)
    assert abs(phi_line - phi_rk) * rg > 0.5 if deg > 45 else abs(phi_line - phi_rk) * rg > 0.05
    # Bouguer's invariant n r sin(psi) gives the tracer's arrival zenith
    n_e = 1.0 + oracle.atm_delta(ATM_SMOOTH, h_e)
    n_g = 1.0 + oracle.atm_delta(ATM_SMOOTH, H_OBS)
    s_g = n_e * (R_E + h_e) * math.sin(psi) / (n_g * rg)
    assert math.asin(s_g) == pytest.approx(zen_rk, abs=1e-9)


@pytest.mark.parametrize("x,y,dz", [(0.0, 0.0, 0.0), (1500.0, -700.0, 0.0), (-30000.0, 42000.0, 12.5)])
def test_azimuthal_equidistant_inverse(x, y, dz):
    """The point lies at radius r_g + dz from the centre, at the central angle
    (ground distance / r_g) from the array centre, at the azimuth of (x, y)."""
    P = oracle.ae_inverse(x, y, dz=dz, h_obs=H_OBS)
    c = np.array([0.0, 0.0, -R_E])
    rg = R_E + H_OBS
    v = P - c
    assert np.linalg.norm(v) == pytest.approx(rg + dz, rel=1e-15)
    ang = math.atan2(math.hypot(v[0], v[1]), v[2])
    assert ang * rg == pytest.approx(math.hypot(x, y), abs=1e-8)
    if x or y:
        assert math.atan2(v[1], v[0]) == pytest.approx(math.atan2(y, x), abs=1e-12)


def _inclined(n, seed, zenith=60.0, azimuth=30.0):
    s = synth.shower_segments(n, zenith, azimuth, 1e13, seed)
    return s


def test_propagate_straight_on_the_sphere_brute_force():
    """Each photon by hand: the emission point from the segment and its
    draws, the 3D straight line to the ground sphere, the ground point's
    azimuthal-equidistant coordinates and the arrival time."""
    segs = _inclined(40, seed=3)
    res = oracle.propagate(segs, ATM, spherical=True, seed=11, bunch=1)
    rec = res["records"]
    landed = rec[rec["status"] == oracle.ST_LANDED]
    assert len(landed) > 500
    key = (11 & 0xFFFFFFFF, 11 >> 32)
    c = np.array([0.0, 0.0, -R_E])
    rg = R_E + H_OBS
    for r in landed[:: max(1, len(landed) // 300)]:
        j = int(r["seg"])
        P = np.array([segs["ux"][j], segs["uy"][j], segs["uz"][j]], np.float64)
        P /= np.linalg.norm(P)
        L = float(segs["length"][j])
        K = max(1, math.ceil(np.float32(L) / np.float32(1.0)))
        w = oracle.philox([j & 0xFFFFFFFF, j >> 32, int(r["k"]), int(r["i"])], key)
        u0 = (w[0] >> 8) * 2.0**-24
        ell = (int(r["k"]) + u0) / K * L
        E = np.array([segs["x0"][j], segs["y0"][j], segs["z0"][j]]) + ell * P
        u = np.array([r["ux"], r["uy"], r["uz"]])
        d = E - c
        b = d @ u
        s = -b - math.sqrt(b * b - (d @ d - rg * rg))
        G = E + s * u
        rho = math.hypot(G[0], G[1])
        a = math.atan2(rho, G[2] + R_E) * rg
        assert r["x"] == pytest.approx(a * G[0] / rho, abs=1e-6)
        assert r["y"] == pytest.approx(a * G[1] / rho, abs=1e-6)
        g = 1.0 / math.sqrt(float(segs["inv_gamma2"][j]))
        beta = math.sqrt(1.0 - 1.0 / (g * g))
        assert r["dt"] == pytest.approx(ell / (beta * C) + s / C, rel=1e-12, abs=1e-18)
        assert r["h_e"] == pytest.approx(np.linalg.norm(d) - R_E, abs=1e-6)


def test_propagate_infinite_earth_is_planar():
    """Full propagation with refraction and transmission: a spherical shell
    with R_E = 1e12 m reproduces the planar photons and detections."""
    segs = _inclined(200, seed=5)
    tel = synth.grid_telescopes()
    hist = synth.histogram_400()
    kw = dict(seed=4, bunch=2, refraction=True, transmission=True, tel=tel, hist=hist)
    pla = oracle.propagate(segs, ATM, **kw)
    sph = oracle.propagate(segs, ATM, spherical=True, earth_radius=1e12, **kw)
    a, b = pla["records"], sph["records"]
    assert len(a) == len(b) and np.array_equal(a["seg"], b["seg"]) and np.array_equal(a["i"], b["i"])
    ok = (a["status"] == oracle.ST_LANDED) & (b["status"] == oracle.ST_LANDED)
    assert ok.sum() > 1000
    # coordinates near 1e12 m carry 1e-4 m of rounding
    np.testing.assert_allclose(b["x"][ok], a["x"][ok], atol=2e-3)
    np.testing.assert_allclose(b["y"][ok], a["y"][ok], atol=2e-3)
    np.testing.assert_allclose(b["dt"][ok], a["dt"][ok], rtol=0, atol=5e-12)   # 1.5 mm of light travel
    np.testing.assert_allclose(b["T"][ok], a["T"][ok], rtol=1e-6)
    same = (a["status"] == b["status"]).mean()
    assert same > 0.999
    assert (a["tel"][ok] == b["tel"][ok]).mean() > 0.999


def test_substep_yield_uses_the_altitude_on_the_sphere():
    """60 km from the array centre a point at frame height z lies ~283 m
    higher above the ground sphere: the sub-step's mean count (Eq. 2.2-2.5)
    takes n at that altitude, not at z."""
    n = 4
    segs = synth._empty(n)
    segs["x0"][:] = 60000.0
    segs["z0"][:] = [6000.0, 9000.0, 12000.0, 15000.0]
    segs["uz"][:] = -1.0
    segs["length"][:] = 2.0
    segs["inv_gamma2"][:] = np.float32(1e-8)
    res = oracle.propagate(segs, ATM, spherical=True, bunch=1, seed=1)
    rec = res["records"]
    alpha = 7.2973525693e-3
    ft = 2.0 * math.pi * alpha * (1.0 / 300e-9 - 1.0 / 600e-9)
    beta2 = 1.0 - float(np.float32(1e-8))
    for j in range(n):
        r = rec[rec["seg"] == j]
        assert len(r) > 0
        for k in (0, 1):
            z_mid = segs["z0"][j] - (k + 0.5)
            alt = math.sqrt(60000.0**2 + (z_mid + R_E) ** 2) - R_E
            assert alt - z_mid == pytest.approx(60000.0**2 / (2 * R_E), rel=1e-2)
            nn = 1.0 + oracle.atm_delta(ATM, alt)
            want = ft * (1.0 - 1.0 / (beta2 * nn * nn))
            got = r["nbar"][r["k"] == k]
            assert len(got) > 0 and np.allclose(got, want, rtol=1e-12)
            n_flat = 1.0 + oracle.atm_delta(ATM, z_mid)
            assert abs(ft * (1.0 - 1.0 / (beta2 * n_flat * n_flat)) / want - 1.0) > 5e-3
