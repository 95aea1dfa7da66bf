"""Pins of the oracle's cylindrical atmosphere (Sec. 3.3.3).

The model leans the index gradient in zenith only, inside the vertical plane
through the array centre and the emission point: per photon the atmosphere is
a set of coaxial cylinders about the horizontal axis through the Earth's
centre normal to that plane.  The oracle integrates the path through the two
invariants of that symmetry (n u_a along the axis, n rho u_chi about it).
Each pin below checks it against something else:

* with no axial component the path is the spherical shell's (pinned there);
* the vacuum straight line against the line-cylinder intersection in closed
  form, through the whole propagation (frame, axis, sign and unrolled ground);
* the refracted path against an independent Runge-Kutta march of the ray
  equation d(n u)/ds = grad n in three dimensions;
* the thesis's Snell stepper in three dimensions converges to it;
* the reach condition against a brute-force scan and against the march;
* a radius of 1e12 m gives the planar atmosphere.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import synth

C = 299_792_458.0
R_E = oracle.EARTH_RADIUS
H_OBS = 2000.0
ATM = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)


# heights where n jumps: the layered profile's density is continuous in its
# overburden, not in itself, so the index steps at every layer boundary
JUMPS = sorted(list(synth.US_STANDARD["layer_h"][1:]) + [synth.US_STANDARD["h_top"]])


def _n(h):
    return 1.0 + oracle.atm_delta(ATM, h)


def _dn(h, eps=0.01):
    """dn/dh by differences that stay inside h's layer (one-sided at its edges)."""
    lo = max([b for b in JUMPS if b <= h], default=-1e30)
    hi = min([b for b in JUMPS if b > h], default=1e30)
    e = min(eps, 0.5 * (h - lo), 0.5 * (hi - h))
    if e > 1e-4:
        return (oracle.atm_delta(ATM, h + e) - oracle.atm_delta(ATM, h - e)) / (2.0 * e)
    if h - lo < hi - h:   # at the layer's lower edge: forward difference
        return (oracle.atm_delta(ATM, h + eps) - oracle.atm_delta(ATM, h)) / eps
    return (oracle.atm_delta(ATM, h) - oracle.atm_delta(ATM, h - eps)) / eps


def _frame(E, R=R_E):
    """e_r (towards E's foot), e_a = z x e_r, and the transverse tangent e_chi at E."""
    d = math.hypot(E[0], E[1])
    er = np.array([E[0] / d, E[1] / d, 0.0]) if d > 0 else np.array([1.0, 0.0, 0.0])
    ea = np.array([-er[1], er[0], 0.0])
    rho = math.hypot(d, E[2] + R)
    s_chi, c_chi = d / rho, (E[2] + R) / rho
    echi = c_chi * er - s_chi * np.array([0.0, 0.0, 1.0])
    return er, ea, echi, rho - R


def _march(E, u, R=R_E, ds=2.0, refraction=True, s_max=2e5):
    """RK4 march of dP/ds = w / n, dw/ds = grad n (w = n u) through n(rho - R),
    rho the distance from the axis through (0, 0, -R) along e_a; at a jump of n
    the step ends on the interface and Snell's law keeps w's tangential part.
    Returns the ground point's (chi, a), the time, the smallest altitude seen,
    and whether it reached the ground cylinder."""
    er, ea, _, _ = _frame(E, R)
    Cc = np.array([0.0, 0.0, -R])
    rg = R + H_OBS

    def rho_h(P):
        q = P - Cc
        t = q - (q @ ea) * ea
        r = math.sqrt(t @ t)
        return r, r - R, t / r

    def f(state):
        P, w = state[:3], state[3:6]
        _, h, rhat = rho_h(P)
        n = _n(h) if refraction else 1.0
        g = (_dn(h) if refraction else 0.0) * rhat
        return np.concatenate([w / n, g, [n / C]])

    def rk4(y, d):
        k1 = f(y)
        k2 = f(y + 0.5 * d * k1)
        k3 = f(y + 0.5 * d * k2)
        k4 = f(y + d * k3)
        return y + d / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)

    def to_height(y, target, d):
        """a step from y that ends at altitude `target` (secant on the step length)."""
        h0 = rho_h(y[:3])[1]
        a, b = 0.0, d
        hb = rho_h(rk4(y, b)[:3])[1]
        ha = h0
        for _ in range(60):
            m = b - (hb - target) * (b - a) / (hb - ha)
            hm = rho_h(rk4(y, m)[:3])[1]
            if abs(hm - target) < 1e-9:
                return rk4(y, m)
            a, ha, b, hb = b, hb, m, hm
        return rk4(y, b)

    n0 = _n(_frame(E, R)[3]) if refraction else 1.0
    y = np.concatenate([np.asarray(E, float), n0 * np.asarray(u, float), [0.0]])
    h_min, s = 1e30, 0.0
    while s < s_max:
        y1 = rk4(y, ds)
        _, h0, _ = rho_h(y[:3])
        r1, h1, _ = rho_h(y1[:3])
        crossed = [b for b in JUMPS if (h0 - b) * (h1 - b) < 0.0] if refraction else []
        if r1 <= rg:   # the ground cylinder: end the march on it
            yg = to_height(y, H_OBS, ds)
            h_min = min(h_min, H_OBS)
            q = yg[:3] - Cc
            return dict(chi=math.atan2(q @ er, q[2]), a=q @ ea, t=yg[6], h_min=h_min, reached=True)
        if crossed:   # step onto the interface and refract there (Eq. 3.15)
            b = crossed[0] if h1 < h0 else crossed[-1]
            y1 = to_height(y, b, ds)
            _, _, rhat = rho_h(y1[:3])
            w = y1[3:6]
            wn = w @ rhat
            n_new = _n(b - 1e-7) if h1 < h0 else _n(b + 1e-7)
            wt = w - wn * rhat
            rad = n_new * n_new - wt @ wt
            y1[3:6] = wt + (math.copysign(math.sqrt(rad), wn) if rad > 0 else -wn) * rhat
            y1[:3] += (-1e-6 if h1 < h0 else 1e-6) * rhat   # past the interface
            h1 = rho_h(y1[:3])[1]
        h_min = min(h_min, h1)
        if h1 > h0 and h1 > 120e3:
            break
        y, s = y1, s + ds
    return dict(h_min=h_min, reached=False)


def _direction(zen_deg, az_deg):
    th, ph = math.radians(zen_deg), math.radians(az_deg)
    return np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), -math.cos(th)])


def _components(E, u, R=R_E):
    er, ea, echi, h_e = _frame(E, R)
    return float(u @ ea), float(u @ echi), h_e, er, ea


# --------------------------------------------------------- reductions ------
@pytest.mark.parametrize("h_e,psi_deg", [(5000.0, 10.0), (12000.0, 40.0), (20000.0, 70.0), (30000.0, 78.0)])
def test_no_axial_component_is_the_spherical_shell(h_e, psi_deg):
    psi = math.radians(psi_deg)
    c = oracle.cyl_path(ATM, H_OBS, h_e, 0.0, math.sin(psi))
    s = oracle.sph_path(ATM, H_OBS, h_e, psi)
    assert c[2] == 0.0
    np.testing.assert_allclose(c[[0, 1, 3, 4]], s, rtol=1e-11)


@pytest.mark.parametrize("E,zen,az", [((3000.0, -1000.0, 9000.0), 35.0, 70.0),
                                      ((-20000.0, 5000.0, 15000.0), 60.0, 200.0),
                                      ((500.0, 800.0, 4000.0), 80.0, 10.0)])
def test_straight_line_is_the_line_cylinder_intersection(E, zen, az):
    """refraction off: chi swept, axial drift and length equal the closed-form
    crossing of E + s u with the ground cylinder."""
    u = _direction(zen, az)
    ua, uchi, h_e, er, ea = _components(E, u)
    p = oracle.cyl_path(ATM, H_OBS, h_e, ua, abs(uchi), refraction=False)
    Cc = np.array([0.0, 0.0, -R_E])
    q0 = np.asarray(E) - Cc
    t0 = q0 - (q0 @ ea) * ea
    ut = u - (u @ ea) * ea
    rg = R_E + H_OBS
    A, B, Cq = ut @ ut, 2 * (t0 @ ut), t0 @ t0 - rg * rg
    s = (-B - math.sqrt(B * B - 4 * A * Cq)) / (2 * A)
    q1 = q0 + s * u
    chi0, chi1 = math.atan2(q0 @ er, q0[2]), math.atan2(q1 @ er, q1[2])
    assert p[0] == pytest.approx(abs(chi1 - chi0), rel=1e-9)
    assert math.copysign(1.0, chi1 - chi0) == math.copysign(1.0, uchi)
    assert p[1] * C == pytest.approx(s, rel=1e-10)
    assert p[2] == pytest.approx(s * ua, rel=1e-9, abs=1e-9)


# ------------------------------------------------------- refracted path ----
@pytest.mark.parametrize("E,zen,az", [((3000.0, -1000.0, 9000.0), 35.0, 70.0),
                                      ((-20000.0, 5000.0, 15000.0), 60.0, 200.0),
                                      ((800.0, 500.0, 6000.0), 75.0, 95.0)])
def test_refracted_path_against_a_ray_march(E, zen, az):
    """The invariants' quadrature lands where a Runge-Kutta march of the ray
    equation does: chi swept and axial drift to 2e-9 of the path, time to 1e-9."""
    u = _direction(zen, az)
    ua, uchi, h_e, er, ea = _components(E, u)
    p = oracle.cyl_path(ATM, H_OBS, h_e, ua, abs(uchi))
    m = _march(E, u, ds=1.0)
    assert m["reached"]
    q0 = np.asarray(E) - np.array([0.0, 0.0, -R_E])
    chi0 = math.atan2(q0 @ er, q0[2])
    path = p[1] * C
    rg = R_E + H_OBS
    assert abs(rg * (m["chi"] - chi0) - rg * math.copysign(p[0], uchi)) < 2e-9 * path
    assert abs(m["a"] - p[2]) < 2e-9 * path
    assert m["t"] == pytest.approx(p[1], rel=1e-9)


def test_refraction_bends_the_axial_drift_and_the_sweep():
    """Against the straight line from the same point, refraction shortens the
    sweep (the ray bends towards the vertical) and the axial drift: the
    invariant n u_a = A makes u_a shrink as n grows on the way down."""
    E = np.array([4000.0, 2000.0, 12000.0])
    u = _direction(70.0, 150.0)
    ua, uchi, h_e, _, _ = _components(E, u)
    r = oracle.cyl_path(ATM, H_OBS, h_e, ua, abs(uchi))
    v = oracle.cyl_path(ATM, H_OBS, h_e, ua, abs(uchi), refraction=False)
    assert r[0] < v[0] and abs(r[2]) < abs(v[2])


@pytest.mark.parametrize("zen,az", [(40.0, 30.0), (70.0, 120.0)])
def test_snell_stepper_converges_to_the_quadrature(zen, az):
    """Eq. 3.15 at coaxial cylinders (three-dimensional vectors): the error of
    every field shrinks with the shell thickness."""
    E = np.array([-6000.0, 3000.0, 14000.0])
    u = _direction(zen, az)
    ua, uchi, h_e, _, _ = _components(E, u)
    exact = oracle.cyl_path(ATM, H_OBS, h_e, ua, abs(uchi))
    cos_z = math.sqrt(max(1.0 - ua * ua - uchi * uchi, 0.0))
    errs = []
    for dh in (40.0, 10.0, 2.5):
        st = oracle.snell_path_cyl(ATM, H_OBS, h_e, abs(uchi), -cos_z, ua, dh)
        errs.append(np.abs(st - exact) / np.abs(exact))
    errs = np.array(errs)
    # geometry and time: at least first order, each 4x refinement cuts the error 3x
    # or more (the index jumps at the layer boundaries refract at the nearest shell
    # boundary instead of their own height)
    assert (errs[2, :3] < 1e-7).all(), errs
    assert (errs[1, :3] <= errs[0, :3] / 3).all() and (errs[2, :3] <= errs[1, :3] / 3).all(), errs
    # slant columns: a shell straddling a density jump holds its midpoint density,
    # an error of first order in dh
    assert (errs[2, 3:] < 1e-5).all() and (errs[2, 3:] <= errs[0, 3:] * 0.1).all(), errs


# ------------------------------------------------------ reach condition ----
def _scan_margin(h_e, ua, uchi, refraction=True, n=200001):
    ne = _n(h_e) if refraction else 1.0
    A, L = ne * ua, ne * (R_E + h_e) * abs(uchi)
    hs = np.linspace(H_OBS, h_e, n)
    nn = np.array([_n(h) for h in hs]) if refraction else np.ones(n)
    return float(((np.sqrt(nn * nn - A * A) * (R_E + hs) - L) / L).min())


@pytest.mark.parametrize("h_e,ua,uchi", [(15000.0, 0.3, 0.94), (8000.0, 0.1, 0.99), (25000.0, 0.9, 0.42),
                                         (6000.0, 0.96, 0.27)])
def test_reach_margin_is_the_scanned_minimum(h_e, ua, uchi):
    """(N rho - L) / L minimised over the path: the golden-section pieces
    agree with a 200001-point scan (the scan can only be larger)."""
    m = oracle.cyl_reach_margin(ATM, H_OBS, h_e, ua, uchi)
    s = _scan_margin(h_e, ua, uchi, n=40001)
    assert m <= s + 1e-12
    assert s - m < 1e-9


def test_grazing_photons_turn_above_the_ground_where_the_margin_is_negative():
    """Photons launched a little below the horizontal from 3 km up: where the
    margin is negative the ray march turns back above the ground cylinder,
    where it is positive the march reaches the ground."""
    seen = set()
    for dip in (0.05, 0.3, 0.6, 1.2):
        E = np.array([2000.0, 1000.0, 3000.0])
        er, ea, echi, h_e = _frame(E)
        vloc = np.cross(echi, ea)   # the local vertical
        d = math.radians(dip)
        u = math.cos(d) * (0.6 * echi + 0.8 * ea) - math.sin(d) * vloc
        ua, uchi = float(u @ ea), float(u @ echi)
        margin = oracle.cyl_reach_margin(ATM, H_OBS, h_e, ua, uchi)
        m = _march(E, u, ds=20.0, s_max=3e5)
        assert m["reached"] == (margin > 0.0), (dip, margin, m)
        seen.add(margin > 0.0)
    assert seen == {True, False}


# ------------------------------------------------- whole propagation -------
def _segments(n, seed, x_spread=20000.0, z_lo=4000.0, z_hi=20000.0):
    """Tracks spread over tens of km with directions up to 70 degrees from the
    vertical (fast electrons, 2 m long)."""
    rng = np.random.default_rng(seed)
    s = synth._empty(n)
    s["x0"][:] = rng.uniform(-x_spread, x_spread, n)
    s["y0"][:] = rng.uniform(-x_spread, x_spread, n)
    s["z0"][:] = rng.uniform(z_lo, z_hi, n)
    th, ph = np.radians(rng.uniform(0.0, 70.0, n)), rng.uniform(0.0, 2 * math.pi, n)
    s["ux"][:] = (np.sin(th) * np.cos(ph)).astype(np.float32)
    s["uy"][:] = (np.sin(th) * np.sin(ph)).astype(np.float32)
    s["uz"][:] = (-np.cos(th)).astype(np.float32)
    s["length"][:] = 2.0
    s["inv_gamma2"][:] = np.float32(1e-8)
    s["charge"][:] = 1.0
    return s


def test_propagation_lays_straight_lines_on_the_unrolled_cylinder():
    """Refraction off: every landed photon's ground point is the closed-form
    crossing of its emission line with the ground cylinder about its own axis,
    unrolled (the emission point rebuilt from the record's footprint and
    altitude); its time is the line's length over c plus an emission delay
    along the 2 m track."""
    s = _segments(60, seed=3)
    r = oracle.propagate(s, ATM, bunch=1, cylindrical=True)
    rec = r["records"]
    rec = rec[rec["status"] == oracle.ST_LANDED]
    assert len(rec) > 500
    rg = R_E + H_OBS
    Cc = np.array([0.0, 0.0, -R_E])
    for p in rec[::5]:
        F = np.array([p["ex"], p["ey"]])
        chi_e = np.hypot(*F) / rg
        er = np.array([F[0], F[1], 0.0]) / np.hypot(*F)
        ea = np.array([-er[1], er[0], 0.0])
        q0 = (R_E + p["h_e"]) * (math.sin(chi_e) * er + math.cos(chi_e) * np.array([0.0, 0.0, 1.0]))
        u = np.array([p["ux"], p["uy"], p["uz"]])
        t0 = q0 - (q0 @ ea) * ea
        ut = u - (u @ ea) * ea
        A, B, Cq = ut @ ut, 2 * (t0 @ ut), t0 @ t0 - rg * rg
        sl = (-B - math.sqrt(B * B - 4 * A * Cq)) / (2 * A)
        q1 = q0 + sl * u
        G = rg * math.atan2(q1 @ er, q1[2]) * er[:2] + (q1 @ ea) * ea[:2]
        assert abs(G[0] - p["x"]) < 1e-9 * sl and abs(G[1] - p["y"]) < 1e-9 * sl, (G, p)
        t_emit = p["dt"] - sl / C
        assert -1e-15 <= t_emit < 1e-8


def test_a_huge_radius_gives_the_planar_atmosphere():
    """R = 1e12 m: the cylinders flatten into the planar layers; statuses agree
    exactly, ground points to 5e-7 of the displacement (FP64 resolves 1.2e-4 m
    at 1e12 m, and the residual curvature d^2 / 2R is 2e-4 m for tracks 20 km
    from the centre), times to 5e-7 (the altitude of an emission point 1e12 m
    from the Earth's centre carries the same 1e-4 m)."""
    s = _segments(40, seed=4, x_spread=20000.0)
    kw = dict(bunch=1, refraction=True, transmission=True, seed=9)
    c = oracle.propagate(s, ATM, cylindrical=True, earth_radius=1e12, **kw)
    pl = oracle.propagate(s, ATM, **kw)
    a, b = c["records"], pl["records"]
    assert len(a) == len(b)
    assert np.array_equal(a["status"], b["status"])
    m = a["status"] == oracle.ST_LANDED
    assert m.sum() > 300
    disp = np.maximum(1.0, np.hypot(b["x"] - b["ex"], b["y"] - b["ey"]))[m]
    assert (np.abs(a["x"] - b["x"])[m] / disp).max() < 5e-7
    assert (np.abs(a["y"] - b["y"])[m] / disp).max() < 5e-7
    assert (np.abs(a["dt"] / b["dt"] - 1.0)[m]).max() < 5e-7
