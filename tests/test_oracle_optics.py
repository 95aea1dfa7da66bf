"""Pins of the oracle's last-mile ray tracing (Sec. 6.4): a parabolic mirror
images rays parallel to its axis onto the focus, tilted rays about f tan(a)
off centre, the camera shadows the rays that meet it first, and the aperture
and camera rims bound the hits."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import synth

OPT = dict(mirror_d=7.0, focal_f=8.0, camera_r=0.5, point_zenith=math.radians(20.0),
           point_azimuth=math.radians(30.0), cam_n=41)
C0 = np.array([100.0, -50.0, 2000.0])


def _frame():
    th, ph = OPT["point_zenith"], OPT["point_azimuth"]
    a = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    e1 = np.cross(a, [0.0, 0.0, 1.0])
    e1 /= np.linalg.norm(e1)
    return a, e1, np.cross(a, e1)


def _ray(rho, phi, tilt=0.0, tilt_dir=0.0):
    """A ray that crosses the aperture plane at (rho, phi) from the axis,
    tilted by `tilt` from the axis towards `tilt_dir`."""
    a, e1, e2 = _frame()
    w = -a * math.cos(tilt) + math.sin(tilt) * (math.cos(tilt_dir) * e1 + math.sin(tilt_dir) * e2)
    V = C0 - 0.5 * OPT["focal_f"] * a
    P = V + rho * (math.cos(phi) * e1 + math.sin(phi) * e2)   # a point on the ray in the vertex plane
    return P, w


@pytest.mark.parametrize("rho", [0.6, 1.3, 2.2, 3.4])
@pytest.mark.parametrize("phi", [0.0, 1.1, 2.9, 4.4])
def test_rays_parallel_to_the_axis_meet_at_the_focus(rho, phi):
    P, w = _ray(rho, phi)
    pix, xy = oracle.camera_trace(C0, P, w, OPT)
    assert pix >= 0
    assert np.hypot(*xy) < 1e-9
    n = OPT["cam_n"]
    assert pix == (n // 2) * n + n // 2          # the centre pixel (odd n: the focus is its centre)


def test_tilted_rays_land_at_f_tan_alpha():
    f = OPT["focal_f"]
    for tilt in (0.005, 0.01, 0.02):
        for tdir in (0.0, 1.0, 2.5):
            pts = [oracle.camera_trace(C0, *_ray(rho, phi, tilt, tdir), OPT)[1]
                   for rho in (0.7, 1.0) for phi in np.linspace(0, 2 * math.pi, 8, endpoint=False)]
            c = np.mean(pts, axis=0)
            assert np.hypot(*c) == pytest.approx(f * math.tan(tilt), rel=0.03)
            # a source on the -t side of the axis (the ray travels towards +t) images on the +t side
            assert np.dot(c, [math.cos(tdir), math.sin(tdir)]) > 0.99 * np.hypot(*c)


def test_camera_shadow_and_rims():
    assert oracle.camera_trace(C0, *_ray(0.3, 0.7), OPT)[0] == -1          # meets the camera first
    assert oracle.camera_trace(C0, *_ray(3.6, 0.7), OPT)[0] == -1          # outside the aperture
    assert oracle.camera_trace(C0, *_ray(3.4, 0.7), OPT)[0] >= 0
    assert oracle.camera_trace(C0, *_ray(2.0, 0.7, 0.08), OPT)[0] == -1    # image beyond the camera rim
    P, w = _ray(2.0, 0.7)
    assert oracle.camera_trace(C0, P, -w, OPT)[0] == -1                     # travelling away from the mirror


def test_propagation_camera_images_equal_the_records():
    segs = synth.shower_segments(1200, 20.0, 30.0, 1e12, seed=4)
    tel = synth.grid_telescopes(nx=4, ny=4, pitch=60.0)
    r = oracle.propagate(segs, oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD), tel=tel, bunch=2,
                         refraction=True, transmission=True, seed=1, optics=OPT)
    rec = r["records"]
    hit = (rec["status"] == oracle.ST_LANDED) & (rec["tel"] >= 0) & (rec["pix"] >= 0)
    assert hit.sum() > 20
    img = np.zeros_like(r["camera"])
    np.add.at(img.reshape(1, len(tel), -1), (0, rec["tel"][hit], rec["pix"][hit]), 2)
    assert np.array_equal(img, r["camera"])
    assert (rec["pix"][rec["tel"] < 0] == -1).all()


def _march(P, w):
    """Independent trace: the ray P + t w in the telescope frame, the mirror
    found by bisection on r^2 - 4 f z along the ray below the camera plane."""
    f, R, rd = OPT["focal_f"], OPT["camera_r"], OPT["mirror_d"] / 2
    a, e1, e2 = _frame()
    V = C0 - 0.5 * f * a
    M = np.stack([e1, e2, a])
    p, d = M @ (P - V), M @ w
    if d[2] >= 0:
        return None
    tc = (f - p[2]) / d[2]
    if np.hypot(*(p[:2] + tc * d[:2])) < R:
        return None
    F = lambda t: (p[0] + t * d[0]) ** 2 + (p[1] + t * d[1]) ** 2 - 4 * f * (p[2] + t * d[2])
    lo, hi = tc, tc + 4 * f / -d[2]          # inside the bowl at the camera plane, below the vertex later
    if not (F(lo) < 0 < F(hi)):
        return None
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if F(mid) < 0 else (lo, mid)
    m = p + 0.5 * (lo + hi) * d
    if np.hypot(m[0], m[1]) > rd:
        return None
    n = np.array([m[0], m[1], -2 * f]) / np.linalg.norm([m[0], m[1], -2 * f])
    r = d - 2 * np.dot(d, n) * n
    q = m + (f - m[2]) / r[2] * r
    return q[:2] if np.hypot(*q[:2]) <= R else None


def test_camera_points_match_an_independent_ray_march():
    rng = np.random.default_rng(11)
    hits = 0
    for _ in range(300):
        rho, phi = rng.uniform(0.0, 3.6), rng.uniform(0, 2 * math.pi)
        tilt, tdir = abs(rng.normal(0.0, 0.02)), rng.uniform(0, 2 * math.pi)
        P, w = _ray(rho, phi, tilt, tdir)
        P = P - 30.0 * w                           # start well before the instrument
        pix, xy = oracle.camera_trace(C0, P, w, OPT)
        ref = _march(P, w)
        if ref is None:
            assert pix == -1
            continue
        hits += 1
        assert pix >= 0
        assert np.allclose(xy, ref, atol=1e-9)
        n = OPT["cam_n"]
        ix, iy = (int(math.floor((v + OPT["camera_r"]) / (2 * OPT["camera_r"]) * n)) for v in ref)
        assert pix == min(max(iy, 0), n - 1) * n + min(max(ix, 0), n - 1)
    assert hits > 150


# ---- absorption in the optics (Sec. 6.4): mirror reflectivity x camera efficiency ----
EFF = dict(lambda_nm=[300.0, 350.0, 420.0, 500.0, 600.0],
           mirror=[0.80, 0.86, 0.90, 0.89, 0.87],
           camera=[0.18, 0.26, 0.24, 0.15, 0.05])


def _curve(x, y, v):
    return np.interp(v, x, y)   # linear between the nodes, constant beyond the ends


def test_optics_survival_is_the_keyed_draw_against_reflectivity_times_efficiency():
    """Brute force per photon: the camera keeps a photon iff the Philox word x
    of counter (segment, sub-step, bunch | 2^30), as a 24-bit uniform, lies
    below R(lambda) eps(lambda); the surviving photons are exactly those of
    the run without absorption that pass this test."""
    segs = synth.shower_segments(1500, 20.0, 30.0, 1e12, seed=4)
    tel = synth.grid_telescopes(nx=4, ny=4, pitch=60.0)
    atm = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
    kw = dict(tel=tel, bunch=1, refraction=True, transmission=True, seed=1)
    free = oracle.propagate(segs, atm, optics=OPT, **kw)["records"]
    lossy = oracle.propagate(segs, atm, optics=dict(OPT, efficiency=EFF), **kw)["records"]
    assert np.array_equal(free["seg"], lossy["seg"]) and np.array_equal(free["tel"], lossy["tel"])
    hit = free["pix"] >= 0
    assert hit.sum() > 100
    seen = 0
    for j in np.nonzero(hit)[0]:
        r = free[j]
        word = oracle.philox([int(r["seg"]) & 0xFFFFFFFF, int(r["seg"]) >> 32, int(r["k"]), int(r["i"]) | 0x40000000],
                             (1, 0))[0]
        u = (word >> 8) * 2.0 ** -24
        lnm = r["lam"] * 1e9
        P = _curve(EFF["lambda_nm"], EFF["mirror"], lnm) * _curve(EFF["lambda_nm"], EFF["camera"], lnm)
        assert lossy["pix"][j] == (r["pix"] if u < P else -1)
        seen += 1
    assert seen == hit.sum()
    assert (lossy["pix"][~hit] == -1).all()


def test_optics_survival_fraction_matches_the_curves():
    """Over many camera photons the surviving fraction equals the mean of
    R(lambda) eps(lambda) over their wavelengths (binomial 5 sigma); with flat
    curves it is the product of the two constants."""
    segs = synth.shower_segments(4000, 20.0, 30.0, 1e12, seed=6)
    tel = synth.grid_telescopes(nx=4, ny=4, pitch=60.0)
    atm = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
    kw = dict(tel=tel, bunch=1, refraction=True, transmission=False, seed=2)
    free = oracle.propagate(segs, atm, optics=OPT, **kw)["records"]
    flat = dict(lambda_nm=[400.0], mirror=[0.9], camera=[0.25])
    for eff in (EFF, flat):
        lossy = oracle.propagate(segs, atm, optics=dict(OPT, efficiency=eff), **kw)["records"]
        hit = free["pix"] >= 0
        lnm = free["lam"][hit] * 1e9
        P = _curve(eff["lambda_nm"], eff["mirror"], lnm) * _curve(eff["lambda_nm"], eff["camera"], lnm)
        kept = int((lossy["pix"][hit] >= 0).sum())
        assert abs(kept - P.sum()) < 5 * math.sqrt((P * (1 - P)).sum()), (kept, P.sum())
        if eff is flat:
            assert np.allclose(P, 0.225)
