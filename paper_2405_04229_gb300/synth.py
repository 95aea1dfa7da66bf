"""Seeded synthetic inputs: atmosphere parameter sets, detector layouts and
charged track segments.

This module is shared by the CUDA path's tests and benchmark and by the FP64
oracle's tests.  It holds input descriptions and random input generation
only; none of the photon method's arithmetic (yield, emission, propagation,
absorption, detection) lives here.  Segments are returned as a dict of
column arrays so that each consumer packs them into its own record layout.

The shower shapes stand in for the CORSIKA productions the thesis uses
(200 x 500 GeV showers, Fig. 6.1; 1 TeV EM showers, Sec. 5.3.4), which are
not available: a Greisen longitudinal profile, a Gaussian lateral spread and
Gaussian direction scatter about the shower axis.
"""
from __future__ import annotations

import functools
import math

import numpy as np

C_LIGHT = 299_792_458.0

# US standard atmosphere after Linsley, in the 5-layer form used by CORSIKA:
# T(h) = a + b exp(-h/c) for the four lower layers, T(h) = a - b h / c in the
# top layer.  T in g/cm^2, c in cm, layer bottoms in m.  The thesis names the
# US standard atmosphere (Sec. 4.3.1) but prints no parameters.
# Synthetic stand-in for a nitrogen fluorescence line list (the measured yields with their
# pressure, temperature and humidity dependence are not available here): five lines of the
# near-UV bands with round yields in photons per MeV deposited, and a minimum-ionising
# energy loss of 2.2 MeV cm^2/g.
FLUORESCENCE = dict(lines_nm=[316.0, 337.0, 358.0, 380.0, 391.0],
                    yield_per_mev=[2.0, 5.0, 4.0, 1.5, 1.5], dedx=2.2)

US_STANDARD = dict(
    layer_h=[0.0, 4000.0, 10000.0, 40000.0, 100000.0],
    a=[-186.555305, -94.919, 0.61289, 0.0, 0.01128292],
    b=[1222.6562, 1144.9069, 1305.5948, 540.1778, 1.0],
    c=[994186.38, 878153.55, 636143.04, 772170.16, 1.0e9],
    h_top=112829.2,
    kappa=2.9e-4,
)

# A user's n(h) table (the tabulated atmosphere kind): nodes every 1.5-7 km to
# 40 km with a falling profile, one rising and one constant interval.
TABLE_PROFILE = dict(
    h=[0.0, 1500.0, 3000.0, 4500.0, 7000.0, 9000.0, 12000.0, 15000.0, 20000.0, 26000.0, 33000.0, 40000.0],
    delta=[2.9e-4, 2.5e-4, 2.15e-4, 2.2e-4, 1.6e-4, 1.6e-4, 1.0e-4, 6.4e-5, 3.1e-5, 1.2e-5, 4.0e-6, 1.5e-6],
)

# Linear test profile of the thesis's propagation cross-check (Sec. 6.3.1):
# n = 1.5 at the ground falling linearly to 1.0 at 100 km.
LINEAR_TEST = dict(lin_h0=0.0, lin_h1=100_000.0, lin_n0=1.5, lin_n1=1.0)

# Transmission constants (Rayleigh + exponential aerosol); the thesis uses
# MODTRAN curves, which are not available.
TRANSMISSION = dict(rayl_X0=2974.0, rayl_lambda0=400e-9,
                    aer_tau0=0.05, aer_lambda0=350e-9, aer_alpha=1.3, aer_H=1200.0)


def _column_depth(h):
    """Vertical column depth of US_STANDARD above height h [m] -> g/cm^2."""
    p = US_STANDARD
    h = np.asarray(h, dtype=np.float64)
    out = np.zeros_like(h)
    lh = p["layer_h"]
    for i in range(5):
        lo = lh[i]
        hi = lh[i + 1] if i + 1 < 5 else p["h_top"]
        m = (h >= lo) & (h < hi) if i > 0 else (h < hi)
        if i == 4:
            out[m] = p["a"][i] - p["b"][i] * h[m] * 100.0 / p["c"][i]
        else:
            out[m] = p["a"][i] + p["b"][i] * np.exp(-h[m] * 100.0 / p["c"][i])
    return out


def height_of_depth(X):
    """Inverse of the vertical column depth (input placement only)."""
    p = US_STANDARD
    X = np.asarray(X, dtype=np.float64)
    bounds = _column_depth(np.array(p["layer_h"][1:] + [p["h_top"] - 1e-6]))
    out = np.empty_like(X)
    for i in range(5):
        upper_T = _column_depth(np.array([p["layer_h"][i]]))[0] if i > 0 else np.inf
        lower_T = bounds[i]
        m = (X <= upper_T) & (X > lower_T) if i < 4 else (X <= upper_T)
        if i == 4:
            out[m] = (p["a"][i] - X[m]) * p["c"][i] / p["b"][i] / 100.0
        else:
            out[m] = -np.log((X[m] - p["a"][i]) / p["b"][i]) * p["c"][i] / 100.0
    return out


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _empty(n):
    return dict(
        x0=np.zeros(n), y0=np.zeros(n), z0=np.zeros(n), t0=np.zeros(n),
        ux=np.zeros(n, np.float32), uy=np.zeros(n, np.float32), uz=np.zeros(n, np.float32),
        length=np.zeros(n, np.float32), inv_gamma2=np.zeros(n, np.float32),
        charge=np.ones(n, np.float32), shower_id=np.zeros(n, np.uint32),
    )


def concat(parts):
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def take(segs, idx):
    return {k: v[idx] for k, v in segs.items()}


def tiny_vertical_segments(n=1000, seed=0):
    """Start at (0, 0, U(8, 12) km), directions normalize(tan tx, tan ty, -1)
    with tx, ty ~ N(0, 3 deg), lengths U(1, 5) m, gamma log-uniform in
    [50, 1e4], charge 1, t0 = 0."""
    rng = np.random.default_rng([seed, 0x5EED])
    s = _empty(n)
    s["z0"] = rng.uniform(8000.0, 12000.0, n)
    tx, ty = np.radians(3.0) * rng.standard_normal((2, n))
    d = _unit(np.stack([np.tan(tx), np.tan(ty), -np.ones(n)], axis=1))
    s["ux"], s["uy"], s["uz"] = (d[:, i].astype(np.float32) for i in range(3))
    s["length"] = rng.uniform(1.0, 5.0, n).astype(np.float32)
    gamma = np.exp(rng.uniform(math.log(50.0), math.log(1e4), n))
    s["inv_gamma2"] = (1.0 / gamma**2).astype(np.float32)
    return s


def _greisen_depths(rng, n, E0_eV, X_cut, Ec_eV=81e6, X0=36.7):
    """Slant depths drawn from the Greisen profile N(t) ~ exp[t (1 - 1.5 ln s)],
    s = 3t / (t + 2 ln(E0/Ec)), t = X / X0, truncated at X_cut."""
    beta0 = math.log(E0_eV / Ec_eV)
    t = np.linspace(1e-4, X_cut / X0, 20001)
    s = 3.0 * t / (t + 2.0 * beta0)
    dens = np.exp(t * (1.0 - 1.5 * np.log(s)))
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(t))])
    cdf /= cdf[-1]
    return np.interp(rng.uniform(0.0, 1.0, n), cdf, t) * X0


def shower_segments(n, zenith_deg, azimuth_deg, E0_eV, seed, shower_id=0, h_obs=2000.0,
                    sigma_lateral=20.0, sigma_dir_deg=3.0, core=(0.0, 0.0)):
    """Segments of one synthetic shower whose axis hits (core, h_obs)."""
    rng = np.random.default_rng([seed, 0x5EED, shower_id])
    th, ph = math.radians(zenith_deg), math.radians(azimuth_deg)
    back = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    axis = -back                                           # direction of motion
    X_cut = float(_column_depth(np.array([h_obs]))[0]) / math.cos(th)
    X = _greisen_depths(rng, n, E0_eV, X_cut)
    h = height_of_depth(np.minimum(X * math.cos(th), _column_depth(np.array([h_obs]))[0]))
    along = (h - h_obs) / math.cos(th)                     # distance above the core along the axis
    e1 = _unit(np.cross(axis, [0.0, 0.0, 1.0]) if abs(axis[2]) < 0.999 else np.array([1.0, 0.0, 0.0]))
    e2 = np.cross(axis, e1)
    lat = sigma_lateral * rng.standard_normal((n, 2))
    pos = (np.array([core[0], core[1], h_obs])[None, :] + along[:, None] * back[None, :]
           + lat[:, :1] * e1[None, :] + lat[:, 1:] * e2[None, :])
    ang = np.radians(sigma_dir_deg) * rng.standard_normal((n, 2))
    d = _unit(axis[None, :] + np.tan(ang[:, :1]) * e1[None, :] + np.tan(ang[:, 1:]) * e2[None, :])
    s = _empty(n)
    s["x0"], s["y0"], s["z0"] = pos[:, 0], pos[:, 1], pos[:, 2]
    s["t0"] = (US_STANDARD["h_top"] - h) / math.cos(th) / C_LIGHT
    s["ux"], s["uy"], s["uz"] = (d[:, i].astype(np.float32) for i in range(3))
    s["length"] = rng.uniform(1.0, 5.0, n).astype(np.float32)
    gamma = np.exp(rng.uniform(math.log(50.0), math.log(1e4), n))
    s["inv_gamma2"] = (1.0 / gamma**2).astype(np.float32)
    s["charge"] = rng.choice(np.array([-1.0, 1.0], np.float32), n)
    s["shower_id"][:] = shower_id
    return s


def refraction_showers(n_showers=10, per_shower=100_000, seed=0, zenith_deg=20.0, E0_eV=1e12):
    """1 TeV-class showers at a fixed zenith (the refraction-corrected workload)."""
    return concat([shower_segments(per_shower, zenith_deg, 0.0, E0_eV, seed, shower_id=i)
                   for i in range(n_showers)])


def uneven_showers(n_showers=64, seed=0, lo=4.0, hi=7.0, max_total=None):
    """Showers with log-uniform segment counts, zenith U(0, 40), azimuth U(0, 360)."""
    rng = np.random.default_rng([seed, 0x5EED, 0xC3])
    counts = np.floor(10.0 ** rng.uniform(lo, hi, n_showers)).astype(np.int64)
    if max_total is not None and counts.sum() > max_total:
        counts = np.maximum(1, (counts * (max_total / counts.sum())).astype(np.int64))
    zen = rng.uniform(0.0, 40.0, n_showers)
    azi = rng.uniform(0.0, 360.0, n_showers)
    parts = [shower_segments(int(c), zen[i], azi[i], 1e12, seed, shower_id=i)
             for i, c in enumerate(counts)]
    return concat(parts), counts


@functools.lru_cache(maxsize=2)
def _inclined_base(n, seed, zenith_deg, azimuth_deg, E0_eV):
    return shower_segments(n, zenith_deg, azimuth_deg, E0_eV, seed)


def inclined_chunk(c, n=10_000_000, seed=0, zenith_deg=60.0, azimuth_deg=0.0, E0_eV=1e14, n_chunks=10,
                   h_obs=2000.0):
    """Chunk c of the large inclined shower (100 TeV-class, zenith 60 deg): one
    seeded draw of n segments turned about the shower axis by 2 pi c / n_chunks.
    The lateral and angular spreads are symmetric about the axis, so every
    chunk is a sample of the same shower; its photons are keyed by the global
    segment ids c n .. (c + 1) n - 1."""
    b = _inclined_base(n, seed, zenith_deg, azimuth_deg, E0_eV)
    th, ph = math.radians(zenith_deg), math.radians(azimuth_deg)
    k = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    a = 2.0 * math.pi * c / n_chunks
    K = np.array([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]])
    Rm = np.eye(3) + math.sin(a) * K + (1.0 - math.cos(a)) * (K @ K)   # Rodrigues
    pos = np.stack([b["x0"], b["y0"], b["z0"] - h_obs], axis=1) @ Rm.T
    d = np.stack([b["ux"], b["uy"], b["uz"]], axis=1).astype(np.float64) @ Rm.T
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    s = dict(b)
    s["x0"], s["y0"], s["z0"] = pos[:, 0], pos[:, 1], pos[:, 2] + h_obs
    s["ux"], s["uy"], s["uz"] = (d[:, i].astype(np.float32) for i in range(3))
    return s


def steep_arrival_segments(n, seed, zenith_deg=80.0, half=560.0, h_obs=2000.0):
    """Segments 50-300 m above the ground moving at a fixed steep zenith (+x
    azimuth), placed so their photons land over [-half, half)^2: arrivals far
    beyond the telescope hash's zenith range, many near the array's edge."""
    rng = np.random.default_rng([seed, 0x5EED, 0x57])
    s = _empty(n)
    th = math.radians(zenith_deg)
    dz = rng.uniform(50.0, 300.0, n)
    s["z0"] = h_obs + dz
    s["x0"] = -dz * math.tan(th) + rng.uniform(-half, half, n)
    s["y0"] = rng.uniform(-half, half, n)
    s["ux"][:], s["uz"][:] = np.float32(math.sin(th)), np.float32(-math.cos(th))
    s["length"][:] = 2.0
    s["inv_gamma2"][:] = np.float32(1e-8)
    return s


def grid_telescopes(nx=10, ny=10, pitch=100.0, radius=6.0, h_obs=2000.0):
    """Telescope spheres on a square grid centred on the origin: n x 4 (x, y, z, r)."""
    xs = (np.arange(nx) - (nx - 1) / 2.0) * pitch
    ys = (np.arange(ny) - (ny - 1) / 2.0) * pitch
    gx, gy = np.meshgrid(xs, ys, indexing="xy")
    n = nx * ny
    return np.stack([gx.ravel(), gy.ravel(), np.full(n, h_obs), np.full(n, radius)], axis=1)


def poisson_disk_telescopes(n=2000, half=1000.0, min_sep=13.0, radius=6.0, h_obs=2000.0, seed=0):
    """Seeded irregular layout by dart throwing with a minimum separation."""
    rng = np.random.default_rng([seed, 0x5EED, 0xC5])
    pts = []
    cell = min_sep / math.sqrt(2.0)
    ncell = int(math.ceil(2 * half / cell))
    grid = -np.ones((ncell, ncell), np.int64)
    tries = 0
    while len(pts) < n and tries < 200 * n:
        tries += 1
        p = rng.uniform(-half, half, 2)
        ci, cj = int((p[0] + half) / cell), int((p[1] + half) / cell)
        ok = True
        for di in range(-2, 3):
            for dj in range(-2, 3):
                a, b = ci + di, cj + dj
                if 0 <= a < ncell and 0 <= b < ncell and grid[a, b] >= 0:
                    if np.hypot(*(pts[grid[a, b]] - p)) < min_sep:
                        ok = False
        if ok:
            grid[ci, cj] = len(pts)
            pts.append(p)
    pts = np.array(pts)
    m = len(pts)
    return np.stack([pts[:, 0], pts[:, 1], np.full(m, h_obs), np.full(m, radius)], axis=1)


def histogram_400():
    """400 x 400 cells of 1 m over [-200, 200)^2 m."""
    return dict(nx=400, ny=400, x0=-200.0, y0=-200.0, dx=1.0, dy=1.0)
