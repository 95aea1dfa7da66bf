"""FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package.  The C source (``cherenkov_oracle.c``) is
an independent, plain FP64 implementation of the method; this module only
builds it with gcc and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cherenkov_oracle.c")
_LIB_DIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

ST_LANDED, ST_UPWARD, ST_BELOW, ST_NO_GROUND, ST_ABSORBED, ST_LV3 = range(6)
ST_SUBSTEP_FLAG = 15
FL_COUNT, FL_ABSORB, FL_HIST_EDGE, FL_TEL_EDGE, FL_GROUND, FL_BELOW, FL_UPWARD, FL_LAYER, FL_LV1, FL_LV3 = (
    1, 2, 4, 8, 16, 32, 64, 128, 256, 512)
FL_SEGMENT = 1024   # the segment's sub-step count is a rounding decision: all its bunches are undetermined
FL_OPTICS = 2048    # the optics survival draw lies within the band of its threshold
LV1_OFF, LV1_ARRAY_CENTRE, LV1_ARRAY_DISC, LV1_TELESCOPES = 0, 1, 2, 3
ATM_LAYERED, ATM_LINEAR, ATM_HOMOGENEOUS, ATM_TABLE = 0, 1, 2, 3
RHO_REF = 1.225e-3   # [g/cm^3]: the table kind's density is RHO_REF (n - 1) / kappa


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no fast-math)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Atm(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_layers", C.c_int), ("last_linear", C.c_int), ("pad", C.c_int),
                ("layer_h", C.c_double * 8), ("a", C.c_double * 8), ("b", C.c_double * 8),
                ("c", C.c_double * 8), ("h_top", C.c_double), ("kappa", C.c_double),
                ("lin_h0", C.c_double), ("lin_h1", C.c_double), ("lin_n0", C.c_double),
                ("lin_n1", C.c_double), ("hom_delta", C.c_double),
                ("n_nodes", C.c_int), ("pad2", C.c_int), ("node_h", C.c_double * 128),
                ("node_d", C.c_double * 128), ("rho_ref", C.c_double)]


class Config(C.Structure):
    _fields_ = [("h_obs", C.c_double), ("lambda1", C.c_double), ("lambda2", C.c_double),
                ("s_max", C.c_double), ("bunch", C.c_int), ("refraction", C.c_int),
                ("transmission", C.c_int), ("pad0", C.c_int),
                ("rayl_X0", C.c_double), ("rayl_lambda0", C.c_double),
                ("aer_tau0", C.c_double), ("aer_lambda0", C.c_double), ("aer_alpha", C.c_double),
                ("aer_H", C.c_double), ("seed", C.c_uint64), ("seg_base", C.c_uint64),
                ("n_showers", C.c_int), ("hist_nx", C.c_int), ("hist_ny", C.c_int), ("n_tel", C.c_int),
                ("hist_x0", C.c_double), ("hist_y0", C.c_double), ("hist_dx", C.c_double),
                ("hist_dy", C.c_double), ("tel", C.POINTER(C.c_double)),
                ("band_pos", C.c_double), ("band_count", C.c_double), ("band_T", C.c_double),
                ("band_h", C.c_double), ("band_w", C.c_double), ("quad_rtol", C.c_double),
                ("spherical", C.c_int), ("cylindrical", C.c_int), ("earth_radius", C.c_double),
                ("lv1_metric", C.c_int), ("pad3", C.c_int), ("lv1_a", C.c_double), ("lv1_b", C.c_double),
                ("lv1_centre", C.c_double * 3), ("lv1_radius", C.c_double), ("band_lv1", C.c_double),
                ("mirror_d", C.c_double), ("focal_f", C.c_double), ("camera_r", C.c_double),
                ("point_zenith", C.c_double), ("point_azimuth", C.c_double), ("cam_n", C.c_int), ("pad4", C.c_int),
                ("lv3", C.c_int), ("pad5", C.c_int), ("lv3_centre", C.c_double * 3), ("lv3_radius", C.c_double),
                ("lv3_margin", C.c_double), ("tracer", C.c_int), ("pad6", C.c_int), ("tracer_dh", C.c_double),
                ("emission", C.c_int), ("fl_n_lines", C.c_int), ("fl_lines_nm", C.c_double * 8),
                ("fl_yield", C.c_double * 8), ("fl_dedx", C.c_double),
                ("eff_n", C.c_int), ("pad7", C.c_int), ("eff_l", C.c_double * 16), ("eff_R", C.c_double * 16),
                ("eff_E", C.c_double * 16)]


SEGMENT_DTYPE = np.dtype([("x0", "<f8"), ("y0", "<f8"), ("z0", "<f8"), ("t0", "<f8"),
                          ("ux", "<f4"), ("uy", "<f4"), ("uz", "<f4"), ("length", "<f4"),
                          ("inv_gamma2", "<f4"), ("charge", "<f4"), ("shower_id", "<u4"),
                          ("flags", "<u4")])

RECORD_DTYPE = np.dtype([("seg", "<u8"), ("k", "<u4"), ("i", "<u4"), ("x", "<f8"), ("y", "<f8"),
                         ("dt", "<f8"), ("lam", "<f8"), ("ex", "<f8"), ("ey", "<f8"), ("h_e", "<f8"),
                         ("ux", "<f8"), ("uy", "<f8"), ("uz", "<f8"), ("theta0", "<f8"),
                         ("T", "<f8"), ("nbar", "<f8"), ("status", "<i4"), ("tel", "<i4"),
                         ("bin", "<i4"), ("flags", "<u4"), ("pix", "<i4"), ("pad", "<i4")])


class Output(C.Structure):
    _fields_ = [("hist", C.POINTER(C.c_uint64)), ("tel_counts", C.POINTER(C.c_uint64)),
                ("tel_time", C.POINTER(C.c_double)), ("counters", C.c_uint64 * 8),
                ("records", C.c_void_p), ("capacity", C.c_size_t), ("count", C.c_size_t),
                ("lv1_dropped", C.c_uint64), ("camera", C.POINTER(C.c_uint64))]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            d, u32p, dp = C.c_double, C.POINTER(C.c_uint32), C.POINTER(C.c_double)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            for f in ("orc_atm_T", "orc_atm_rho", "orc_atm_delta"):
                getattr(L, f).argtypes = [C.POINTER(Atm), d]
                getattr(L, f).restype = d
            L.orc_column.argtypes = [C.POINTER(Atm), d, d]
            L.orc_column.restype = d
            L.orc_gauss_legendre.argtypes = [C.c_int, dp, dp]
            L.orc_refract_quad.argtypes = [C.POINTER(Atm), d, d, d, d, d, dp]
            L.orc_straight.argtypes = [C.POINTER(Atm), d, d, d, d, dp]
            L.orc_refract_closed.argtypes = [C.POINTER(Atm), d, d, d, dp]
            L.orc_refract_closed.restype = C.c_int
            L.orc_snell_stepper.argtypes = [C.POINTER(Atm), d, d, d, d, dp]
            L.orc_snell_path.argtypes = [C.POINTER(Atm), d, d, d, d, d, dp]
            L.orc_snell_path_sph.argtypes = [C.POINTER(Atm), d, d, d, d, d, d, dp]
            L.orc_sph_path.argtypes = [C.POINTER(Atm), d, d, d, d, d, C.c_int, d, dp]
            L.orc_ae_inverse.argtypes = [d, d, d, d, d, dp]
            L.orc_cyl_path.argtypes = [C.POINTER(Atm), d, d, d, d, d, d, C.c_int, d, dp]
            L.orc_snell_path_cyl.argtypes = [C.POINTER(Atm), d, d, d, d, d, d, d, d, C.c_int, dp]
            L.orc_cyl_reach_margin.argtypes = [C.POINTER(Atm), C.c_int, d, d, d, d, d]
            L.orc_cyl_reach_margin.restype = d
            L.orc_propagate.argtypes = [C.c_void_p, C.c_size_t, C.POINTER(Atm), C.POINTER(Config),
                                        C.POINTER(Output)]
            L.orc_propagate.restype = C.c_int
            L.orc_mlp_n_params.argtypes = [C.c_int, C.c_int, C.c_int]
            L.orc_mlp_n_params.restype = C.c_size_t
            L.orc_mlp_forward.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, C.c_int, dp, dp]
            L.orc_mlp_loss_grad.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, dp, C.c_int, dp]
            L.orc_mlp_loss_grad.restype = d
            L.orc_adam.argtypes = [dp, dp, dp, dp, C.c_size_t, d, d, d, d, C.c_int]
            for f in ("orc_sizeof_segment", "orc_sizeof_record", "orc_sizeof_config", "orc_sizeof_atm"):
                getattr(L, f).restype = C.c_size_t
            assert L.orc_sizeof_segment() == SEGMENT_DTYPE.itemsize
            assert L.orc_sizeof_record() == RECORD_DTYPE.itemsize
            assert L.orc_sizeof_config() == C.sizeof(Config)
            assert L.orc_sizeof_atm() == C.sizeof(Atm)
            _lib = L
    return _lib


# ---------------------------------------------------------------------------
# argument helpers
# ---------------------------------------------------------------------------
def make_atm(kind=ATM_LAYERED, layered=None, linear=None, hom_delta=0.0, table=None, kappa=2.9e-4):
    """table: dict(h=[...], delta=[...]) of n - 1 at ascending node heights (table kind)."""
    a = Atm()
    a.kind = kind
    if kind == ATM_TABLE:
        h, d = list(table["h"]), list(table["delta"])
        assert 2 <= len(h) <= 128 and len(h) == len(d)
        a.n_nodes = len(h)
        for i in range(len(h)):
            a.node_h[i], a.node_d[i] = h[i], d[i]
        a.kappa, a.rho_ref, a.h_top = kappa, RHO_REF, h[-1]
        return a
    if kind == ATM_LAYERED:
        p = layered
        n = len(p["layer_h"])
        a.n_layers, a.last_linear = n, 1
        for i in range(n):
            a.layer_h[i], a.a[i], a.b[i], a.c[i] = p["layer_h"][i], p["a"][i], p["b"][i], p["c"][i]
        a.h_top, a.kappa = p["h_top"], p["kappa"]
    elif kind == ATM_LINEAR:
        a.lin_h0, a.lin_h1, a.lin_n0, a.lin_n1 = (linear[k] for k in ("lin_h0", "lin_h1", "lin_n0", "lin_n1"))
        a.h_top = linear["lin_h1"]
    else:
        a.hom_delta = hom_delta
        a.h_top = 1e9
    return a


def philox(ctr, key):
    L = lib()
    ci = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    ki = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    out = (C.c_uint32 * 4)()
    L.orc_philox4x32_10(ci, ki, out)
    return [int(x) for x in out]


def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    lib().orc_gauss_legendre(n, x.ctypes.data_as(C.POINTER(C.c_double)),
                             w.ctypes.data_as(C.POINTER(C.c_double)))
    return x, w


def atm_T(atm, h):
    return lib().orc_atm_T(C.byref(atm), float(h))


def column(atm, lo, hi):
    return lib().orc_column(C.byref(atm), float(lo), float(hi))


def atm_rho(atm, h):
    return lib().orc_atm_rho(C.byref(atm), float(h))


def atm_delta(atm, h):
    return lib().orc_atm_delta(C.byref(atm), float(h))


def refract_quad(atm, h_obs, h_e, theta0, H_A=1200.0, rtol=1e-12):
    out = (C.c_double * 4)()
    lib().orc_refract_quad(C.byref(atm), h_obs, h_e, theta0, H_A, rtol, out)
    return np.array(out[:])


def straight(atm, h_obs, h_e, theta0, H_A=1200.0):
    out = (C.c_double * 4)()
    lib().orc_straight(C.byref(atm), h_obs, h_e, theta0, H_A, out)
    return np.array(out[:])


def refract_closed(atm, h_obs, h_e, theta0):
    out = (C.c_double * 3)()
    rc = lib().orc_refract_closed(C.byref(atm), h_obs, h_e, theta0, out)
    if rc != 0:
        raise ValueError("no closed form for these arguments")
    return np.array(out[:])


def snell_path(atm, h_obs, h_e, theta0, dh, H_A=1200.0):
    """{R, t_path, X_slant, A_slant} of the Snell vector stepper."""
    out = (C.c_double * 4)()
    lib().orc_snell_path(C.byref(atm), h_obs, h_e, theta0, dh, H_A, out)
    return np.array(out[:])


def snell_path_sph(atm, h_obs, h_e, psi0, dh, R=None, H_A=1200.0):
    """{central angle, t_path, X_slant, A_slant} of the stepper on the spherical shell."""
    out = (C.c_double * 4)()
    lib().orc_snell_path_sph(C.byref(atm), EARTH_RADIUS if R is None else R, h_obs, h_e, psi0, dh, H_A, out)
    return np.array(out[:])


def snell_stepper(atm, h_obs, h_e, theta0, dh):
    out = (C.c_double * 2)()
    lib().orc_snell_stepper(C.byref(atm), h_obs, h_e, theta0, dh, out)
    return np.array(out[:])


EARTH_RADIUS = 6_370_000.0


def sph_path(atm, h_obs, h_e, psi0, refraction=True, R=EARTH_RADIUS, H_A=1200.0, rtol=1e-12):
    """{central angle, t_path, X_slant, A_slant} in the spherical-shell atmosphere."""
    out = (C.c_double * 4)()
    lib().orc_sph_path(C.byref(atm), R, h_obs, h_e, psi0, H_A, int(refraction), rtol, out)
    return np.array(out[:])


def cyl_path(atm, h_obs, h_e, u_a, u_chi, refraction=True, R=EARTH_RADIUS, H_A=1200.0, rtol=1e-12):
    """{chi swept, t_path, axial drift, X_slant, A_slant} in the cylindrical atmosphere
    for a photon at altitude h_e with direction components u_a (axial) and u_chi >= 0
    (transverse tangent)."""
    out = (C.c_double * 5)()
    lib().orc_cyl_path(C.byref(atm), R, h_obs, h_e, u_a, u_chi, H_A, int(refraction), rtol, out)
    return np.array(out[:])


def snell_path_cyl(atm, h_obs, h_e, u_chi, u_rho, u_a, dh, refraction=True, R=EARTH_RADIUS, H_A=1200.0):
    """The three-dimensional Snell stepper through the cylindrical atmosphere."""
    out = (C.c_double * 5)()
    lib().orc_snell_path_cyl(C.byref(atm), R, h_obs, h_e, u_chi, u_rho, u_a, dh, H_A, int(refraction), out)
    return np.array(out[:])


def cyl_reach_margin(atm, h_obs, h_e, u_a, u_chi, refraction=True, R=EARTH_RADIUS):
    return lib().orc_cyl_reach_margin(C.byref(atm), int(refraction), R, h_obs, h_e, u_a, u_chi)


def ae_inverse(x, y, dz=0.0, h_obs=2000.0, R=EARTH_RADIUS):
    out = (C.c_double * 3)()
    lib().orc_ae_inverse(R, h_obs, x, y, dz, out)
    return np.array(out[:])


def camera_trace(centre, ground, u, optics):
    """(pixel or -1, camera-plane point) of the ray ground + t u through the
    telescope whose sphere is centred at `centre`."""
    cfg = Config()
    for k in ("mirror_d", "focal_f", "camera_r", "point_zenith", "point_azimuth", "cam_n"):
        setattr(cfg, k, optics[k])
    xy = (C.c_double * 2)()
    d3 = C.c_double * 3
    pix = lib().orc_camera_trace(C.byref(cfg), d3(*centre), d3(*ground), d3(*u), xy)
    return int(pix), np.array(xy[:])


def pack_segments(cols) -> np.ndarray:
    n = len(cols["z0"])
    a = np.zeros(n, SEGMENT_DTYPE)
    for k in SEGMENT_DTYPE.names:
        if k in cols:
            a[k] = cols[k]
    return a


DEFAULT_BANDS = dict(band_pos=1e-4, band_count=1e-4, band_T=1e-5, band_h=1e-3, band_w=1e-6)


def propagate(segs, atm, *, h_obs=2000.0, lambda_nm=(300.0, 600.0), s_max=1.0, bunch=1,
              refraction=False, transmission=False, seed=0,
              seg_base=0, n_showers=1, hist=None, tel=None, records=True, record_capacity=None,
              transmission_params=None, bands=None, quad_rtol=1e-10, spherical=False, earth_radius=EARTH_RADIUS,
              lv1=None, optics=None, lv3=None, snell_dh=None, fluorescence=None, cylindrical=False):
    """Run the oracle over ``segs`` (dict of columns or SEGMENT_DTYPE array).

    Returns a dict with hist [n_showers, ny, nx], tel_counts [n_showers, n_tel],
    tel_time, counters (8) and, if requested, the per-photon records.
    """
    L = lib()
    arr = segs if isinstance(segs, np.ndarray) else pack_segments(segs)
    arr = np.ascontiguousarray(arr)
    cfg = Config()
    cfg.h_obs = h_obs
    cfg.lambda1, cfg.lambda2 = lambda_nm[0] * 1e-9, lambda_nm[1] * 1e-9
    cfg.s_max, cfg.bunch = s_max, bunch
    cfg.refraction, cfg.transmission = int(refraction), int(transmission)
    tp = dict(rayl_X0=2974.0, rayl_lambda0=400e-9, aer_tau0=0.05, aer_lambda0=350e-9,
              aer_alpha=1.3, aer_H=1200.0)
    if transmission_params:
        tp.update(transmission_params)
    for k, v in tp.items():
        setattr(cfg, k, v)
    cfg.seed, cfg.seg_base = seed, seg_base
    cfg.n_showers = n_showers
    h = hist or dict(nx=0, ny=0, x0=0.0, y0=0.0, dx=1.0, dy=1.0)
    cfg.hist_nx, cfg.hist_ny = h["nx"], h["ny"]
    cfg.hist_x0, cfg.hist_y0, cfg.hist_dx, cfg.hist_dy = h["x0"], h["y0"], h["dx"], h["dy"]
    tel_arr = np.ascontiguousarray(np.zeros((0, 4)) if tel is None else np.asarray(tel, np.float64))
    cfg.n_tel = tel_arr.shape[0]
    cfg.tel = tel_arr.ctypes.data_as(C.POINTER(C.c_double))
    b = dict(DEFAULT_BANDS)
    if bands:
        b.update(bands)
    for k, v in b.items():
        setattr(cfg, k, v)
    cfg.quad_rtol = quad_rtol
    cfg.spherical, cfg.earth_radius = int(spherical or cylindrical), earth_radius
    cfg.cylindrical = int(cylindrical)
    if lv1:   # dict(metric, a, b, centre=(x, y, z), radius, band)
        cfg.lv1_metric, cfg.lv1_a, cfg.lv1_b = lv1["metric"], lv1["a"], lv1["b"]
        for i, v in enumerate(lv1.get("centre", (0.0, 0.0, h_obs))):
            cfg.lv1_centre[i] = v
        cfg.lv1_radius, cfg.band_lv1 = lv1.get("radius", 0.0), lv1.get("band", 1e-4)
    if fluorescence:   # dict(half=bool, lines_nm, yield_per_mev, dedx): isotropic line emission
        cfg.emission = 2 if fluorescence.get("half") else 1
        lines, ys = fluorescence["lines_nm"], fluorescence["yield_per_mev"]
        cfg.fl_n_lines = len(lines)
        for j, (l, y) in enumerate(zip(lines, ys)):
            cfg.fl_lines_nm[j], cfg.fl_yield[j] = l, y
        cfg.fl_dedx = fluorescence["dedx"]
    if snell_dh:   # refraction by the Snell vector stepper through slabs <= snell_dh [m]
        cfg.tracer, cfg.tracer_dh = 1, snell_dh
    if lv3:   # dict(centre=(x, y, z), radius, margin)
        cfg.lv3 = 1
        for i, v in enumerate(lv3.get("centre", (0.0, 0.0, h_obs))):
            cfg.lv3_centre[i] = v
        cfg.lv3_radius, cfg.lv3_margin = lv3["radius"], lv3.get("margin", 0.0)
    if optics:   # dict(mirror_d, focal_f, camera_r, point_zenith, point_azimuth [rad], cam_n
        #            [, efficiency=dict(lambda_nm, mirror, camera)])
        for k in ("mirror_d", "focal_f", "camera_r", "point_zenith", "point_azimuth", "cam_n"):
            setattr(cfg, k, optics[k])
        eff = optics.get("efficiency")
        if eff:
            n_eff = len(eff["lambda_nm"])
            assert 1 <= n_eff <= 16
            cfg.eff_n = n_eff
            for j in range(n_eff):
                cfg.eff_l[j], cfg.eff_R[j], cfg.eff_E[j] = eff["lambda_nm"][j], eff["mirror"][j], eff["camera"][j]

    hist_out = np.zeros((n_showers, max(h["ny"], 0), max(h["nx"], 0)), np.uint64)
    tel_counts = np.zeros((n_showers, cfg.n_tel), np.uint64)
    tel_time = np.zeros((n_showers, cfg.n_tel), np.float64)
    out = Output()
    cam = None
    if optics:
        cam = np.zeros((n_showers, cfg.n_tel, optics["cam_n"], optics["cam_n"]), np.uint64)
        out.camera = cam.ctypes.data_as(C.POINTER(C.c_uint64))
    out.hist = hist_out.ctypes.data_as(C.POINTER(C.c_uint64))
    out.tel_counts = tel_counts.ctypes.data_as(C.POINTER(C.c_uint64))
    out.tel_time = tel_time.ctypes.data_as(C.POINTER(C.c_double))
    rec = None
    if records:
        cap = record_capacity if record_capacity is not None else max(1024, 400 * len(arr))
        rec = np.zeros(cap, RECORD_DTYPE)
        out.records, out.capacity = rec.ctypes.data, cap
    rc = L.orc_propagate(arr.ctypes.data, len(arr), C.byref(atm), C.byref(cfg), C.byref(out))
    if rc != 0:
        raise RuntimeError("oracle failed: %d" % rc)
    res = dict(hist=hist_out, tel_counts=tel_counts, tel_time=tel_time,
               counters=np.array(out.counters[:], np.uint64), n_records=int(out.count),
               lv1_dropped=int(out.lv1_dropped), camera=cam)
    if records:
        if out.count > cap:
            raise RuntimeError("record capacity %d too small (%d)" % (cap, out.count))
        res["records"] = rec[: out.count].copy()
    return res


# ---------------------------------------------------------------------------
# surrogate network (FP64)
# ---------------------------------------------------------------------------
def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def mlp_n_params(din=3, dh=64, dout=3):
    return int(lib().orc_mlp_n_params(din, dh, dout))


def mlp_forward(theta, x, din=3, dh=64, dout=3, return_acts=False):
    theta = np.ascontiguousarray(theta, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    B = x.shape[0]
    y = np.zeros((B, dout))
    acts = np.zeros((B, 3, dh)) if return_acts else None
    lib().orc_mlp_forward(_p(theta), din, dh, dout, _p(x), B, _p(y), _p(acts) if return_acts else None)
    return (y, acts) if return_acts else y


def mlp_loss_grad(theta, x, t, din=3, dh=64, dout=3):
    theta = np.ascontiguousarray(theta, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    t = np.ascontiguousarray(t, np.float64)
    g = np.zeros_like(theta)
    loss = lib().orc_mlp_loss_grad(_p(theta), din, dh, dout, _p(x), _p(t), x.shape[0], _p(g))
    return loss, g


def adam(theta, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    grad = np.ascontiguousarray(grad, np.float64)
    lib().orc_adam(_p(theta), _p(grad), _p(m), _p(v), theta.size, lr, beta1, beta2, eps, step)
