"""Thin ctypes binding of the C ABI in ``include/cherenkov.h``.

Argument marshalling only: every step of the photon path runs in the CUDA
library.  The library is loaded from the package's ``lib/`` directory and is
never replaced by a CPU fallback: if it is missing or cannot load, the first
call raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libcherenkov.so")
_lock = threading.Lock()
_lib = None

CS_OK, CS_ERR_INVALID_ARG, CS_ERR_CUDA, CS_ERR_CAPACITY, CS_ERR_TIMEOUT, CS_ERR_DOMAIN, CS_ERR_NO_DEVICE = range(7)
CS_ATM_LAYERED, CS_ATM_LINEAR, CS_ATM_HOMOGENEOUS, CS_ATM_TABLE = 0, 1, 2, 3
CS_GEOM_PLANAR, CS_GEOM_SPHERICAL, CS_GEOM_CYLINDRICAL = 0, 1, 2
CS_LV1_OFF, CS_LV1_ARRAY_CENTRE, CS_LV1_ARRAY_DISC, CS_LV1_TELESCOPES = 0, 1, 2, 3


def set_lv1(o, lv1):
    """Fill the LV1 filter fields of a cs_opts from dict(metric, a, b, centre, radius)."""
    if not lv1:
        return
    o.lv1_metric, o.lv1_a, o.lv1_b = lv1["metric"], lv1["a"], lv1["b"]
    for i, v in enumerate(lv1.get("centre", (0.0, 0.0, 0.0))):
        o.lv1_centre[i] = v
    o.lv1_radius = lv1.get("radius", 0.0)


def set_lv3(o, lv3):
    """Fill the LV3 photon pre-filter fields of a cs_opts from dict(centre, radius, margin)."""
    if not lv3:
        return
    o.lv3 = 1
    for i, v in enumerate(lv3["centre"]):
        o.lv3_centre[i] = v
    o.lv3_radius, o.lv3_margin = lv3["radius"], lv3.get("margin", 0.0)
(CS_CNT_EMITTED, CS_CNT_ABSORBED, CS_CNT_HIST, CS_CNT_TEL, CS_CNT_MISSED_HIST, CS_CNT_MISSED_TEL,
 CS_CNT_UPWARD, CS_CNT_INVALID_SEGMENTS) = range(8)
CS_N_COUNTERS = 8
CS_ST_LANDED, CS_ST_UPWARD, CS_ST_BELOW, CS_ST_NO_GROUND, CS_ST_ABSORBED, CS_ST_LV3 = range(6)


class CSError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = "%s failed: %s" % (where, status_string(status))
        if status == CS_ERR_CUDA:
            msg += " (%s)" % last_error()
        super().__init__(msg)


SEGMENT_DTYPE = np.dtype([("x0", "<f8"), ("y0", "<f8"), ("z0", "<f8"), ("t0", "<f8"),
                          ("ux", "<f4"), ("uy", "<f4"), ("uz", "<f4"), ("length", "<f4"),
                          ("inv_gamma2", "<f4"), ("charge", "<f4"), ("shower_id", "<u4"),
                          ("flags", "<u4")])
RECORD_DTYPE = np.dtype([("seg", "<u8"), ("k", "<u4"), ("i", "<u4"), ("x", "<f4"), ("y", "<f4"),
                         ("dt_ns", "<f4"), ("lambda_nm", "<f4"), ("tel", "<i4"), ("bin", "<i4"),
                         ("status", "<u4"), ("pix", "<i4"), ("x_lo", "<f4"), ("y_lo", "<f4")])


class cs_atmosphere_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_layers", C.c_int),
                ("layer_h", C.POINTER(C.c_double)), ("layer_a", C.POINTER(C.c_double)),
                ("layer_b", C.POINTER(C.c_double)), ("layer_c", C.POINTER(C.c_double)),
                ("h_top", C.c_double), ("kappa", C.c_double),
                ("lin_h0", C.c_double), ("lin_h1", C.c_double), ("lin_n0", C.c_double), ("lin_n1", C.c_double),
                ("hom_delta", C.c_double), ("h_obs", C.c_double),
                ("lambda_min", C.c_double), ("lambda_max", C.c_double),
                ("refraction", C.c_int), ("transmission", C.c_int),
                ("rayl_X0", C.c_double), ("rayl_lambda0", C.c_double),
                ("aer_tau0", C.c_double), ("aer_lambda0", C.c_double), ("aer_alpha", C.c_double),
                ("aer_H", C.c_double), ("theta_max", C.c_double), ("table_nw", C.c_int),
                ("table_dh", C.c_double), ("geometry", C.c_int), ("earth_radius", C.c_double),
                ("table_n", C.c_int), ("table_h", C.POINTER(C.c_double)), ("table_delta", C.POINTER(C.c_double))]


class cs_detector_desc(C.Structure):
    _fields_ = [("n_showers", C.c_int), ("h_obs", C.c_double), ("hist_nx", C.c_int), ("hist_ny", C.c_int),
                ("hist_x0", C.c_double), ("hist_y0", C.c_double), ("hist_dx", C.c_double),
                ("hist_dy", C.c_double), ("n_tel", C.c_int), ("tel_xyzr", C.POINTER(C.c_double)),
                ("geometry", C.c_int), ("earth_radius", C.c_double),
                ("mirror_d", C.c_double), ("focal_f", C.c_double), ("camera_r", C.c_double),
                ("point_zenith", C.c_double), ("point_azimuth", C.c_double), ("cam_n", C.c_int),
                ("eff_n", C.c_int), ("eff_lambda_nm", C.POINTER(C.c_double)), ("eff_mirror", C.POINTER(C.c_double)),
                ("eff_camera", C.POINTER(C.c_double))]


OPTICS_KEYS = ("mirror_d", "focal_f", "camera_r", "point_zenith", "point_azimuth", "cam_n")


class cs_output(C.Structure):
    _fields_ = [("hist", C.c_void_p), ("tel_counts", C.c_void_p), ("tel_time", C.c_void_p),
                ("counters", C.c_void_p), ("records", C.c_void_p), ("record_capacity", C.c_uint64),
                ("record_count", C.c_void_p), ("camera", C.c_void_p)]


class cs_tune_result(C.Structure):
    _fields_ = [("blocks_per_sm", C.c_int), ("n_tried", C.c_int), ("ms", C.c_float * 8)]


class cs_surrogate_config(C.Structure):
    _fields_ = [("n_train", C.c_int), ("n_heldout", C.c_int), ("batch", C.c_int), ("epochs", C.c_int),
                ("seed", C.c_uint64), ("lr", C.c_double), ("lr_min", C.c_double), ("h_min", C.c_double),
                ("h_max", C.c_double), ("theta_max", C.c_double), ("split_activations", C.c_int),
                ("boundary_band", C.c_double), ("height_scale", C.c_double)]


class cs_surrogate_stats(C.Structure):
    _fields_ = [("heldout_p99", C.c_double * 3), ("heldout_max", C.c_double * 3), ("final_loss", C.c_double),
                ("steps", C.c_int), ("train_seconds", C.c_double)]


N_MLP_PARAMS = 64 * 3 + 64 + 2 * (64 * 64 + 64) + 8 * 64 + 8


class cs_opts(C.Structure):
    _fields_ = [("bunch", C.c_int), ("s_max", C.c_double), ("seg_base", C.c_uint64),
                ("device_ptrs", C.c_int), ("accumulate", C.c_int), ("block_threads", C.c_int),
                ("blocks_per_sm", C.c_int), ("surrogate", C.c_void_p),
                ("lv1_metric", C.c_int), ("lv1_a", C.c_double), ("lv1_b", C.c_double),
                ("lv1_centre", C.c_double * 3), ("lv1_radius", C.c_double), ("lv1_dropped", C.c_void_p),
                ("lv3", C.c_int), ("lv3_centre", C.c_double * 3), ("lv3_radius", C.c_double),
                ("lv3_margin", C.c_double), ("tracer", C.c_int), ("tracer_dh", C.c_double),
                ("emission", C.c_int), ("fl_n_lines", C.c_int), ("fl_lines_nm", C.c_void_p),
                ("fl_yield_per_mev", C.c_void_p), ("fl_dedx", C.c_double), ("tc_poll_limit", C.c_int),
                ("exact_queue", C.c_int)]


CS_TRACER_TABLES, CS_TRACER_SNELL = 0, 1
CS_EMIT_CHERENKOV, CS_EMIT_FLUORESCENCE, CS_EMIT_FLUORESCENCE_HALF = 0, 1, 2


def set_fluorescence(o, fl):
    """Fill the emission fields of a cs_opts from dict(lines_nm, yield_per_mev, dedx, half);
    returns the arrays the struct points to (keep them alive for the call)."""
    if not fl:
        return None
    lines = np.ascontiguousarray(fl["lines_nm"], np.float64)
    ys = np.ascontiguousarray(fl["yield_per_mev"], np.float64)
    o.emission = CS_EMIT_FLUORESCENCE_HALF if fl.get("half") else CS_EMIT_FLUORESCENCE
    o.fl_n_lines = len(lines)
    o.fl_lines_nm, o.fl_yield_per_mev = lines.ctypes.data, ys.ctypes.data
    o.fl_dedx = fl.get("dedx", 2.2)
    return lines, ys


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError("CUDA library not built: %s (run __graft_entry__.build())" % _LIB_PATH)
            L = C.CDLL(_LIB_PATH)
            vp, st = C.c_void_p, C.c_int
            L.cs_status_string.restype = C.c_char_p
            L.cs_status_string.argtypes = [st]
            L.cs_last_error.restype = C.c_char_p
            L.cs_atmosphere_create.argtypes = [C.POINTER(cs_atmosphere_desc), C.POINTER(vp)]
            L.cs_atmosphere_create.restype = st
            L.cs_atmosphere_destroy.argtypes = [vp]
            L.cs_atmosphere_table_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                                   C.POINTER(C.c_double), C.POINTER(C.c_double),
                                                   C.POINTER(C.c_double)]
            L.cs_atmosphere_table_info.restype = st
            L.cs_atmosphere_copy_table.argtypes = [vp, vp, C.c_size_t]
            L.cs_atmosphere_copy_table.restype = st
            L.cs_detector_create.argtypes = [C.POINTER(cs_detector_desc), C.POINTER(vp)]
            L.cs_detector_create.restype = st
            L.cs_detector_destroy.argtypes = [vp]
            L.cs_opts_default.argtypes = [C.POINTER(cs_opts)]
            L.cs_propagate.argtypes = [vp, C.c_size_t, vp, vp, C.c_uint64, C.POINTER(cs_output)]
            L.cs_propagate.restype = st
            L.cs_propagate_ex.argtypes = [vp, C.c_size_t, vp, vp, C.c_uint64, C.POINTER(cs_opts),
                                          C.POINTER(cs_output), vp]
            L.cs_propagate_ex.restype = st
            L.cs_batch_create.argtypes = [vp, C.c_size_t, vp, vp, C.c_uint64, vp, C.POINTER(cs_opts),
                                          C.POINTER(cs_output), C.POINTER(vp)]
            L.cs_batch_create.restype = st
            L.cs_batch_launch.argtypes = [vp, vp]
            L.cs_batch_launch.restype = st
            L.cs_batch_destroy.argtypes = [vp]
            L.cs_streamer_create.argtypes = [C.c_size_t, C.POINTER(vp)]
            L.cs_streamer_create.restype = st
            L.cs_streamer_run.argtypes = [vp, vp, C.c_size_t, vp, vp, C.c_uint64, C.POINTER(cs_opts),
                                          C.POINTER(cs_output), vp]
            L.cs_streamer_run.restype = st
            L.cs_streamer_destroy.argtypes = [vp]
            L.cs_autotune_tiling.argtypes = [vp, C.c_size_t, vp, vp, C.c_uint64, vp, C.POINTER(cs_opts),
                                             C.POINTER(cs_output), vp, C.POINTER(cs_tune_result)]
            L.cs_autotune_tiling.restype = st
            L.cs_autotune_bunches.argtypes = [vp, C.c_size_t, vp, vp, C.c_uint64, C.c_double, vp, C.c_int,
                                              C.POINTER(cs_opts), C.POINTER(cs_output), vp, vp]
            L.cs_autotune_bunches.restype = st
            L.cs_surrogate_config_default.argtypes = [C.POINTER(cs_surrogate_config)]
            L.cs_surrogate_train.argtypes = [vp, C.POINTER(cs_surrogate_config), C.POINTER(vp),
                                             C.POINTER(cs_surrogate_stats)]
            L.cs_surrogate_train.restype = st
            L.cs_surrogate_destroy.argtypes = [vp]
            L.cs_surrogate_eval.argtypes = [vp, vp, C.c_size_t, vp, vp]
            L.cs_surrogate_eval.restype = st
            L.cs_surrogate_eval_network.argtypes = [vp, vp, C.c_size_t, vp, vp]
            L.cs_surrogate_eval_network.restype = st
            L.cs_surrogate_info.argtypes = [vp, vp, C.c_size_t, C.POINTER(cs_surrogate_stats), vp]
            L.cs_surrogate_info.restype = st
            L.cs_mlp_loss_grad.argtypes = [vp, vp, vp, C.c_int, vp, vp]
            L.cs_mlp_loss_grad.restype = st
            L.cs_propagate_noalloc.argtypes = L.cs_propagate_ex.argtypes
            L.cs_propagate_noalloc.restype = st
            L.cs_philox4x32_10.argtypes = [vp, C.c_size_t, C.c_uint32, C.c_uint32, vp, vp]
            L.cs_philox4x32_10.restype = st
            L.cs_device_sm_count.argtypes = [C.POINTER(C.c_int)]
            L.cs_device_sm_count.restype = st
            L.cs_check_timeout.argtypes = []
            L.cs_check_timeout.restype = st
            _lib = L
    return _lib


def status_string(s):
    return lib().cs_status_string(int(s)).decode()


def last_error():
    return lib().cs_last_error().decode()


def _check(status, where):
    if status != CS_OK:
        raise CSError(status, where)


def _dptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------
# C-ABI calls (same names as include/cherenkov.h)
# --------------------------------------------------------------------------
def cs_atmosphere_create(desc: cs_atmosphere_desc):
    h = C.c_void_p()
    _check(lib().cs_atmosphere_create(C.byref(desc), C.byref(h)), "cs_atmosphere_create")
    return h


def cs_atmosphere_destroy(h):
    lib().cs_atmosphere_destroy(h)


def cs_atmosphere_table_info(h):
    nh, nw = C.c_int(), C.c_int()
    h0, dh, dw = C.c_double(), C.c_double(), C.c_double()
    _check(lib().cs_atmosphere_table_info(h, C.byref(nh), C.byref(nw), C.byref(h0), C.byref(dh), C.byref(dw)),
           "cs_atmosphere_table_info")
    return dict(nh=nh.value, nw=nw.value, h0=h0.value, dh=dh.value, dw=dw.value)


def cs_atmosphere_copy_table(h):
    info = cs_atmosphere_table_info(h)
    buf = np.zeros((info["nh"], info["nw"], 2, 4), np.float32)
    _check(lib().cs_atmosphere_copy_table(h, _dptr(buf), buf.size), "cs_atmosphere_copy_table")
    return buf


def cs_detector_create(desc: cs_detector_desc):
    h = C.c_void_p()
    _check(lib().cs_detector_create(C.byref(desc), C.byref(h)), "cs_detector_create")
    return h


def cs_detector_destroy(h):
    lib().cs_detector_destroy(h)


def cs_opts_default():
    o = cs_opts()
    lib().cs_opts_default(C.byref(o))
    return o


def cs_propagate(segs_ptr, n, atm, det, seed, out: cs_output):
    return lib().cs_propagate(segs_ptr, n, atm, det, seed, C.byref(out))


def cs_propagate_ex(segs_ptr, n, atm, det, seed, opts: cs_opts, out: cs_output, stream=None):
    return lib().cs_propagate_ex(segs_ptr, n, atm, det, seed, C.byref(opts), C.byref(out), stream)


def cs_batch_create(segs_ptr, n, atm, det, seed, shower_bunch, opts: cs_opts, out: cs_output):
    """shower_bunch: numpy int32 array (n_showers) or None."""
    h = C.c_void_p()
    sb = None if shower_bunch is None else np.ascontiguousarray(shower_bunch, np.int32)
    _check(lib().cs_batch_create(segs_ptr, n, atm, det, seed, None if sb is None else _dptr(sb), C.byref(opts),
                                 C.byref(out), C.byref(h)), "cs_batch_create")
    return h


def cs_batch_launch(batch, stream=None):
    return lib().cs_batch_launch(batch, stream)


def cs_batch_destroy(batch):
    lib().cs_batch_destroy(batch)


def cs_autotune_tiling(segs_ptr, n, atm, det, seed, shower_bunch, opts: cs_opts, out: cs_output, stream=None):
    r = cs_tune_result()
    sb = None if shower_bunch is None else np.ascontiguousarray(shower_bunch, np.int32)
    _check(lib().cs_autotune_tiling(segs_ptr, n, atm, det, seed, None if sb is None else _dptr(sb), C.byref(opts),
                                    C.byref(out), stream, C.byref(r)), "cs_autotune_tiling")
    return r


def cs_autotune_bunches(segs_ptr, n, atm, det, seed, rel_noise, allowed, opts: cs_opts, out: cs_output,
                        n_showers, stream=None):
    al = np.ascontiguousarray(allowed, np.int32)
    res = np.zeros(n_showers, np.int32)
    _check(lib().cs_autotune_bunches(segs_ptr, n, atm, det, seed, rel_noise, _dptr(al), len(al), C.byref(opts),
                                     C.byref(out), stream, _dptr(res)), "cs_autotune_bunches")
    return res


def cs_propagate_noalloc(segs_ptr, n, atm, det, seed, opts: cs_opts, out: cs_output, stream=None):
    return lib().cs_propagate_noalloc(segs_ptr, n, atm, det, seed, C.byref(opts), C.byref(out), stream)


def cs_philox4x32_10(ctr_ptr, n, key0, key1, out_ptr, stream=None):
    return lib().cs_philox4x32_10(ctr_ptr, n, key0, key1, out_ptr, stream)


def cs_check_timeout():
    """CS_ERR_TIMEOUT if a tensor-core wait of the surrogate gave up in a device-pointer,
    batched or streamed call since the last check (synchronises the device)."""
    return lib().cs_check_timeout()


def cs_device_sm_count():
    n = C.c_int()
    _check(lib().cs_device_sm_count(C.byref(n)), "cs_device_sm_count")
    return n.value


# --------------------------------------------------------------------------
# Descriptor and buffer helpers
# --------------------------------------------------------------------------
def pack_segments(cols) -> np.ndarray:
    n = len(cols["z0"])
    a = np.zeros(n, SEGMENT_DTYPE)
    for k in SEGMENT_DTYPE.names:
        if k in cols:
            a[k] = cols[k]
    return a


def _geometry(spherical, cylindrical):
    return CS_GEOM_CYLINDRICAL if cylindrical else CS_GEOM_SPHERICAL if spherical else CS_GEOM_PLANAR


class Atmosphere:
    """Owns a cs_atmosphere handle."""

    def __init__(self, kind=CS_ATM_LAYERED, layered=None, linear=None, hom_delta=0.0, h_obs=2000.0,
                 lambda_nm=(300.0, 600.0), refraction=False, transmission=False, transmission_params=None,
                 theta_max_deg=75.0, table_nw=0, table_dh=0.0, spherical=False, earth_radius=0.0, table=None,
                 kappa=2.9e-4, cylindrical=False):
        d = cs_atmosphere_desc()
        d.kind = kind
        self._keep = []
        if kind == CS_ATM_LAYERED:
            n = len(layered["layer_h"])
            arrs = [np.ascontiguousarray(layered[k], np.float64) for k in ("layer_h", "a", "b", "c")]
            self._keep += arrs
            d.n_layers = n
            d.layer_h, d.layer_a, d.layer_b, d.layer_c = (a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs)
            d.h_top, d.kappa = layered["h_top"], layered["kappa"]
        elif kind == CS_ATM_TABLE:
            arrs = [np.ascontiguousarray(table[k], np.float64) for k in ("h", "delta")]
            self._keep += arrs
            d.table_n = len(arrs[0])
            d.table_h, d.table_delta = (a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs)
            d.kappa = kappa
        elif kind == CS_ATM_LINEAR:
            d.lin_h0, d.lin_h1, d.lin_n0, d.lin_n1 = (linear[k] for k in ("lin_h0", "lin_h1", "lin_n0", "lin_n1"))
        else:
            d.hom_delta = hom_delta
        d.h_obs = h_obs
        d.lambda_min, d.lambda_max = lambda_nm[0] * 1e-9, lambda_nm[1] * 1e-9
        d.refraction, d.transmission = int(refraction), int(transmission)
        tp = dict(rayl_X0=2974.0, rayl_lambda0=400e-9, aer_tau0=0.05, aer_lambda0=350e-9, aer_alpha=1.3,
                  aer_H=1200.0)
        if transmission_params:
            tp.update(transmission_params)
        for k, v in tp.items():
            setattr(d, k, v)
        d.theta_max = math.radians(theta_max_deg)
        d.table_nw, d.table_dh = table_nw, table_dh
        d.geometry, d.earth_radius = _geometry(spherical, cylindrical), earth_radius
        self.desc = d
        self.h_obs = h_obs
        self.handle = cs_atmosphere_create(d)

    def table(self):
        return cs_atmosphere_copy_table(self.handle), cs_atmosphere_table_info(self.handle)

    def close(self):
        if self.handle:
            cs_atmosphere_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Detector:
    """Owns a cs_detector handle."""

    def __init__(self, n_showers=1, h_obs=2000.0, hist=None, tel=None, spherical=False, earth_radius=0.0,
                 optics=None, cylindrical=False):
        """optics: dict(mirror_d, focal_f, camera_r, point_zenith, point_azimuth [rad], cam_n
        [, efficiency=dict(lambda_nm, mirror, camera)]) for the last-mile ray tracing into
        per-telescope camera images, with the optics' absorption when efficiency is given."""
        d = cs_detector_desc()
        d.n_showers, d.h_obs = n_showers, h_obs
        self._eff = None
        if optics:
            for k in OPTICS_KEYS:
                setattr(d, k, optics[k])
            eff = optics.get("efficiency")
            if eff:
                self._eff = [np.ascontiguousarray(eff[k], np.float64) for k in ("lambda_nm", "mirror", "camera")]
                d.eff_n = len(self._eff[0])
                d.eff_lambda_nm, d.eff_mirror, d.eff_camera = (a.ctypes.data_as(C.POINTER(C.c_double))
                                                               for a in self._eff)
        d.geometry, d.earth_radius = _geometry(spherical, cylindrical), earth_radius
        if hist:
            d.hist_nx, d.hist_ny = hist["nx"], hist["ny"]
            d.hist_x0, d.hist_y0, d.hist_dx, d.hist_dy = hist["x0"], hist["y0"], hist["dx"], hist["dy"]
        self.tel = np.ascontiguousarray(np.zeros((0, 4)) if tel is None else np.asarray(tel, np.float64))
        d.n_tel = self.tel.shape[0]
        d.tel_xyzr = self.tel.ctypes.data_as(C.POINTER(C.c_double))
        self.n_showers, self.nx, self.ny, self.n_tel = n_showers, d.hist_nx, d.hist_ny, d.n_tel
        self.cam_n = d.cam_n if d.n_tel else 0
        self.desc = d
        self.handle = cs_detector_create(d)

    def close(self):
        if self.handle:
            cs_detector_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def propagate_host(segs, atm: Atmosphere, det: Detector, seed=0, bunch=1, s_max=1.0, seg_base=0,
                   records=False, record_capacity=None, blocks_per_sm=0, surrogate=None, lv1=None, lv3=None,
                   snell_dh=None, fluorescence=None, tc_poll_limit=0, allow_timeout=False, exact_queue=0):
    """cs_propagate_ex with host numpy buffers; returns a dict of outputs (with the
    call's status, CS_ERR_TIMEOUT accepted when allow_timeout)."""
    arr = segs if isinstance(segs, np.ndarray) else pack_segments(segs)
    arr = np.ascontiguousarray(arr)
    hist = np.zeros((det.n_showers, det.ny, det.nx), np.uint64)
    tel_counts = np.zeros((det.n_showers, det.n_tel), np.uint64)
    tel_time = np.zeros((det.n_showers, det.n_tel), np.float64)
    counters = np.zeros(CS_N_COUNTERS, np.uint64)
    rc = np.zeros(1, np.uint64)
    out = cs_output()
    out.hist = _dptr(hist) if det.nx else None
    out.tel_counts = _dptr(tel_counts) if det.n_tel else None
    out.tel_time = _dptr(tel_time) if det.n_tel else None
    out.counters = _dptr(counters)
    out.record_count = _dptr(rc)
    camera = np.zeros((det.n_showers, det.n_tel, det.cam_n, det.cam_n), np.uint64)
    out.camera = _dptr(camera) if det.cam_n else None
    rec = None
    if records:
        cap = record_capacity if record_capacity is not None else max(1024, 120 * len(arr))
        rec = np.zeros(cap, RECORD_DTYPE)
        out.records, out.record_capacity = _dptr(rec), cap
    o = cs_opts_default()
    o.bunch, o.s_max, o.seg_base, o.device_ptrs, o.blocks_per_sm = bunch, s_max, seg_base, 0, blocks_per_sm
    o.surrogate = surrogate.handle if surrogate is not None else None
    dropped = np.zeros(1, np.uint64)
    if lv1:
        set_lv1(o, lv1)
        o.lv1_dropped = dropped.ctypes.data
    set_lv3(o, lv3)
    if snell_dh:   # the Snell vector stepper through slabs <= snell_dh [m] instead of the tables
        o.tracer, o.tracer_dh = CS_TRACER_SNELL, snell_dh
    keep = set_fluorescence(o, fluorescence)   # noqa: F841 (the arrays must outlive the call)
    o.tc_poll_limit = tc_poll_limit
    o.exact_queue = exact_queue
    st = cs_propagate_ex(_dptr(arr) if len(arr) else None, len(arr), atm.handle, det.handle, seed, o, out)
    if not (allow_timeout and st == CS_ERR_TIMEOUT):
        _check(st, "cs_propagate_ex")
    res = dict(hist=hist, tel_counts=tel_counts, tel_time=tel_time, counters=counters, n_records=int(rc[0]),
               lv1_dropped=int(dropped[0]), camera=camera, status=st)
    if records:
        res["records"] = rec[: int(rc[0])]
    return res


def philox_device(ctr, key):
    """Philox4x32-10 of host counters (n x 4 uint32) on the device."""
    import torch
    c = torch.as_tensor(np.ascontiguousarray(ctr, np.uint32).view(np.int32)).cuda()
    o = torch.empty_like(c)
    st = cs_philox4x32_10(C.c_void_p(c.data_ptr()), c.shape[0], key[0], key[1], C.c_void_p(o.data_ptr()),
                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    _check(st, "cs_philox4x32_10")
    torch.cuda.synchronize()
    return o.cpu().numpy().view(np.uint32)


class DeviceOutputs:
    """Device output buffers (torch tensors) for a detector, with the matching
    cs_output struct."""

    def __init__(self, det: Detector, record_capacity=0, device="cuda:0"):
        import torch
        self.torch = torch
        d = torch.device(device)
        self.hist = torch.zeros((det.n_showers, max(det.ny, 1), max(det.nx, 1)), dtype=torch.int64, device=d)
        self.tel_counts = torch.zeros((det.n_showers, max(det.n_tel, 1)), dtype=torch.int64, device=d)
        self.tel_time = torch.zeros((det.n_showers, max(det.n_tel, 1)), dtype=torch.float64, device=d)
        self.counters = torch.zeros(CS_N_COUNTERS, dtype=torch.int64, device=d)
        self.record_count = torch.zeros(1, dtype=torch.int64, device=d)
        self.records = torch.zeros(record_capacity * RECORD_DTYPE.itemsize, dtype=torch.uint8, device=d) \
            if record_capacity else None
        self.camera = torch.zeros((det.n_showers, det.n_tel, det.cam_n, det.cam_n), dtype=torch.int64, device=d) \
            if det.cam_n else None
        o = cs_output()
        o.hist = self.hist.data_ptr() if det.nx else None
        o.tel_counts = self.tel_counts.data_ptr() if det.n_tel else None
        o.tel_time = self.tel_time.data_ptr() if det.n_tel else None
        o.counters = self.counters.data_ptr()
        o.record_count = self.record_count.data_ptr()
        if record_capacity:
            o.records, o.record_capacity = self.records.data_ptr(), record_capacity
        o.camera = self.camera.data_ptr() if self.camera is not None else None
        self.out = o

    def host(self):
        self.torch.cuda.synchronize()
        r = dict(hist=self.hist.cpu().numpy().astype(np.uint64), tel_counts=self.tel_counts.cpu().numpy().astype(np.uint64),
                 tel_time=self.tel_time.cpu().numpy(), counters=self.counters.cpu().numpy().astype(np.uint64),
                 n_records=int(self.record_count.item()))
        if self.camera is not None:
            r["camera"] = self.camera.cpu().numpy().astype(np.uint64)
        if self.records is not None:
            n = min(r["n_records"], self.out.record_capacity)
            r["records"] = self.records[: n * RECORD_DTYPE.itemsize].cpu().numpy().view(RECORD_DTYPE)
        return r


def stream_ptr():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# --------------------------------------------------------------------------
# surrogate network
# --------------------------------------------------------------------------
def cs_surrogate_config_default():
    c = cs_surrogate_config()
    lib().cs_surrogate_config_default(C.byref(c))
    return c


class Streamer:
    """Owns a cs_streamer: host segments streamed in chunks through two device
    buffers on two streams (copies overlap kernels)."""

    def __init__(self, chunk):
        h = C.c_void_p()
        _check(lib().cs_streamer_create(chunk, C.byref(h)), "cs_streamer_create")
        self.handle, self.chunk = h, chunk

    def run(self, host_segs_ptr, n, atm, det, out, seed=0, bunch=1, s_max=1.0, seg_base=0, accumulate=False,
            surrogate=None, stream=None, lv3=None):
        """host_segs_ptr: address of n packed segments in host memory; out: a
        cs_output of device pointers.  Enqueues on `stream` (default: torch's)."""
        o = cs_opts_default()
        o.bunch, o.s_max, o.seg_base, o.device_ptrs, o.accumulate = bunch, s_max, seg_base, 1, int(accumulate)
        if surrogate is not None:
            o.surrogate = surrogate.handle
        set_lv3(o, lv3)
        _check(lib().cs_streamer_run(self.handle, C.c_void_p(host_segs_ptr), n, atm.handle, det.handle, seed,
                                     C.byref(o), C.byref(out), stream if stream is not None else stream_ptr()),
               "cs_streamer_run")

    def close(self):
        if self.handle:
            lib().cs_streamer_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """Owns a trained cs_surrogate handle."""

    def __init__(self, atm: Atmosphere, cfg: cs_surrogate_config = None, **kw):
        c = cfg if cfg is not None else cs_surrogate_config_default()
        for k, v in kw.items():
            setattr(c, k, v)
        self.cfg = c
        h = C.c_void_p()
        st = cs_surrogate_stats()
        _check(lib().cs_surrogate_train(atm.handle, C.byref(c), C.byref(h), C.byref(st)), "cs_surrogate_train")
        self.handle = h
        self.stats = dict(p99=list(st.heldout_p99), max=list(st.heldout_max), final_loss=st.final_loss,
                          steps=st.steps, train_seconds=st.train_seconds)

    def info(self):
        p = np.zeros(N_MLP_PARAMS, np.float32)
        norm = np.zeros(15, np.float32)
        _check(lib().cs_surrogate_info(self.handle, _dptr(p), p.size, None, _dptr(norm)), "cs_surrogate_info")
        return p, norm

    def eval(self, inputs, network_only=False):
        """inputs: n x 3 (h_e - h_obs [m], cos(theta0), 1/lambda [1/nm]) -> n x 3 (G_R, G_t, T); with
        network_only, the network's part (G_R, G_t, ln T less the first-order baseline)."""
        import torch
        x = np.zeros((len(inputs), 4), np.float32)
        x[:, :3] = inputs
        d_in = torch.from_numpy(x).cuda()
        d_out = torch.zeros_like(d_in)
        fn = lib().cs_surrogate_eval_network if network_only else lib().cs_surrogate_eval
        _check(fn(self.handle, C.c_void_p(d_in.data_ptr()), len(x), C.c_void_p(d_out.data_ptr()), stream_ptr()),
               "cs_surrogate_eval")
        torch.cuda.synchronize()
        return d_out.cpu().numpy()[:, :3]

    def close(self):
        if self.handle:
            lib().cs_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cs_mlp_loss_grad(params, x, t):
    """One training-path forward/backward on the GPU (host arrays)."""
    p = np.ascontiguousarray(params, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    g = np.zeros_like(p)
    loss = np.zeros(1, np.float32)
    _check(lib().cs_mlp_loss_grad(_dptr(p), _dptr(x), _dptr(t), x.shape[0], _dptr(g), _dptr(loss)), "cs_mlp_loss_grad")
    return float(loss[0]), g


def mlp_padded_to_flat(p):
    """GPU parameter layout (W4, b4 padded to 8 rows) -> unpadded 3-64-64-64-3 layout."""
    o = 0
    parts = []
    for n in (64 * 3, 64, 64 * 64, 64, 64 * 64, 64):
        parts.append(p[o:o + n])
        o += n
    parts.append(p[o:o + 3 * 64])
    o += 8 * 64
    parts.append(p[o:o + 3])
    return np.concatenate(parts)


def mlp_flat_to_padded(f):
    out = np.zeros(N_MLP_PARAMS, np.float32)
    n_head = 64 * 3 + 64 + 2 * (64 * 64 + 64)
    out[:n_head] = f[:n_head]
    out[n_head:n_head + 3 * 64] = f[n_head:n_head + 3 * 64]
    out[n_head + 8 * 64:n_head + 8 * 64 + 3] = f[n_head + 3 * 64:]
    return out
