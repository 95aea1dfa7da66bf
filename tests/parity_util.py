"""Photon-by-photon comparison of the CUDA path's records with the oracle's.

Bunches are matched by their key (segment, sub-step, bunch index).  Tolerances
follow the method's parity rules: per-photon positions and times agree to a
relative 1e-5 (positions relative to the horizontal displacement from the
emission point, floor 1 m); counts are bit-exact except bunches the oracle
flags as lying within an edge band (bin or sphere edge, count-rounding,
absorption threshold, the condition for reaching the ground, layer
boundary).  A segment whose sub-step count is itself a rounding decision is
left out as a whole.
"""
import numpy as np

import oracle

POS_REL = 1e-5
T_REL = 1e-5
LAMBDA_REL = 1e-6


def _key(seg, k, i):
    seg = np.asarray(seg, np.uint64)
    k = np.asarray(k, np.uint64)
    i = np.asarray(i, np.uint64)
    assert np.all(k < 2**16) and np.all(i < 2**16) and np.all(seg < 2**32)
    return (seg << np.uint64(32)) | (k << np.uint64(16)) | i


def position(rec):
    """Ground position of GPU records in FP64: the float-float pair summed."""
    return (rec["x"].astype(np.float64) + rec["x_lo"].astype(np.float64),
            rec["y"].astype(np.float64) + rec["y_lo"].astype(np.float64))


def compare(gpu, orc, bunch=1, shower_of_seg=None, pos_rel=POS_REL, t_rel=T_REL, check_hist=True):
    """Asserts parity; returns summary statistics.  Positions agree to pos_rel
    times max(1 m, the horizontal displacement from the emission point)."""
    g = g_all = gpu["records"]
    assert gpu["n_records"] == len(g), "GPU record capacity exceeded"
    o_all = orc["records"]
    sub = o_all[o_all["status"] == oracle.ST_SUBSTEP_FLAG]
    o = o_all[o_all["status"] != oracle.ST_SUBSTEP_FLAG]
    flagged_sub = set(zip(sub["seg"].tolist(), sub["k"].tolist()))
    # segments whose sub-step count K = ceil(L / s_max) is a rounding decision: every
    # bunch of them may differ, so they take no part in the per-photon comparison
    seg_out = np.unique(sub["seg"][(sub["flags"] & oracle.FL_SEGMENT) != 0])
    n_seg_out = int(np.isin(g["seg"], seg_out).sum())
    g = g[~np.isin(g["seg"], seg_out)]
    o = o[~np.isin(o["seg"], seg_out)]

    kg, ko = _key(g["seg"], g["k"], g["i"]), _key(o["seg"], o["k"], o["i"])
    assert len(np.unique(kg)) == len(kg), "duplicate GPU records"
    og, oo = np.argsort(kg), np.argsort(ko)
    g, kg = g[og], kg[og]
    o, ko = o[oo], ko[oo]
    common, ig, io = np.intersect1d(kg, ko, assume_unique=True, return_indices=True)
    only_g = np.setdiff1d(np.arange(len(g)), ig)
    only_o = np.setdiff1d(np.arange(len(o)), io)
    for j in only_o:
        assert o["flags"][j] & (oracle.FL_COUNT | oracle.FL_LV1), "oracle bunch missing on the GPU: %r" % (o[j],)
    for j in only_g:
        assert (int(g["seg"][j]), int(g["k"][j])) in flagged_sub, "extra GPU bunch: %r" % (g[j],)

    G, O = g[ig], o[io]
    fl = O["flags"]
    status_flags = (oracle.FL_ABSORB | oracle.FL_GROUND | oracle.FL_BELOW | oracle.FL_UPWARD | oracle.FL_LAYER |
                    oracle.FL_LV3)
    same_status = G["status"].astype(np.int64) == O["status"].astype(np.int64)
    bad = ~same_status & ((fl & status_flags) == 0)
    assert not bad.any(), "status mismatch: gpu %r oracle %r" % (G[bad][:3], O[bad][:3])

    # continuous values for bunches that were propagated to the ground on both sides
    prop = same_status & np.isin(O["status"], [oracle.ST_LANDED, oracle.ST_ABSORBED]) & ((fl & oracle.FL_LAYER) == 0)
    disp = np.maximum(1.0, np.hypot(O["x"] - O["ex"], O["y"] - O["ey"]))
    gx, gy = position(G)
    ex = np.abs(gx - O["x"]) / disp
    ey = np.abs(gy - O["y"]) / disp
    et = np.abs(G["dt_ns"].astype(np.float64) * 1e-9 - O["dt"]) / np.maximum(O["dt"], 1e-12)
    el = np.abs(G["lambda_nm"].astype(np.float64) * 1e-9 - O["lam"]) / O["lam"]
    max_pos = float(max(ex[prop].max(initial=0.0), ey[prop].max(initial=0.0)))
    max_t = float(et[prop].max(initial=0.0))
    assert max_pos <= pos_rel, "position error %.3g > %.3g" % (max_pos, pos_rel)
    assert max_t <= t_rel, "time error %.3g > %.3g" % (max_t, t_rel)
    assert float(el.max(initial=0.0)) <= LAMBDA_REL
    abs_pos = np.maximum(np.abs(gx - O["x"]), np.abs(gy - O["y"]))

    landed = same_status & (O["status"] == oracle.ST_LANDED)
    bin_bad = landed & (G["bin"] != O["bin"]) & ((fl & (oracle.FL_HIST_EDGE | oracle.FL_LAYER)) == 0)
    assert not bin_bad.any(), "bin mismatch outside the edge band: %r / %r" % (G[bin_bad][:3], O[bin_bad][:3])
    tel_bad = landed & (G["tel"] != O["tel"]) & ((fl & (oracle.FL_TEL_EDGE | oracle.FL_LAYER)) == 0)
    assert not tel_bad.any(), "telescope mismatch outside the edge band: %r / %r" % (G[tel_bad][:3], O[tel_bad][:3])
    # camera pixels (-1 on both sides without optics); rim and pixel edges carry the telescope flag
    pix_bad = landed & (G["pix"] != O["pix"]) & ((fl & (oracle.FL_TEL_EDGE | oracle.FL_LAYER | oracle.FL_OPTICS)) == 0)
    assert not pix_bad.any(), "camera pixel mismatch outside the edge band: %r / %r" % (G[pix_bad][:3], O[pix_bad][:3])

    # aggregates equal the records they summarise (the GPU's counts are its records')
    if check_hist and "hist" in gpu and gpu["hist"].size:
        h = np.zeros_like(gpu["hist"])
        m = g_all["bin"] >= 0
        sh = shower_of_seg
        showers = np.zeros(m.sum(), np.int64) if sh is None else np.asarray(sh, np.int64)[g_all["seg"][m].astype(np.int64)]
        np.add.at(h.reshape(h.shape[0], -1), (showers, g_all["bin"][m]), bunch)
        assert np.array_equal(h, gpu["hist"]), "GPU histogram differs from its records"
    cam = gpu.get("camera")
    if check_hist and cam is not None and cam.size:
        c = np.zeros_like(cam)
        m = g_all["pix"] >= 0
        sh = shower_of_seg
        showers = np.zeros(m.sum(), np.int64) if sh is None else np.asarray(sh, np.int64)[g_all["seg"][m].astype(np.int64)]
        np.add.at(c.reshape(cam.shape[0], cam.shape[1], -1), (showers, g_all["tel"][m], g_all["pix"][m]), bunch)
        assert np.array_equal(c, cam), "GPU camera images differ from their records"
    n_diff_bins = int(((G["bin"] != O["bin"]) & landed).sum())
    n_diff_tel = int(((G["tel"] != O["tel"]) & landed).sum())
    return dict(matched=len(common), flagged=int((fl != 0).sum()), only_gpu=len(only_g), only_oracle=len(only_o),
                segments_out=len(seg_out), gpu_bunches_out=n_seg_out,
                max_pos_rel=max_pos, max_t_rel=max_t, max_abs_pos=float(abs_pos[prop].max(initial=0.0)),
                status_flips=int((~same_status).sum()), bin_flips=n_diff_bins, tel_flips=n_diff_tel,
                pix_flips=int(((G["pix"] != O["pix"]) & landed).sum()),
                pix_hits=int((landed & (G["pix"] >= 0) & (G["pix"] == O["pix"]) & (fl == 0)).sum()))


def check_conservation(c):
    c = [int(v) for v in c]
    assert c[0] == c[1] + c[2] + c[4] == c[1] + c[3] + c[5], c
