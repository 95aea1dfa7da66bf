"""The LV1 particle filter's cut (thesis Sec. 4.3.2 and 6.2.1), fitted per detector.

The filter drops a segment before any photon is generated when its start
height y above the observation level and the angle x [deg] between its
direction and the point of interest satisfy y >= a x^b.  The thesis fits the
line (a, b) in the (angle, height) plane per experiment on labelled
simulations; here the labels come from a run with records: a segment
contributes when any of its bunches hit a telescope (or land in the
histogram).  For each slope b on a grid, a is the smallest value that keeps
every contributing segment (times a safety margin); the b removing the most
segments wins.
"""
from __future__ import annotations

import numpy as np

from .binding import CS_LV1_ARRAY_CENTRE, CS_LV1_ARRAY_DISC, CS_LV1_TELESCOPES


def _angle_to_spheres(segs, centres, radii):
    S = np.stack([segs["x0"], segs["y0"], segs["z0"]], 1)
    P = np.stack([segs["ux"], segs["uy"], segs["uz"]], 1).astype(np.float64)
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    best = np.full(len(S), 180.0)
    for C, r in zip(centres, radii):
        d = np.asarray(C, np.float64)[None, :] - S
        dn = np.linalg.norm(d, axis=1)
        c = np.clip(np.sum(P * d, 1) / dn, -1.0, 1.0)
        a = np.degrees(np.arccos(c) - np.arcsin(np.minimum(r / dn, 1.0)))
        best = np.minimum(best, np.where(dn > r, np.maximum(a, 0.0), 0.0))
    return best


def cut_parameters(segs, metric, h_obs=2000.0, centre=(0.0, 0.0, 2000.0), radius=0.0, tel=None):
    """(x [deg], y [m]) of every segment for the planar frame."""
    if metric == CS_LV1_TELESCOPES:
        tel = np.asarray(tel, np.float64)
        x = _angle_to_spheres(segs, tel[:, :3], tel[:, 3])
    else:
        x = _angle_to_spheres(segs, [centre], [radius if metric == CS_LV1_ARRAY_DISC else 0.0])
    return np.maximum(x, 1e-3), np.asarray(segs["z0"], np.float64) - h_obs


def contributing(records, n_segments, seg_base=0, histogram=False):
    """Segments with a bunch that hit a telescope (or, with histogram=True, a cell)."""
    hit = records["tel"] >= 0
    if histogram:
        hit |= records["bin"] >= 0
    mask = np.zeros(n_segments, bool)
    mask[(records["seg"][hit].astype(np.int64) - seg_base)] = True
    return mask


def fit_cut(x, y, keep, margin=1.1, b_grid=None):
    """The cut y >= a x^b removing the most segments while keeping every
    segment marked in `keep` (with a margin on a).  Returns dict(a, b, removed)."""
    b_grid = np.linspace(-10.0, 2.0, 241) if b_grid is None else b_grid
    lx, ly = np.log(x), np.log(np.maximum(y, 1e-3))
    best = dict(a=np.inf, b=0.0, removed=0.0)
    for b in b_grid:
        if keep.any():
            a = margin * float(np.exp(np.max(ly[keep] - b * lx[keep])))
        else:
            a = 0.0
        removed = float(np.mean(y >= a * x ** b))
        if removed > best["removed"]:
            best = dict(a=a, b=float(b), removed=removed)
    return best


__all__ = ["cut_parameters", "contributing", "fit_cut", "CS_LV1_ARRAY_CENTRE", "CS_LV1_ARRAY_DISC",
           "CS_LV1_TELESCOPES"]
