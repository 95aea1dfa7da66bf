"""Pins of the oracle's Snell vector stepper as a propagation method (Sec.
3.4.2, Eq. 3.15): its slant columns converge to the exact path's quadrature
as the slabs thin, a homogeneous medium is a straight line, the vertical
columns follow the midpoint rule, and the photon pipeline with the stepper
lands its photons where the exact path does, up to the stepper's own
discretisation."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import synth

C = 299792458.0
LAY = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
TAB = oracle.make_atm(oracle.ATM_TABLE, table=synth.TABLE_PROFILE)


@pytest.mark.parametrize("atm", [LAY, TAB], ids=["layered", "table"])
@pytest.mark.parametrize("deg", [0.0, 35.0, 65.0])
def test_columns_converge_to_the_exact_path(atm, deg):
    th = math.radians(deg)
    q = oracle.refract_quad(atm, 2000.0, 13000.0, th)
    errs = []
    for dh in (20.0, 2.0, 0.2):
        p = oracle.snell_path(atm, 2000.0, 13000.0, th, dh)
        errs.append(np.abs(p[1:] - q[1:]) / np.abs(q[1:]))
    errs = np.array(errs)
    assert (errs[2] < 2e-5).all(), errs
    assert (errs[2] <= errs[0] + 1e-12).all()
    if deg > 0:
        p = oracle.snell_path(atm, 2000.0, 13000.0, th, 0.2)
        assert abs(p[0] - q[0]) / q[0] < 1e-4


def test_homogeneous_medium_is_a_straight_line():
    for delta in (0.0, 2.5e-4):
        hom = oracle.make_atm(oracle.ATM_HOMOGENEOUS, hom_delta=delta)
        for deg in (0.0, 25.0, 70.0):
            th = math.radians(deg)
            p = oracle.snell_path(hom, 2000.0, 9000.0, th, 7.0)
            assert abs(p[0] - 7000.0 * math.tan(th)) < 1e-8
            assert abs(p[1] - (1.0 + delta) * 7000.0 / math.cos(th) / C) < 1e-15
            assert p[2] == 0.0


def test_vertical_aerosol_column_is_the_midpoint_rule():
    """Vertically the slabs are the midpoint rule of the aerosol integral
    H (e^{-h_obs/H} - e^{-h_e/H}): error (step^2 / 24) f'' per unit height."""
    H = 1200.0
    for dh in (10.0, 1.0):
        p = oracle.snell_path(LAY, 2000.0, 8000.0, 0.0, dh, H_A=H)
        n = math.ceil(6000.0 / dh - 1e-9)
        step = 6000.0 / n
        mid = sum(math.exp(-(8000.0 - (j + 0.5) * step) / H) * step for j in range(n))
        assert abs(p[3] - mid) < 1e-9 * mid
        exact = H * (math.exp(-2000.0 / H) - math.exp(-8000.0 / H))
        assert abs(p[3] - exact) <= (step ** 2 / 24.0) / H ** 2 * exact * 1.01


def test_pipeline_stepper_lands_where_the_exact_path_does():
    segs = synth.shower_segments(300, 30.0, 20.0, 1e12, seed=3)
    kw = dict(bunch=2, refraction=True, transmission=False, seed=4)
    ex = oracle.propagate(segs, LAY, **kw)["records"]
    st = oracle.propagate(segs, LAY, snell_dh=1.0, **kw)["records"]
    assert np.array_equal(ex["seg"], st["seg"]) and np.array_equal(ex["status"], st["status"])
    m = ex["status"] == oracle.ST_LANDED
    assert m.sum() > 5000
    line = oracle.propagate(segs, LAY, bunch=2, refraction=False, transmission=False,
                            seed=4)["records"]
    shift = np.hypot(ex["x"] - line["x"], ex["y"] - line["y"])[m]   # the refraction correction
    err = np.hypot(ex["x"] - st["x"], ex["y"] - st["y"])[m]
    assert shift.max() > 0.1
    assert (err <= 2e-3 * shift + 1e-6).all(), float((err / np.maximum(shift, 1e-9)).max())
    dt = np.abs(ex["dt"] - st["dt"])[m] / ex["dt"][m]
    assert dt.max() < 1e-7


# ---- the spherical shell ----------------------------------------------------
@pytest.mark.parametrize("deg", [30.0, 60.0, 75.0])
def test_shell_stepper_converges_to_the_bouguer_quadrature(deg):
    th = math.radians(deg)
    q = oracle.sph_path(LAY, 2000.0, 15000.0, th, rtol=1e-12)
    errs = np.array([np.abs(oracle.snell_path_sph(LAY, 2000.0, 15000.0, th, dh) - q) / np.abs(q)
                     for dh in (20.0, 2.0, 0.2)])
    assert (errs[2] < 2e-8).all(), errs
    assert (errs[1] < errs[0]).all() and (errs[2][:2] < errs[1][:2]).all()


def test_shell_stepper_vertical_equals_the_slab_stepper():
    """Straight down, shells and slabs are the same layers."""
    s = oracle.snell_path_sph(LAY, 2000.0, 12000.0, 0.0, 7.0)
    p = oracle.snell_path(LAY, 2000.0, 12000.0, 0.0, 7.0)
    assert s[0] == 0.0
    np.testing.assert_allclose(s[1:], p[1:], rtol=1e-12)


def test_shell_stepper_in_a_homogeneous_medium_is_the_straight_line():
    hom = oracle.make_atm(oracle.ATM_HOMOGENEOUS, hom_delta=3e-4)
    for deg in (20.0, 70.0):
        th = math.radians(deg)
        s = oracle.snell_path_sph(hom, 2000.0, 9000.0, th, 5.0)
        line = oracle.sph_path(hom, 2000.0, 9000.0, th, refraction=False)
        assert abs(s[0] - line[0]) < 1e-10 * max(line[0], 1e-3)   # FP64 with r^2 ~ 4e13 m^2
        assert abs(s[1] - (1 + 3e-4) * line[1]) < 1e-10 * s[1]


def test_pipeline_shell_stepper_lands_where_the_exact_path_does():
    segs = synth.shower_segments(300, 60.0, 20.0, 1e13, seed=5)
    kw = dict(bunch=2, refraction=True, transmission=False, seed=4, spherical=True)
    ex = oracle.propagate(segs, LAY, **kw)["records"]
    st = oracle.propagate(segs, LAY, snell_dh=1.0, **kw)["records"]
    assert np.array_equal(ex["seg"], st["seg"]) and np.array_equal(ex["status"], st["status"])
    m = ex["status"] == oracle.ST_LANDED
    assert m.sum() > 3000
    line = oracle.propagate(segs, LAY, bunch=2, refraction=False, transmission=False, seed=4,
                            spherical=True)["records"]
    shift = np.hypot(ex["x"] - line["x"], ex["y"] - line["y"])[m]
    err = np.hypot(ex["x"] - st["x"], ex["y"] - st["y"])[m]
    assert shift.max() > 1.0
    assert (err <= 1e-3 * shift + 1e-4).all(), float((err / np.maximum(shift, 1e-9)).max())
