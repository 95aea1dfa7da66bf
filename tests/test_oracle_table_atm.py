"""Pins of the oracle's tabulated atmosphere (a user's n(h) table, Sec. 3.3):
n - 1 log-linear between nodes, so every interval is one exponential layer.

* A table sampled from the US-standard fit inside its lowest layer (where the
  fit is one exponential) is that layer exactly.
* Per-interval closed forms (exponential layers, Sec. 3.4.3) equal the
  adaptive quadrature.
* Columns equal a Gauss-Legendre integral of the density (numpy's nodes).
* A constant table is the homogeneous medium."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_04229_gb300 import synth

LAY = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
KAPPA = synth.US_STANDARD["kappa"]


def _layer0_table(top=4000.0, step=250.0):
    h = np.arange(0.0, top + 1e-9, step)
    h[-1] = top - 1e-6            # the last node is the top: stay inside layer 0
    return dict(h=h, delta=[oracle.atm_delta(LAY, x) for x in h])


def _rough_table():
    return synth.TABLE_PROFILE


def test_nodes_and_log_linear_interpolation():
    t = _rough_table()
    a = oracle.make_atm(oracle.ATM_TABLE, table=t)
    for h, d in zip(t["h"][:-1], t["delta"][:-1]):
        assert oracle.atm_delta(a, h) == pytest.approx(d, rel=1e-15)
    for i in range(len(t["h"]) - 2):
        mid = 0.5 * (t["h"][i] + t["h"][i + 1])
        assert oracle.atm_delta(a, mid) == pytest.approx(math.sqrt(t["delta"][i] * t["delta"][i + 1]), rel=1e-13)
    assert oracle.atm_delta(a, 40000.0) == 0.0 and oracle.atm_delta(a, 50000.0) == 0.0
    # density from n - 1
    assert oracle.atm_rho(a, 5000.0) == pytest.approx(oracle.RHO_REF * oracle.atm_delta(a, 5000.0) / KAPPA,
                                                      rel=1e-15)


def test_table_inside_one_fit_layer_is_that_layer():
    a = oracle.make_atm(oracle.ATM_TABLE, table=_layer0_table(), kappa=KAPPA)
    for h in (0.0, 1234.5, 2000.0, 3999.0):
        assert oracle.atm_delta(a, h) == pytest.approx(oracle.atm_delta(LAY, h), rel=1e-12)
    for h_e, deg in [(3500.0, 10.0), (3990.0, 45.0), (2800.0, 70.0)]:
        th = math.radians(deg)
        qt = oracle.refract_quad(a, 2000.0, h_e, th)
        ql = oracle.refract_quad(LAY, 2000.0, h_e, th)
        np.testing.assert_allclose(qt[:2], ql[:2], rtol=1e-10)


def test_closed_forms_equal_the_quadrature():
    a = oracle.make_atm(oracle.ATM_TABLE, table=_rough_table())
    for h_e, deg in [(2500.0, 0.0), (8000.0, 30.0), (14000.0, 55.0), (30000.0, 70.0), (39000.0, 75.0)]:
        th = math.radians(deg)
        c = oracle.refract_closed(a, 2000.0, h_e, th)
        q = oracle.refract_quad(a, 2000.0, h_e, th)
        assert c[0] == pytest.approx(q[0], rel=1e-9, abs=1e-9)
        assert c[1] == pytest.approx(q[1], rel=1e-11)
        assert c[2] == pytest.approx(q[2], rel=1e-9)


def test_column_equals_gauss_integral_of_density():
    t = _rough_table()
    a = oracle.make_atm(oracle.ATM_TABLE, table=t)
    x, w = np.polynomial.legendre.leggauss(40)
    edges = [2000.0] + [h for h in t["h"] if 2000.0 < h < 37000.0] + [37000.0]
    tot = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        pts = 0.5 * (lo + hi) + 0.5 * (hi - lo) * x
        tot += 0.5 * (hi - lo) * sum(wi * 100.0 * oracle.atm_rho(a, p) for wi, p in zip(w, pts))
    assert oracle.column(a, 2000.0, 37000.0) == pytest.approx(tot, rel=1e-13)
    # vertical slant column of the straight line is that column
    assert oracle.straight(a, 2000.0, 37000.0, 0.0)[2] == pytest.approx(tot, rel=1e-12)


def test_constant_table_is_the_homogeneous_medium():
    a = oracle.make_atm(oracle.ATM_TABLE, table=dict(h=[0.0, 1e5], delta=[3e-4, 3e-4]))
    hom = oracle.make_atm(oracle.ATM_HOMOGENEOUS, hom_delta=3e-4)
    for h_e, deg in [(5000.0, 20.0), (20000.0, 60.0)]:
        th = math.radians(deg)
        np.testing.assert_allclose(oracle.refract_quad(a, 2000.0, h_e, th)[:2],
                                   oracle.refract_quad(hom, 2000.0, h_e, th)[:2], rtol=1e-12)
        np.testing.assert_allclose(oracle.refract_closed(a, 2000.0, h_e, th)[:2],
                                   oracle.refract_closed(hom, 2000.0, h_e, th)[:2], rtol=1e-12)


def test_snell_stepper_converges_on_the_table():
    a = oracle.make_atm(oracle.ATM_TABLE, table=_rough_table())
    th = math.radians(50.0)
    q = oracle.refract_quad(a, 2000.0, 12000.0, th)
    errs = [abs(oracle.snell_stepper(a, 2000.0, 12000.0, th, dh)[0] - q[0]) for dh in (10.0, 1.0, 0.1)]
    assert errs[2] < errs[1] < errs[0] and errs[2] < 1e-3


def test_propagation_in_layer0_table_equals_layered():
    segs = synth.tiny_vertical_segments(40, seed=3)
    segs["z0"][:] = 3000.0 + 0.1 * np.arange(40)
    a = oracle.make_atm(oracle.ATM_TABLE, table=_layer0_table(), kappa=KAPPA)
    kw = dict(hist=synth.histogram_400(), bunch=1, refraction=True, transmission=False, seed=2)
    rt = oracle.propagate(segs, a, **kw)["records"]
    rl = oracle.propagate(segs, LAY, **kw)["records"]
    assert len(rt) == len(rl) > 1000
    np.testing.assert_allclose(rt["x"], rl["x"], rtol=0, atol=1e-7)
    np.testing.assert_allclose(rt["dt"], rl["dt"], rtol=1e-11)
    assert np.array_equal(rt["status"], rl["status"])
