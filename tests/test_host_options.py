"""Host-side option handling (no GPU): the library's defaults, the binding's
helpers that fill the LV1, LV3, stepper and fluorescence fields of cs_opts,
and the benchmark's use of the committed ncu capture."""
import ctypes as C
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def B():
    from paper_2405_04229_gb300 import build
    build.build()
    from paper_2405_04229_gb300 import binding
    return binding


def test_defaults(B):
    o = B.cs_opts_default()
    assert o.bunch == 1 and o.s_max == 1.0 and o.device_ptrs == 0 and o.accumulate == 0
    assert o.lv1_metric == B.CS_LV1_OFF and o.lv3 == 0
    assert o.tracer == B.CS_TRACER_TABLES and o.tracer_dh == 10.0
    assert o.emission == B.CS_EMIT_CHERENKOV and o.fl_n_lines == 0 and o.fl_dedx == 2.2
    assert o.exact_queue == 0 and o.tc_poll_limit == 0   # default queue (8 entries per warp tile); default polls


def test_filter_and_emission_helpers_fill_the_struct(B):
    from paper_2405_04229_gb300 import synth
    o = B.cs_opts_default()
    B.set_lv1(o, dict(metric=B.CS_LV1_ARRAY_DISC, a=2.0, b=-1.5, centre=(1.0, 2.0, 2000.0), radius=30.0))
    assert (o.lv1_metric, o.lv1_a, o.lv1_b, o.lv1_radius) == (B.CS_LV1_ARRAY_DISC, 2.0, -1.5, 30.0)
    assert list(o.lv1_centre) == [1.0, 2.0, 2000.0]
    B.set_lv3(o, dict(centre=(5.0, -5.0, 2000.0), radius=100.0, margin=7.0))
    assert o.lv3 == 1 and list(o.lv3_centre) == [5.0, -5.0, 2000.0] and (o.lv3_radius, o.lv3_margin) == (100.0, 7.0)
    keep = B.set_fluorescence(o, dict(synth.FLUORESCENCE, half=True))
    assert o.emission == B.CS_EMIT_FLUORESCENCE_HALF and o.fl_n_lines == 5 and o.fl_dedx == 2.2
    lines = np.ctypeslib.as_array(C.cast(o.fl_lines_nm, C.POINTER(C.c_double)), shape=(5,))
    ys = np.ctypeslib.as_array(C.cast(o.fl_yield_per_mev, C.POINTER(C.c_double)), shape=(5,))
    assert lines.tolist() == synth.FLUORESCENCE["lines_nm"]
    assert ys.tolist() == synth.FLUORESCENCE["yield_per_mev"]
    assert keep[0] is not None
    o2 = B.cs_opts_default()
    assert B.set_fluorescence(o2, None) is None and o2.emission == B.CS_EMIT_CHERENKOV


def test_fluorescence_line_list_is_synthetic_and_in_band():
    from paper_2405_04229_gb300 import synth
    fl = synth.FLUORESCENCE
    assert len(fl["lines_nm"]) == len(fl["yield_per_mev"]) <= 8
    assert all(300.0 <= l <= 600.0 for l in fl["lines_nm"])   # inside the default wavelength band
    assert all(y > 0 for y in fl["yield_per_mev"])


def test_bench_uses_the_capture_only_for_the_captured_sources(monkeypatch):
    import bench
    kv = dict(l.strip().split("=", 1) for l in open(os.path.join(ROOT, "profiles", "propagate_kernel_traffic.txt"))
              if "=" in l and not l.startswith("#"))
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: kv["kernel_sources_sha256"])
    traffic, pipes = bench.kernel_profile()
    assert traffic == float(kv["bytes_per_launch"]) and traffic > 64e6   # at least the segments' bytes
    assert set(pipes) >= {"issue_active", "alu", "fma"}
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: "0" * 16)
    assert bench.kernel_profile() == (None, None)   # a changed kernel reports no stale counters


def test_bench_reads_the_inclined_chunk_traffic_scaled_from_its_capture(monkeypatch):
    import bench
    name = "propagate_kernel_spherical_traffic.txt"
    kv = dict(l.strip().split("=", 1) for l in open(os.path.join(ROOT, "profiles", name)) if "=" in l and not l.startswith("#"))
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: kv["kernel_sources_sha256"])
    traffic, _ = bench.kernel_profile(name)
    assert traffic == float(kv["bytes_per_launch"])
    assert 640e6 <= traffic <= 1.2 * 640e6   # a 1e7-segment chunk reads its 640 MB of segments, little more
