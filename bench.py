#!/usr/bin/env python
"""Benchmark: Cherenkov photons propagated per second on GB300.

Workload (default): the refraction-corrected exact tracer -- 1e6 track
segments from 10 seeded 1 TeV-class showers at 20 deg zenith, bunch size 5,
US-standard layered atmosphere with refraction tables and Rayleigh + aerosol
transmission, a 400 x 400 ground histogram of 1 m cells per shower and 100
telescope spheres of 6 m radius on a 100 m grid, observation level 2 km.

One step = one call of the C ABI over the whole batch (zeroing the outputs,
importing the segments, generating, propagating and detecting every bunch).
Inputs are resident in HBM for ``value``; ``e2e`` repeats the measurement
through the host-pointer call (segments copied in, outputs copied out).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Cherenkov photons propagated/sec on 1 GB300 (exact vs surrogate) at stated error"
UNIT = "photons/s"
WORKLOAD = "refraction-corrected exact tracer: 1e6 segments, 10 showers, zenith 20 deg, bunch 5, 100 telescopes"

# Algorithmic FP32/INT lane operations per bunch of the method's hot path as
# planned before any kernel was written (Philox ~60, cone and rotation ~27,
# straight line ~9, four bilinear fields ~24, transmission ~7, detector ~11,
# plus index math: 130-160); the roofline's `achieved` uses the upper end.
OPS_PER_BUNCH_PLAN = 160
# The same counted item by item from the formulas as implemented (the
# float-float origins, both Philox draws, every index computation): per bunch,
# per sub-step, per segment.  Reported beside the planned count.
OPS_PER_BUNCH = 285
OPS_PER_SUBSTEP = 150
OPS_PER_SEGMENT = 120
SM_COUNT_NOMINAL = 152
LANES_PER_SM = 128


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("propagate.cu", "device_math.cuh", "common.cuh", "mlp_common.cuh", "mlp_tc.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2405_04229_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def kernel_profile(name="propagate_kernel_traffic.txt"):
    """Per-launch DRAM traffic and pipe utilisation of the photon kernel from the
    committed ncu captures, or None when the kernel sources changed since they
    were taken."""
    try:
        kv = dict(l.strip().split("=", 1) for l in open(os.path.join(ROOT, "profiles", name))
                  if "=" in l and not l.startswith("#"))
        if kv.get("kernel_sources_sha256") == kernel_sources_hash():
            pipes = {k[len("pipe_"):]: float(v) for k, v in kv.items() if k.startswith("pipe_")}
            return float(kv["bytes_per_launch"]), pipes or None
    except (OSError, ValueError, KeyError):
        pass
    return None, None


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def workload(seed, n_showers=10, per_shower=100_000):
    from paper_2405_04229_gb300 import synth
    segs = synth.refraction_showers(n_showers=n_showers, per_shower=per_shower, seed=seed)
    return segs, synth.grid_telescopes(), synth.histogram_400()


def substeps(segs, s_max=1.0):
    L = segs["length"].astype(np.float32)
    return int(np.maximum(1, np.ceil(L / np.float32(s_max))).sum())


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.strip().split("\n") if l.strip()]

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(segs, tel, hist, budget_s=12.0, chunk=250, bunch=5, seed=0, threads=None):
    """The FP64 oracle as it stands, on the host cores, over a bounded prefix
    of every shower of the workload; returns (photons/s, threads, sample)."""
    import concurrent.futures as cf

    import oracle
    from paper_2405_04229_gb300 import synth
    atm = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
    n = len(segs["z0"])
    n_showers = int(segs["shower_id"].max()) + 1
    per = n // n_showers
    threads = threads or os.cpu_count() or 1
    # interleave chunks across showers so the sample has every shower's shape
    starts = [s * per + j for j in range(0, per, chunk) for s in range(n_showers)]
    done_photons, done_segs = 0, 0
    t0 = time.perf_counter()
    lock = threading.Lock()

    def work(st):
        sl = slice(st, min(st + chunk, n))
        r = oracle.propagate(synth.take(segs, sl), atm, hist=hist, tel=tel, bunch=bunch, refraction=True,
                             transmission=True, seed=seed, seg_base=st, n_showers=n_showers, records=False)
        return int(r["counters"][0]), sl.stop - sl.start

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        it = iter(starts)
        futs = set()
        for _ in range(threads):
            st = next(it, None)
            if st is not None:
                futs.add(ex.submit(work, st))
        while futs:
            done, futs = cf.wait(futs, return_when=cf.FIRST_COMPLETED)
            for f in done:
                p, s = f.result()
                with lock:
                    done_photons += p
                    done_segs += s
            if time.perf_counter() - t0 < budget_s:
                for _ in done:
                    st = next(it, None)
                    if st is not None:
                        futs.add(ex.submit(work, st))
    dt = time.perf_counter() - t0
    return done_photons / dt, threads, "%d segments (%d-segment chunks spread over all %d showers), %.1f s" % (
        done_segs, chunk, n_showers, dt)


def cpu_model():
    """The host CPU's model string (x86 'model name', else lscpu's 'Model name')."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline_entry(segs, tel, hist):
    """The oracle on all host cores (the reported value) and on one core."""
    rate, cores, sample = cpu_oracle_rate(segs, tel, hist)
    rate1, _, sample1 = cpu_oracle_rate(segs, tel, hist, budget_s=4.0, threads=1)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "single_core": {"value": rate1, "sample": sample1}, "cpu_model": cpu_model()}


def cpu_baseline_sampled(segs, tel, hist, shower_bunch, budget_s=12.0, chunk=200, seed=0):
    """The oracle on all host cores over seeded random chunks of an uneven batch
    (each chunk with its shower's bunch size); photons/s of the sample."""
    import concurrent.futures as cf

    import oracle
    from paper_2405_04229_gb300 import synth
    atm = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
    n = len(segs["z0"])
    n_showers = int(segs["shower_id"].max()) + 1
    rng = np.random.default_rng([seed, 0xC9])
    starts = iter(rng.integers(0, max(1, n - chunk), 100000))
    threads = os.cpu_count() or 1
    photons, done = 0, 0
    t0 = time.perf_counter()

    def work(st):
        sl = slice(int(st), min(int(st) + chunk, n))
        sub = synth.take(segs, sl)
        # one shower per call: the chunk's first shower and its bunch size
        sid = sub["shower_id"] == sub["shower_id"][0]
        sub = synth.take(sub, sid)
        b = int(shower_bunch[int(sub["shower_id"][0])])
        r = oracle.propagate(sub, atm, hist=hist, tel=tel, bunch=b, refraction=True, transmission=True, seed=seed,
                             seg_base=int(st), n_showers=n_showers, records=False)
        return int(r["counters"][0]), len(sub["z0"])

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        futs = {ex.submit(work, next(starts)) for _ in range(threads)}
        while futs:
            fin, futs = cf.wait(futs, return_when=cf.FIRST_COMPLETED)
            for f in fin:
                p, s_ = f.result()
                photons += p
                done += s_
            if time.perf_counter() - t0 < budget_s:
                for _ in fin:
                    futs.add(ex.submit(work, next(starts)))
    dt = time.perf_counter() - t0
    return {"value": photons / dt, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": "%d segments in seeded random %d-segment chunks of the batch, %.1f s" % (done, chunk, dt)}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    segs, tel, hist = workload(args.seed)
    budget = max(5.0, min(60.0, 3.0 * (args.steps + args.warmup)))
    rate, cores, sample = cpu_oracle_rate(segs, tel, hist, budget_s=budget)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "inputs re-read per chunk on the host"},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """64 showers with log-uniform segment counts (1e4..1e7), zenith U(0, 40),
    one persistent graph-captured launch per step, bunch sizes and tiling
    chosen by the autotuner."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_04229_gb300 import binding as B
    from paper_2405_04229_gb300 import synth
    t0 = time.perf_counter()
    segs, counts = synth.uneven_showers(n_showers=64, seed=args.seed)
    gen_s = time.perf_counter() - t0
    segs_all = segs
    n = len(segs["z0"])
    tel = synth.grid_telescopes(nx=20, ny=20, pitch=100.0)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    det = B.Detector(n_showers=64, hist=synth.histogram_400(), tel=tel)
    arr = B.pack_segments(segs)
    del segs
    d_segs = torch.from_numpy(arr.view(np.uint8)).cuda()
    outs = B.DeviceOutputs(det)
    sp = B.stream_ptr()
    o = B.cs_opts_default()
    o.device_ptrs = 1
    segp = C.c_void_p(d_segs.data_ptr())
    sb = B.cs_autotune_bunches(segp, n, atm.handle, det.handle, args.seed, 0.05, [1, 2, 5, 10], o, outs.out, 64, sp)
    tune = B.cs_autotune_tiling(segp, n, atm.handle, det.handle, args.seed, sb, o, outs.out, sp)
    o.blocks_per_sm = tune.blocks_per_sm
    batch = B.cs_batch_create(segp, n, atm.handle, det.handle, args.seed, sb, o, outs.out)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        B.cs_batch_launch(batch, sp)
    torch.cuda.synchronize()
    photons = int(outs.counters[0].item())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(0) as clk:
        time.sleep(0.5)
        for a, b in ev:
            a.record(stream)
            B.cs_batch_launch(batch, sp)
            b.record(stream)
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    assert int(outs.counters[0].item()) == photons
    B.cs_batch_destroy(batch)
    h = outs.host()
    per_shower_bunch = {int(b): int((sb == b).sum()) for b in np.unique(sb)}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline_sampled(segs_all, tel, synth.histogram_400(), sb)
    line = {"metric": METRIC, "value": photons * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched uneven showers: 64 showers, log-uniform 1e4..1e7 segments, zenith 0-40 deg, "
                                   "400 telescopes, one graph-captured persistent launch",
                       "segments": n, "photons_per_step": photons, "bunch_sizes": per_shower_bunch,
                       "blocks_per_sm": tune.blocks_per_sm, "tiling_ms": [round(tune.ms[i], 3) for i in range(4)],
                       "generation_s": round(gen_s, 1), "l2": "inputs (%.1f GB) larger than L2" % (arr.nbytes / 1e9)},
            "counters": [int(x) for x in h["counters"]], "cpu_baseline": cpu, "gpu_launches": 2 * args.steps,
            "clocks": clk.summary()}
    if getattr(args, "quiet", False):
        return line
    print(json.dumps(line), flush=True)


# Extra lane operations per bunch on the spherical shell: the local vertical
# along the track, the local zenith, the straight line to the ground sphere,
# the ground tangent, the azimuthal-equidistant projection and Bouguer's
# arrival direction (counted from the formulas like the planar figures).
OPS_PER_BUNCH_SPHERICAL = OPS_PER_BUNCH + 85


def run_inclined(args):
    """Large inclined shower: 1e8 segments of a 100 TeV-class shower at zenith
    60 deg through the spherical-shell layered atmosphere, bunch 10, 2,000
    telescopes of 6 m radius (Poisson disk, separation >= 13 m, over
    [-1, 1) km^2) and the 400 x 400 histogram, streamed in 10 chunks of 1e7;
    the exact tracer and the surrogate."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_04229_gb300 import binding as B
    from paper_2405_04229_gb300 import synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    bunch, chunk, n_chunks = 10, args.chunk, args.chunks
    n = chunk * n_chunks
    seg_bytes = 64
    t0 = time.perf_counter()
    pinned = torch.empty(n * seg_bytes, dtype=torch.uint8).pin_memory()
    host = pinned.numpy()
    n_sub = 0
    for c in range(n_chunks):
        segs = synth.inclined_chunk(c, n=chunk, seed=args.seed)
        n_sub += substeps(segs)
        host[c * chunk * seg_bytes:(c + 1) * chunk * seg_bytes] = B.pack_segments(segs).view(np.uint8)
        if c == 0:
            sample_segs = synth.take(segs, slice(0, 20_000))
        del segs
    gen_s = time.perf_counter() - t0
    tel = synth.poisson_disk_telescopes(n=2000, half=1000.0, min_sep=13.0, radius=6.0, seed=args.seed)
    hist = synth.histogram_400()
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True, spherical=True)
    det = B.Detector(n_showers=1, hist=hist, tel=tel, spherical=True)
    outs = B.DeviceOutputs(det)
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)
    d_all = pinned.to(dev)
    base_ptr = d_all.data_ptr()
    o = B.cs_opts_default()
    o.bunch, o.device_ptrs = bunch, 1
    ev_k = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_chunks)]

    def step(timed_launches=False):
        for c in range(n_chunks):
            o.seg_base, o.accumulate = c * chunk, int(c > 0)
            if timed_launches:
                ev_k[c][0].record(stream)
            st = B.cs_propagate_ex(C.c_void_p(base_ptr + c * chunk * seg_bytes), chunk, atm.handle, det.handle,
                                   args.seed, o, outs.out, sp)
            if st != B.CS_OK:
                raise B.CSError(st, "cs_propagate_ex")
            if timed_launches:
                ev_k[c][1].record(stream)

    def timed(steps, fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b_ in ev:
            a.record(stream)
            fn()
            b_.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b_) for a, b_ in ev)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    photons = int(outs.counters[0].item())
    with ClockSampler(0) as clk:
        time.sleep(0.5)
        ms = timed(args.steps, step)
    assert int(outs.counters[0].item()) == photons
    value = photons * args.steps / (ms / 1e3)
    # launch durations of the photon kernel (one per chunk) for the roofline
    step(timed_launches=True)
    torch.cuda.synchronize()
    k_ms = sum(a.elapsed_time(b_) for a, b_ in ev_k) / n_chunks
    bunches = photons // bunch
    ops = OPS_PER_BUNCH_SPHERICAL * bunches + OPS_PER_SUBSTEP * n_sub + OPS_PER_SEGMENT * n
    achieved = ops / n_chunks / (k_ms / 1e3) / 1e12
    max_mhz = 2070.0
    try:
        max_mhz = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", max_mhz)
    except Exception:
        pass
    peak = B.cs_device_sm_count() * LANES_PER_SM * max_mhz * 1e6 / 1e12
    counters = [int(x) for x in outs.counters.cpu()]
    tel_full = int(outs.tel_counts.sum().item())
    hist_full = int(outs.hist.sum().item())
    tel_ref, hist_ref = outs.tel_counts.clone(), outs.hist.clone()

    # LV1 particle filter (Sec. 4.3.2, 6.2.1): cut fitted on a labelled sample of chunk 0
    lv1_res = None
    if args.lv1:
        from paper_2405_04229_gb300 import lv1 as L
        n_lab = min(chunk, 1_000_000)
        lab = synth.take(synth.inclined_chunk(0, n=chunk, seed=args.seed), slice(0, n_lab))
        lab_out = B.DeviceOutputs(det, record_capacity=40 * n_lab)
        ol = B.cs_opts_default()
        ol.bunch, ol.device_ptrs = bunch, 1
        st = B.cs_propagate_ex(C.c_void_p(base_ptr), n_lab, atm.handle, det.handle, args.seed, ol, lab_out.out, sp)
        if st != B.CS_OK:
            raise B.CSError(st, "cs_propagate_ex(labels)")
        recs = lab_out.host()["records"]
        keep = L.contributing(recs, n_lab, histogram=True)
        centre, radius = (0.0, 0.0, 2000.0), 1000.0 * math.sqrt(2.0) + 30.0
        x, y = L.cut_parameters(lab, B.CS_LV1_ARRAY_DISC, centre=centre, radius=radius)
        cut = L.fit_cut(x, y, keep, margin=1.2)
        del lab_out
        dropped = torch.zeros(1, dtype=torch.int64, device=dev)
        B.set_lv1(o, dict(metric=B.CS_LV1_ARRAY_DISC, a=cut["a"], b=cut["b"], centre=centre, radius=radius))
        o.lv1_dropped = dropped.data_ptr()
        step()
        torch.cuda.synchronize()
        f_photons = int(outs.counters[0].item())
        f_ms = timed(args.steps, step)
        lv1_res = {"metric": "disc about the array centre", "radius_m": radius, "a": cut["a"], "b": cut["b"],
                   "label_sample_segments": n_lab, "removed_in_sample": cut["removed"],
                   "dropped_segments_fraction": int(dropped.item()) / n, "ms_per_step": f_ms / args.steps,
                   "photons_per_s": f_photons * args.steps / (f_ms / 1e3),
                   "equivalent_photons_per_s": photons * args.steps / (f_ms / 1e3),
                   "speedup": ms / f_ms,
                   "telescope_count_retention": int(outs.tel_counts.sum().item()) / max(tel_full, 1),
                   "histogram_count_retention": int(outs.hist.sum().item()) / max(hist_full, 1)}
        o.lv1_metric, o.lv1_dropped = B.CS_LV1_OFF, None

    # LV3 photon pre-filter (Sec. 4.3.4, 6.2.2): photons whose straight line lands outside
    # the disc holding the array and the histogram, widened by a margin for the refraction
    # correction, skip the lookups, the transmission and the detection.  The margin is the
    # largest correction displacement seen on a sample (same photons with refraction on and
    # off) with 50 % headroom; the detector counts over the whole workload must not change.
    lv3_res = None
    if args.lv3:
        n_lab = min(chunk, 200_000)
        atm_line = B.Atmosphere(layered=synth.US_STANDARD, refraction=False, transmission=True, spherical=True)
        ol = B.cs_opts_default()
        ol.bunch, ol.device_ptrs = bunch, 1
        recs = []
        for a in (atm, atm_line):
            lab_out = B.DeviceOutputs(det, record_capacity=60 * n_lab)
            st = B.cs_propagate_ex(C.c_void_p(base_ptr), n_lab, a.handle, det.handle, args.seed, ol, lab_out.out, sp)
            if st != B.CS_OK:
                raise B.CSError(st, "cs_propagate_ex(sample)")
            recs.append(lab_out.host()["records"])
            del lab_out
        atm_line.close()
        key = [(r["seg"].astype(np.int64) << 24) | (r["k"].astype(np.int64) << 12) | r["i"].astype(np.int64)
               for r in recs]
        _, ia, ib = np.intersect1d(key[0], key[1], assume_unique=True, return_indices=True)
        ra, rb = recs[0][ia], recs[1][ib]
        both = np.isin(ra["status"], [B.CS_ST_LANDED, B.CS_ST_ABSORBED]) & \
            np.isin(rb["status"], [B.CS_ST_LANDED, B.CS_ST_ABSORBED])
        shift = float(np.hypot(ra["x"].astype(np.float64) - rb["x"], ra["y"].astype(np.float64) - rb["y"])[both].max())
        radius, margin = 1000.0 * math.sqrt(2.0) + 6.0, 1.5 * shift + 1.0
        straight = np.hypot(rb["x"].astype(np.float64), rb["y"].astype(np.float64))
        B.set_lv3(o, dict(centre=(0.0, 0.0, 2000.0), radius=radius, margin=margin))
        step()
        torch.cuda.synchronize()
        f_ms = timed(args.steps, step)
        lv3_res = {"metric": "straight-line landing point against a disc about the array centre",
                   "radius_m": radius, "margin_m": margin, "largest_correction_shift_m": shift,
                   "sample_segments": n_lab,
                   "dropped_photon_fraction_in_sample": float(((straight > radius + margin) & both).sum()) /
                   max(int(np.isin(rb["status"], [B.CS_ST_LANDED, B.CS_ST_ABSORBED]).sum()), 1),
                   "ms_per_step": f_ms / args.steps,
                   "equivalent_photons_per_s": photons * args.steps / (f_ms / 1e3),
                   "speedup": ms / f_ms,
                   "telescope_counts_unchanged": bool(torch.equal(outs.tel_counts, tel_ref)),
                   "histogram_counts_unchanged": bool(torch.equal(outs.hist, hist_ref))}
        o.lv3 = 0

    # end to end: pinned host segments streamed through the library's two-stream
    # double buffer, outputs read back every step
    e2e = None
    if not args.no_e2e:
        streamer = B.Streamer(chunk)
        cnt_h = torch.zeros(8, dtype=torch.int64).pin_memory()
        tel_h = torch.zeros(tel.shape[0], dtype=torch.int64).pin_memory()
        hist_h = torch.zeros(400 * 400, dtype=torch.int64).pin_memory()

        def estep():
            streamer.run(pinned.data_ptr(), n, atm, det, outs.out, seed=args.seed, bunch=bunch, stream=sp)
            cnt_h.copy_(outs.counters, non_blocking=True)
            tel_h.copy_(outs.tel_counts.view(-1), non_blocking=True)
            hist_h.copy_(outs.hist.view(-1), non_blocking=True)
            stream.synchronize()

        for _ in range(2):
            estep()
        assert int(cnt_h[0].item()) == photons
        e_s, e_dev = 0.0, 0.0
        for _ in range(args.steps):
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a = time.perf_counter()
            ea.record(stream)
            estep()
            eb.record(stream)
            e_s += time.perf_counter() - a
            eb.synchronize()
            e_dev += ea.elapsed_time(eb) / 1e3
        e2e = {"value": photons * args.steps / e_s, "unit": UNIT, "h2d_bytes_per_step": n * seg_bytes,
               "d2h_bytes_per_step": 8 * (8 + tel.shape[0] + 400 * 400),
               "form": "cs_streamer_run: %d chunks of %d segments, two streams, pinned host memory" % (n_chunks, chunk),
               "device_ms_per_step": 1e3 * e_dev / args.steps}
        streamer.close()

    # surrogate form on the same stream of chunks
    surrogate = None
    if not args.no_surrogate:
        t_tr = time.perf_counter()
        sur = B.Surrogate(atm, **({"epochs": args.surrogate_epochs} if args.surrogate_epochs else {}))
        train_s = time.perf_counter() - t_tr
        o.surrogate = sur.handle
        step()
        torch.cuda.synchronize()
        s_photons = int(outs.counters[0].item())
        s_ms = timed(args.steps, step)
        o.surrogate = None
        surrogate = {"value": s_photons * args.steps / (s_ms / 1e3), "unit": UNIT, "ms_per_step": s_ms / args.steps,
                     "speedup_vs_exact": (s_photons / s_ms) / (photons / ms),
                     "heldout_p99": {"displacement_m": sur.stats["p99"][0], "delay_s": sur.stats["p99"][1],
                                     "transmission": sur.stats["p99"][2]},
                     "heldout_max": {"displacement_m": sur.stats["max"][0], "delay_s": sur.stats["max"][1],
                                     "transmission": sur.stats["max"][2]},
                     "train_seconds": round(train_s, 2)}
        sur.close()

    cpu = None
    if not args.no_cpu_baseline:
        rate, cores, sample = cpu_oracle_rate_sph(sample_segs, tel, hist, bunch=bunch, seed=args.seed)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "large inclined shower: %d segments (%d chunks of %d), 100 TeV-class, zenith 60 deg, "
                                   "spherical-shell layered atmosphere, bunch 10, 2000 telescopes, exact tracer"
                                   % (n, n_chunks, chunk),
                       "segments": n, "photons_per_step": photons, "generation_s": round(gen_s, 1),
                       "l2": "inputs (%.1f GB) larger than L2" % (n * seg_bytes / 1e9)},
            "counters": counters,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": kernel_profile("propagate_kernel_spherical_traffic.txt")[0],
                         "note": "per chunk launch; spherical lane-op count per bunch %d" % OPS_PER_BUNCH_SPHERICAL},
            "kernel_ms": k_ms, "cpu_baseline": cpu, "surrogate": surrogate, "e2e": e2e, "lv1_filter": lv1_res, "lv3_filter": lv3_res,
            "gpu_launches": 2 * args.steps * n_chunks, "clocks": clk.summary()}
    if getattr(args, "quiet", False):
        return line
    print(json.dumps(line), flush=True)


def cpu_oracle_rate_sph(segs, tel, hist, bunch, seed, budget_s=12.0, chunk=200):
    """The oracle on the spherical shell over a bounded prefix of the shower."""
    import concurrent.futures as cf

    import oracle
    from paper_2405_04229_gb300 import synth
    atm = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
    n = len(segs["z0"])
    threads = os.cpu_count() or 1
    starts = list(range(0, n, chunk))
    photons, done = 0, 0
    t0 = time.perf_counter()

    def work(st):
        sl = slice(st, min(st + chunk, n))
        r = oracle.propagate(synth.take(segs, sl), atm, hist=hist, tel=tel, bunch=bunch, refraction=True,
                             transmission=True, seed=seed, seg_base=st, records=False, spherical=True)
        return int(r["counters"][0]), sl.stop - sl.start

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        it = iter(starts)
        futs = {ex.submit(work, st) for st in [next(it, None) for _ in range(threads)] if st is not None}
        while futs:
            fin, futs = cf.wait(futs, return_when=cf.FIRST_COMPLETED)
            for f in fin:
                p, s_ = f.result()
                photons += p
                done += s_
            if time.perf_counter() - t0 < budget_s:
                for _ in fin:
                    st = next(it, None)
                    if st is not None:
                        futs.add(ex.submit(work, st))
    dt = time.perf_counter() - t0
    return photons / dt, threads, "first %d segments of chunk 0 (%d-segment pieces), %.1f s" % (done, chunk, dt)


def run_tiny(steps=20, warmup=5, seed=0):
    """The plain method at its smallest: 1,000 electron tracks from 8-12 km, straight
    lines, bunch 1, the 400 x 400 histogram (launch-bound: a few thousand photons)."""
    import torch
    from paper_2405_04229_gb300 import binding as B
    from paper_2405_04229_gb300 import synth
    segs = synth.tiny_vertical_segments(1000, seed=seed)
    arr = B.pack_segments(segs)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=False, transmission=False)
    det = B.Detector(n_showers=1, hist=synth.histogram_400())
    outs = B.DeviceOutputs(det)
    d = torch.from_numpy(arr.view(np.uint8)).cuda()
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)
    o = B.cs_opts_default()
    o.bunch, o.device_ptrs = 1, 1

    def step():
        st = B.cs_propagate_ex(C.c_void_p(d.data_ptr()), len(arr), atm.handle, det.handle, seed, o, outs.out, sp)
        if st != B.CS_OK:
            raise B.CSError(st, "cs_propagate_ex(tiny)")

    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize()
    photons = int(outs.counters[0].item())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b_ in ev:
        a.record(stream)
        step()
        b_.record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b_) for a, b_ in ev) / steps
    h = outs.host()
    res = {"value": photons / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "photons_per_step": photons, "histogram_photons": int(h["hist"].sum()),
           "workload": "1,000 tracks 8-12 km, straight lines, bunch 1, 400 x 400 histogram (launch-bound)"}
    atm.close()
    det.close()
    return res


def extra_configs(args):
    """The other configurations as keys of the default line: the tiny straight-line
    case, the batched uneven showers (full size, one graph-captured launch) and the
    large inclined shower (full size, 10 chunks, with the LV1 and LV3 filters)."""
    sub = dict(seed=args.seed, warmup=3, steps=3, quiet=True, no_cpu_baseline=True)
    out = {"c1_tiny": run_tiny(seed=args.seed)}
    b = run_batched(argparse.Namespace(**sub))
    out["c3_batched"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "steps", "config", "gpu_launches", "clocks")}
    i = run_inclined(argparse.Namespace(**sub, chunk=args.chunk, chunks=args.chunks, lv1=True, lv3=True,
                                        no_e2e=False, no_surrogate=True))
    out["c5_inclined"] = {k: i[k] for k in ("value", "unit", "ms_per_step", "steps", "kernel_ms", "roofline", "e2e",
                                            "lv1_filter", "lv3_filter", "config", "gpu_launches", "clocks")}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--config", default="refraction", choices=["refraction", "batched", "inclined"])
    ap.add_argument("--chunk", type=int, default=10_000_000)
    ap.add_argument("--chunks", type=int, default=10)
    ap.add_argument("--lv1", action="store_true", help="inclined: also time the LV1 particle filter")
    ap.add_argument("--lv3", action="store_true", help="inclined: also time the LV3 photon pre-filter")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--per-shower", type=int, default=100_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--surrogate-epochs", type=int, default=0,
                    help="train the surrogate for this many epochs (0: the library's default); a short "
                         "training serves profiling runs of the surrogate kernel")
    ap.add_argument("--no-optics", action="store_true")
    ap.add_argument("--no-snell", action="store_true")
    ap.add_argument("--no-fluorescence", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave out the tiny, batched and inclined configurations' keys")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "batched":
        return run_batched(args)
    if args.config == "inclined":
        return run_inclined(args)

    import torch
    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2405_04229_gb300 import binding as B
    from paper_2405_04229_gb300 import synth

    bunch = 5
    # weak scaling: every rank propagates its own batch of showers (seeds differ,
    # segment ids are disjoint), no collective on the data path
    segs, tel, hist = workload(args.seed + 1000 * rank, per_shower=args.per_shower)
    n = len(segs["z0"])
    seg_base = rank * n
    n_sub = substeps(segs)
    arr = B.pack_segments(segs)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    det = B.Detector(n_showers=10, hist=hist, tel=tel)
    d_segs = torch.from_numpy(arr.view(np.uint8)).to(dev)
    hist_t = torch.zeros((10, 400, 400), dtype=torch.int64, device=dev)
    tel_c = torch.zeros((10, tel.shape[0]), dtype=torch.int64, device=dev)
    tel_t = torch.zeros((10, tel.shape[0]), dtype=torch.float64, device=dev)
    cnt = torch.zeros(8, dtype=torch.int64, device=dev)
    out = B.cs_output()
    out.hist, out.tel_counts, out.tel_time, out.counters = (hist_t.data_ptr(), tel_c.data_ptr(), tel_t.data_ptr(),
                                                            cnt.data_ptr())
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)
    o = B.cs_opts_default()
    o.bunch, o.device_ptrs, o.seg_base = bunch, 1, seg_base

    def step(accumulate=0, det_=det):
        o.accumulate = accumulate
        st = B.cs_propagate_ex(C.c_void_p(d_segs.data_ptr()), n, atm.handle, det_.handle, args.seed, o, out, sp)
        if st != B.CS_OK:
            raise B.CSError(st, "cs_propagate_ex")

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    photons_per_step = int(cnt[0].item())
    bunches_per_step = photons_per_step // bunch

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.5)   # let the sampler start before the timed region
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    ms_t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    assert int(cnt[0].item()) == photons_per_step
    photons_all_ranks = photons_per_step
    if world > 1:   # combined outputs of all shards (exact integer sums), outside the timed region
        from paper_2405_04229_gb300 import shard
        comb = [cnt.clone(), hist_t.clone(), tel_c.clone()]
        shard.reduce_counts(comb)
        pps = torch.tensor([photons_per_step], dtype=torch.int64, device=dev)
        torch.distributed.all_reduce(pps)
        photons_all_ranks = int(pps.item())
        assert int(comb[0][0].item()) == photons_all_ranks
    total_photons = photons_all_ranks * args.steps
    value = total_photons / (ms_max / 1e3)

    # kernel-only timing for the roofline: the same launch without the output memsets
    kstarts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        kstarts[k].record(stream)
        step(accumulate=1)
        kends[k].record(stream)
    torch.cuda.synchronize()
    k_ms = sum(s.elapsed_time(e) for s, e in zip(kstarts, kends)) / args.steps
    sm_clk = clk.summary()
    ops = OPS_PER_BUNCH_PLAN * bunches_per_step
    achieved = ops / (k_ms / 1e3) / 1e12
    ops_full = OPS_PER_BUNCH * bunches_per_step + OPS_PER_SUBSTEP * n_sub + OPS_PER_SEGMENT * n
    achieved_full = ops_full / (k_ms / 1e3) / 1e12
    max_mhz = 2070.0
    try:
        max_mhz = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", max_mhz)
    except Exception:
        pass
    n_sm = B.cs_device_sm_count()
    peak = n_sm * LANES_PER_SM * max_mhz * 1e6 / 1e12
    traffic, pipes = kernel_profile()

    # the surrogate form: the network replaces the table lookups inside its domain
    surrogate = None
    if not args.no_surrogate:
        t_tr = time.perf_counter()
        sur = B.Surrogate(atm, **({"epochs": args.surrogate_epochs} if args.surrogate_epochs else {}))
        train_s = time.perf_counter() - t_tr
        o.surrogate = sur.handle
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        s_photons = int(cnt[0].item())
        s_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a, b_ in s_ev:
            flush.zero_()
            a.record(stream)
            step()
            b_.record(stream)
        torch.cuda.synchronize()
        s_ms = sum(a.elapsed_time(b_) for a, b_ in s_ev)
        o.surrogate = None
        s_value = s_photons * args.steps / (s_ms / 1e3)
        surrogate = {"value": s_value, "unit": UNIT, "ms_per_step": s_ms / args.steps,
                     "speedup_vs_exact": s_value / (photons_per_step * args.steps / (ms_max / 1e3)),
                     "heldout_p99": {"displacement_m": sur.stats["p99"][0], "delay_s": sur.stats["p99"][1],
                                     "transmission": sur.stats["p99"][2]},
                     "heldout_max": {"displacement_m": sur.stats["max"][0], "delay_s": sur.stats["max"][1],
                                     "transmission": sur.stats["max"][2]},
                     "train_seconds": round(train_s, 2), "train_steps": sur.stats["steps"],
                     "network": "MLP 3-64-64-64-3 tanh on the fields less their first-order expansion in n - 1; BF16 "
                                "weights and activations (packed hardware tanh), FP32 accumulation in tensor memory "
                                "(tcgen05.mma M=128 per warpgroup)"}
        sur.close()

    optics = None
    if not args.no_optics:
        # last-mile ray tracing (Sec. 6.4): every telescope a 7 m parabolic mirror (f = 8 m) pointing
        # along the showers with a 1 m camera of 41 x 41 pixels; the same step with the trace on
        opt = dict(mirror_d=7.0, focal_f=8.0, camera_r=0.5, point_zenith=math.radians(20.0), point_azimuth=0.0,
                   cam_n=41)
        det_o = B.Detector(n_showers=10, hist=hist, tel=tel, optics=opt)
        cam_t = torch.zeros((10, tel.shape[0], 41, 41), dtype=torch.int64, device=dev)
        out.camera = cam_t.data_ptr()
        for _ in range(3):
            step(det_=det_o)
        torch.cuda.synchronize()
        o_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a, b_ in o_ev:
            flush.zero_()
            a.record(stream)
            step(det_=det_o)
            b_.record(stream)
        torch.cuda.synchronize()
        o_ms = sum(a.elapsed_time(b_) for a, b_ in o_ev) / args.steps
        optics = {"value": int(cnt[0].item()) / (o_ms / 1e3), "unit": UNIT, "ms_per_step": o_ms,
                  "time_vs_without": o_ms / (ms_max / args.steps),
                  "camera_photons": int(cam_t.sum().item()), "telescope_photons": int(tel_c.sum().item()),
                  "optics": "7 m parabolic mirror, f 8 m, 1 m camera, 41 x 41 pixels, pointing zenith 20 deg"}
        out.camera = None
        det_o.close()

    snell = None
    if not args.no_snell:
        # the general-atmosphere fallback: every photon traced through 10 m slabs with the
        # Snell vector stepper (Sec. 3.4.2, Eq. 3.15) instead of the table lookup; the thesis
        # times this method per photon on one CPU core (Table 4.2: 0.157 ms at 0 deg, 10 m steps)
        o.tracer, o.tracer_dh = B.CS_TRACER_SNELL, 10.0
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        k_snell = max(3, args.steps // 50)
        sn_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k_snell)]
        for a, b_ in sn_ev:
            flush.zero_()
            a.record(stream)
            step()
            b_.record(stream)
        torch.cuda.synchronize()
        sn_ms = sum(a.elapsed_time(b_) for a, b_ in sn_ev) / k_snell
        o.tracer = B.CS_TRACER_TABLES
        snell = {"value": int(cnt[0].item()) / (sn_ms / 1e3), "unit": UNIT, "ms_per_step": sn_ms, "steps": k_snell,
                 "time_vs_tables": sn_ms / (ms_max / args.steps),
                 "bunches_per_s": int(cnt[0].item()) / bunch / (sn_ms / 1e3),
                 "method": "Snell vector stepper, slabs <= 10 m, FP32, one traced path per bunch"}

    fluor = None
    if not args.no_fluorescence:
        # the second emission workload: nitrogen fluorescence (Eq. 2.6, Sec. 4.2.2) from the same
        # segments, isotropic into the downward half sphere, synthetic five-line list
        keep = B.set_fluorescence(o, dict(synth.FLUORESCENCE, half=True))   # noqa: F841
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        k_fl = max(3, args.steps // 10)
        fl_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k_fl)]
        for a, b_ in fl_ev:
            flush.zero_()
            a.record(stream)
            step()
            b_.record(stream)
        torch.cuda.synchronize()
        fl_ms = sum(a.elapsed_time(b_) for a, b_ in fl_ev) / k_fl
        fl_photons = int(cnt[0].item())
        o.emission = B.CS_EMIT_CHERENKOV
        fluor = {"value": fl_photons / (fl_ms / 1e3), "unit": UNIT, "ms_per_step": fl_ms, "steps": k_fl,
                 "photons_per_step": fl_photons, "bunches_per_s": fl_photons / bunch / (fl_ms / 1e3),
                 "emission": "nitrogen fluorescence, downward half sphere, 5 synthetic lines, dE/dX 2.2 MeV cm^2/g"}

    e2e = None
    if not args.no_e2e:
        # end to end through the host-pointer call: pinned segments in, outputs out
        seg_pin = torch.from_numpy(arr.view(np.uint8)).pin_memory()
        hist_h = torch.zeros((10, 400, 400), dtype=torch.int64).pin_memory()
        tel_h = torch.zeros((10, tel.shape[0]), dtype=torch.int64).pin_memory()
        tt_h = torch.zeros((10, tel.shape[0]), dtype=torch.float64).pin_memory()
        cnt_h = torch.zeros(8, dtype=torch.int64).pin_memory()
        rc_h = torch.zeros(1, dtype=torch.int64).pin_memory()
        oh = B.cs_output()
        oh.hist, oh.tel_counts, oh.tel_time, oh.counters, oh.record_count = (
            hist_h.data_ptr(), tel_h.data_ptr(), tt_h.data_ptr(), cnt_h.data_ptr(), rc_h.data_ptr())
        oo = B.cs_opts_default()
        oo.bunch, oo.seg_base = bunch, seg_base

        def hstep():
            st = B.cs_propagate_ex(C.c_void_p(seg_pin.data_ptr()), n, atm.handle, det.handle, args.seed, oo, oh, sp)
            if st != B.CS_OK:
                raise B.CSError(st, "cs_propagate_ex(host)")

        for _ in range(3):
            hstep()
        torch.cuda.synchronize()
        e2e_s = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            a = time.perf_counter()
            hstep()
            e2e_s += time.perf_counter() - a   # synchronous: copies in, kernel, copies out
        assert int(cnt_h[0].item()) == photons_per_step
        h2d = arr.nbytes
        d2h = hist_h.numel() * 8 + tel_h.numel() * 16 + 8 * 8 + 8
        e2e = {"value": photons_per_step * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_entry(segs, tel, hist)

    configs = None
    if world == 1 and not args.no_configs:
        configs = extra_configs(args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "segments_per_gpu": n, "bunch": bunch,
                       "bunches_per_step_per_gpu": bunches_per_step, "form": "exact tracer (tables)",
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": "dp%d (shards)" % world},
            "bunches_per_s": value / bunch,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "achieved_full_count": achieved_full, "frac_full_count": achieved_full / peak,
                         "ncu_pipes_pct": pipes,
                         "note": "achieved: %d planned FP32/INT lane ops per bunch x bunches per launch / launch "
                                 "time; *_full_count: the itemised count of the implemented formulas (%d per bunch "
                                 "+ %d per sub-step + %d per segment); peak = SMs x 128 lanes x max SM clock; "
                                 "ncu_pipes_pct: issue-slot and busiest-pipe utilisation from the committed capture"
                                 % (OPS_PER_BUNCH_PLAN, OPS_PER_BUNCH, OPS_PER_SUBSTEP, OPS_PER_SEGMENT)},
            "kernel_ms": k_ms,
            "cpu_baseline": cpu,
            "surrogate": surrogate,
            "optics": optics,
            "snell_tracer": snell,
            "fluorescence": fluor,
            "e2e": e2e,
            "gpu_launches": 2 * args.steps,   # the photon kernel and its exact pass, per step
            "clocks": sm_clk,
        }
        if configs:
            line.update(configs)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
