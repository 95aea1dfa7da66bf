"""The allocation-free device call gives the regular device call's results.

cs_propagate_noalloc is for callers that cannot let the library allocate
device memory (a pool or arena owning the device, hosts that forbid
allocation after start-up).  Its only scratch is a counter in a statically
declared device array that every call reuses, so this test makes two calls in
a row and checks both against cs_propagate_ex with device pointers.  It runs
last and also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_04229_gb300 import binding as B
    from paper_2405_04229_gb300 import synth
    segs = synth.refraction_showers(n_showers=3, per_shower=20_000, seed=5)
    tel = synth.grid_telescopes()
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    det = B.Detector(n_showers=3, hist=synth.histogram_400(), tel=tel)
    dev = torch.device("cuda:0")
    d_segs = torch.from_numpy(B.pack_segments(segs).view(np.uint8)).to(dev)
    return torch, B, atm, det, d_segs, len(segs["z0"]), tel.shape[0], dev


def _call(env, fn, seed=9):
    torch, B, atm, det, d_segs, n, n_tel, dev = env
    hist = torch.zeros((3, 400, 400), dtype=torch.int64, device=dev)
    tel_counts = torch.zeros((3, n_tel), dtype=torch.int64, device=dev)
    tel_time = torch.zeros((3, n_tel), dtype=torch.float64, device=dev)
    counters = torch.zeros(8, dtype=torch.int64, device=dev)
    out = B.cs_output()
    out.hist, out.tel_counts, out.tel_time, out.counters = (hist.data_ptr(), tel_counts.data_ptr(),
                                                            tel_time.data_ptr(), counters.data_ptr())
    o = B.cs_opts_default()
    o.bunch, o.device_ptrs = 5, 1
    st = fn(C.c_void_p(d_segs.data_ptr()), n, atm.handle, det.handle, seed, o, out,
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == B.CS_OK, B.status_string(st)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in (hist, tel_counts, tel_time, counters)]


def test_noalloc_matches_device_call_twice(env):
    B = env[1]
    ref = _call(env, B.cs_propagate_ex)
    assert ref[3][0] > 0
    for _ in range(2):   # the second call reuses the scratch left by the first
        got = _call(env, B.cs_propagate_noalloc)
        for k in (0, 1, 3):   # integer counts: identical
            assert np.array_equal(got[k], ref[k])
        # per-telescope FP64 time sums: same terms, atomic summation order differs
        np.testing.assert_allclose(got[2], ref[2], rtol=1e-12)


def test_noalloc_rejects_host_pointers(env):
    torch, B, atm, det, d_segs, n, n_tel, dev = env
    out = B.cs_output()
    counters = np.zeros(8, np.uint64)
    out.counters = counters.ctypes.data
    o = B.cs_opts_default()
    o.device_ptrs = 0
    assert B.cs_propagate_noalloc(None, 0, atm.handle, det.handle, 0, o, out) == B.CS_ERR_INVALID_ARG
