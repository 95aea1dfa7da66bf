"""The surrogate's bounded tensor-core waits, made to give up on purpose.

Every wait of the network on a tcgen05 completion polls its mbarrier a
bounded number of times.  With the poll limit set below zero the first wait
of every warpgroup gives up at once: no GPU fault, hang or trap is involved,
the MMAs already issued finish and are waited for (at the normal bound)
before the tensor memory is freed.  The warpgroup then stops using the
network, so every photon takes the correction tables: the counts equal the
exact tracer's bit for bit, and the call reports CS_ERR_TIMEOUT."""
import ctypes as C

import numpy as np
import pytest

from paper_2405_04229_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_04229_gb300 import binding
    return binding


def test_wait_that_gives_up_falls_back_to_the_tables(B):
    segs = synth.refraction_showers(n_showers=1, per_shower=3000, seed=12)
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    det = B.Detector(n_showers=1, hist=synth.histogram_400(), tel=synth.grid_telescopes())
    sur = B.Surrogate(atm, epochs=2, n_train=1 << 16, n_heldout=1 << 12)
    tables = B.propagate_host(segs, atm, det, seed=4, bunch=5)
    gave_up = B.propagate_host(segs, atm, det, seed=4, bunch=5, surrogate=sur, tc_poll_limit=-1, allow_timeout=True)
    assert gave_up["status"] == B.CS_ERR_TIMEOUT
    for k in ("hist", "tel_counts", "counters"):
        assert np.array_equal(gave_up[k], tables[k]), k
    assert int(tables["counters"][B.CS_CNT_TEL]) > 0
    # the flag was read and cleared: the next call uses the network and succeeds
    normal = B.propagate_host(segs, atm, det, seed=4, bunch=5, surrogate=sur)
    assert normal["status"] == B.CS_OK
    assert np.array_equal(normal["counters"][:1], tables["counters"][:1])   # the same bunches are emitted
    # device-pointer calls report through cs_check_timeout
    torch = pytest.importorskip("torch")
    arr = B.pack_segments(segs)
    d_segs = torch.from_numpy(arr.view(np.uint8)).cuda()
    outs = B.DeviceOutputs(det)
    o = B.cs_opts_default()
    o.bunch, o.device_ptrs, o.surrogate, o.tc_poll_limit = 5, 1, sur.handle, -1
    st = B.cs_propagate_ex(C.c_void_p(d_segs.data_ptr()), len(arr), atm.handle, det.handle, 4, o, outs.out,
                           B.stream_ptr())
    assert st == B.CS_OK                                   # enqueued; the give-up is reported later
    assert B.cs_check_timeout() == B.CS_ERR_TIMEOUT
    assert B.cs_check_timeout() == B.CS_OK                 # cleared by the first check
    dev = outs.host()
    for k in ("hist", "tel_counts", "counters"):
        assert np.array_equal(dev[k], tables[k]), k
    sur.close()
