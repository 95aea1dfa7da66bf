"""Multi-rank path with the CUDA propagator: two ranks (processes) each run the
library on their contiguous share of the segments with global segment ids,
and reduce their outputs over gloo; the sums equal one call over all
segments -- counts bit for bit, the FP64 time sums to a relative 1e-12.
Both ranks use the one visible GPU; their kernels are independent (no rank
waits on another's kernel), and only host tensors enter the collective."""
import os
import socket

import numpy as np
import pytest

from paper_2405_04229_gb300 import shard, synth

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _inputs():
    return synth.refraction_showers(n_showers=3, per_shower=20_000, seed=21)


def _propagate(segs, a, b):
    from paper_2405_04229_gb300 import binding as B
    atm = B.Atmosphere(layered=synth.US_STANDARD, refraction=True, transmission=True)
    det = B.Detector(n_showers=3, hist=synth.histogram_400(), tel=synth.grid_telescopes())
    r = B.propagate_host(synth.take(segs, slice(a, b)), atm, det, seed=4, bunch=5, seg_base=a)
    atm.close()
    det.close()
    return r


def _rank(rank, world, port, out_q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    segs = _inputs()
    a, b = shard.shard_range(len(segs["z0"]), rank, world)
    r = _propagate(segs, a, b)
    t = [torch.from_numpy(r["hist"].astype(np.int64)), torch.from_numpy(r["tel_counts"].astype(np.int64)),
         torch.from_numpy(r["counters"].astype(np.int64)), torch.from_numpy(r["tel_time"].copy())]
    shard.reduce_counts(t)
    if rank == 0:
        out_q.put([x.numpy() for x in t])
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_of_the_cuda_path_reduce_to_one_call():
    import torch.multiprocessing as mp
    import __graft_entry__
    __graft_entry__.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=600)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    segs = _inputs()
    ref = _propagate(segs, 0, len(segs["z0"]))
    assert int(ref["counters"][3]) > 0
    assert np.array_equal(got[0], ref["hist"].astype(np.int64))
    assert np.array_equal(got[1], ref["tel_counts"].astype(np.int64))
    assert np.array_equal(got[2], ref["counters"].astype(np.int64))
    np.testing.assert_allclose(got[3], ref["tel_time"], rtol=1e-12)
