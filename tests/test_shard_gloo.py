"""Multi-rank path on CPU: two gloo ranks each propagate their contiguous
share of the segments (with global segment ids) and reduce the integer
outputs; the result equals one process over all segments, bit for bit.
The per-rank compute here is the oracle (this host has no GPU); the sharding
and the reduction are the code under test."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2405_04229_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, segs, out_q):
    import torch.distributed as dist

    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = len(segs["z0"])
    a, b = shard.shard_range(n, rank, world)
    atm = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
    r = oracle.propagate(synth.take(segs, slice(a, b)), atm, hist=synth.histogram_400(), tel=synth.grid_telescopes(),
                         bunch=5, refraction=True, transmission=True, seed=3, seg_base=a, n_showers=2, records=False)
    t = [torch.from_numpy(r["hist"].astype(np.int64)), torch.from_numpy(r["tel_counts"].astype(np.int64)),
         torch.from_numpy(r["counters"].astype(np.int64))]
    shard.reduce_counts(t)
    if rank == 0:
        out_q.put([x.numpy() for x in t])
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_partition():
    for n in (0, 1, 7, 1000, 1001):
        for w in (1, 2, 3, 8):
            rs = [shard.shard_range(n, r, w) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(w - 1))
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


def test_two_gloo_ranks_reduce_equals_single_run():
    import oracle
    segs = synth.refraction_showers(n_showers=2, per_shower=120, seed=5)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, segs, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    atm = oracle.make_atm(oracle.ATM_LAYERED, layered=synth.US_STANDARD)
    ref = oracle.propagate(segs, atm, hist=synth.histogram_400(), tel=synth.grid_telescopes(), bunch=5,
                           refraction=True, transmission=True, seed=3, n_showers=2, records=False)
    assert np.array_equal(got[0], ref["hist"].astype(np.int64))
    assert np.array_equal(got[1], ref["tel_counts"].astype(np.int64))
    assert np.array_equal(got[2], ref["counters"].astype(np.int64))
