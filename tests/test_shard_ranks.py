"""Particle shards of one configuration on CPU ranks (gloo): the partition, the exchanges of ShardGroup through
torch.distributed, and a rank that leaves between steps.

The shard contexts here are the CPU stand-in of shard_fake.py, which keeps the exchange contract of the library's
shards (exact integer density partials, dot products per 2048-particle chunk, each shard moving only its own
particles).  A configuration split over two ranks, or over three shards in one process, must give the same bits as
one shard holding every particle: Phi, S_max, every force and every position after FIRE steps.
"""
import datetime
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

N, D, STEPS = 5000, 2, 12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _config():
    from paper_2304_09139_b300 import synth
    s = synth.positions(123, N, D)
    L = math.sqrt(N)
    n = np.array([(a, b) for a in range(0, 6) for b in range(-5, 6) if (a > 0 or b > 0) and a * a + b * b <= 25])
    return s, n, L


def _alloc(n, kind):
    return torch.zeros(n, dtype=torch.int64 if kind == "i64" else torch.float64)


def _run(shards, comm=None):
    from paper_2304_09139_b300.shard import ShardGroup
    g = ShardGroup(shards, comm=comm, alloc=_alloc, pointer=lambda t: t)
    g.eval(True)
    first = [(sh.phi, sh.smax, sh.F[sh.loc].copy()) for sh in shards]
    g.fire_begin(dt0=0.02)
    g.steps(STEPS)
    return first, g.state(), [sh.s[sh.loc].copy() for sh in shards]


def _whole():
    from shard_fake import FakeShard
    s, n, L = _config()
    return _run([FakeShard(s, n, L, 0, N)])


def test_shard_ranges_align_and_cover():
    from paper_2304_09139_b300.shard import shard_ranges
    for n_, g in [(5000, 2), (10_000, 3), (2_000_000, 8), (4096, 2), (2049, 2)]:
        r = shard_ranges(n_, g)
        assert len(r) == g and r[0][0] == 0 and sum(c for _, c in r) == n_
        for (f0, c0), (f1, _) in zip(r, r[1:]):
            assert f0 + c0 == f1 and f1 % 2048 == 0 and c0 % 2048 == 0 and c0 > 0
    with pytest.raises(ValueError):
        shard_ranges(3000, 3)


def test_three_shards_in_one_process_equal_one():
    from paper_2304_09139_b300.shard import shard_ranges
    from shard_fake import FakeShard
    s, n, L = _config()
    ref_first, ref_state, ref_pos = _whole()
    shards = [FakeShard(s, n, L, f, c) for f, c in shard_ranges(N, 3)]
    first, state, pos = _run(shards)
    assert ref_state == state
    for (phi, smax, F), sh in zip(first, shards):
        assert phi == ref_first[0][0] and smax == ref_first[0][1]
        assert np.array_equal(F, ref_first[0][2][sh.loc])
    assert np.array_equal(np.concatenate(pos), ref_pos[0])


def _rank_main(rank, world, port, out, leave_early):
    import torch.distributed as dist
    from paper_2304_09139_b300.shard import ShardGroup, TorchComm, shard_ranges
    from shard_fake import FakeShard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    s, n, L = _config()
    f, c = shard_ranges(N, world)[rank]
    sh = FakeShard(s, n, L, f, c)
    if not leave_early:
        first, state, pos = _run([sh], comm=TorchComm())
        out[rank] = (f, c, first[0][0], first[0][1], first[0][2], state, pos[0])
        dist.barrier()
        dist.destroy_process_group()
        return
    g = ShardGroup([sh], comm=TorchComm(), alloc=_alloc, pointer=lambda t: t)
    g.fire_begin(dt0=0.02)
    if rank == 1:
        out[rank] = "left between steps"
        os._exit(0)        # no destroy: the process is gone, as after a crash between steps
    try:
        g.steps(STEPS)
        out[rank] = "finished"
    except Exception as e:  # the next exchange reports the missing rank
        out[rank] = f"error: {type(e).__name__}"


def test_two_ranks_equal_one_shard_bit_for_bit():
    world = 2
    ref_first, ref_state, ref_pos = _whole()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out, False), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        f, c, phi, smax, F, state, pos = res[rank]
        assert phi == ref_first[0][0] and smax == ref_first[0][1]
        assert np.array_equal(F, ref_first[0][2][f:f + c])
        assert state == ref_state
        assert np.array_equal(pos, ref_pos[0][f:f + c])


def test_rank_leaving_between_steps_is_reported():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        ctx = mp.start_processes(_rank_main, args=(world, _free_port(), out, True), nprocs=world, join=False,
                                 start_method="spawn")
        for p in ctx.processes:
            p.join(120)
        res = dict(out)
    assert res[1] == "left between steps"
    assert res[0].startswith("error"), res[0]
