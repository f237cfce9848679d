"""The N>1 path of bench.py on CPU ranks (gloo, world size 2): replicas with their own draws, the
slowest rank's time, and the whole-job value; the reference arm does no work on ranks other than 0."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, loc = bench.dist_info()
    local_ms = 10.0 + 7.5 * rank                       # rank 1 is the slow one
    tot = bench.max_over_ranks(local_ms, dist)
    seed = bench.replica_seed(2, r)
    seeds = [None] * w
    dist.all_gather_object(seeds, seed)
    dist.barrier()
    out[rank] = (r, w, tot, tuple(seeds), bench.job_value(1000, w, 4, tot))
    dist.destroy_process_group()


def test_two_rank_timing_and_replicas():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        r, w, tot, seeds, value = res[rank]
        assert (r, w) == (rank, world)
        assert tot == 17.5                              # max over ranks, the same on every rank
        assert seeds == (2, 3)                          # each replica draws its own configuration
        assert value == pytest.approx(1000 * 2 * 4 / 17.5e-3)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "cpu_sample", lambda *a, **k: called.append(1))
    class A:
        steps, warmup = 2, 1
    assert bench.run_reference(A()) == 0
    assert not called
