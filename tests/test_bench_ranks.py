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


def test_serving_summary_censors_unfinished_requests():
    """The serving figures: p50 / p99 over every submitted request, an unfinished one counted at the end of the run
    (its latency is at least that), the completed-only figures beside them, and the offered and sustained load."""
    import bench
    done = {1: {"status": 0, "steps": 10, "t_submit": 0.0, "t_done": 1.0},
            2: {"status": 0, "steps": 20, "t_submit": 1.0, "t_done": 4.0},
            3: {"status": 5, "steps": 5, "t_submit": 2.0, "t_done": 2.5}}
    tickets = [1, 2, 3, 4, 5]
    sub_t = {1: 0.0, 2: 1.0, 3: 2.0, 4: 3.0, 5: 9.0}
    sub_work = [100, 200, 300, 400, 500]
    out = bench.serving_summary(done, tickets, sub_t, sub_work, elapsed=10.0, window_s=5.0)
    # latencies 1, 3, 0.5 (finished) and 10 - 3 = 7, 10 - 9 = 1 (censored)
    assert out["submitted"] == 5 and out["completed"] == 3 and out["converged"] == 2
    assert out["p50_s"] == 1.0 and abs(out["p99_s"] - (3 + 0.96 * 4)) < 1e-12
    assert out["p50_completed_s"] == 2.0            # the converged ones: 1 and 3
    assert out["completion_fraction"] == 0.6
    assert out["offered_pairs_per_s"] == 1500 / 5.0
    assert out["sustained_pairs_per_s"] == (100 * 10 + 200 * 20 + 300 * 5) / 10.0
    assert out["configs_per_hour"] == 2 / 10.0 * 3600.0
