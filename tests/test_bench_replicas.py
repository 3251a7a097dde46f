"""The multi-GPU form of bench.py is N independent replicas (the search does not shard): rank r
anneals with seed + r, the timed region ends with a barrier, and the job's rate is every rank's
work over the slowest rank's time.  These host pieces run here as two gloo ranks on the CPU."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank), BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    got_ws, got_rank, _ = bench.dist_setup()
    assert (got_ws, got_rank) == (ws, rank)
    bench.barrier(ws)
    # rank r "took" 1 + r seconds for 1000 units
    rate, t = bench.job_rate(1.0 + rank, 1000.0, ws)
    q.put((rank, rate, t, bench.replica_seed(240801470, rank)))
    import torch.distributed as dist
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_time_by_the_slowest_and_use_distinct_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ws, port = 2, 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, rate, t, seed in out:
        assert t == 2.0                       # the slowest rank's seconds, on every rank
        assert rate == pytest.approx(ws * 1000.0 / 2.0)
    assert [o[3] for o in out] == [240801470, 240801471]
