"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks, each with
its own timed region, agree on the slowest rank's time, and the whole-job
throughput counts every rank's replica (weak scaling).  No GPU."""
import os
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = 10.0 + 5.0 * rank                    # rank 1 is the slower one
    ms = bench.slowest_rank_ms(mine, dist, "cpu")
    q.put((rank, ms, bench.job_mps(262144, world, 20, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    # 2 ranks x 20 steps x 262144 pixels in 15 ms
    assert abs(res[0][2] - 2 * 20 * 262144 / 15e-3 / 1e6) < 1e-9
    assert res[0][2] == res[1][2]


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(12.5, None, "cpu") == 12.5
    assert abs(bench.job_mps(1000, 1, 4, 2.0) - 4 * 1000 / 2e-3 / 1e6) < 1e-12
