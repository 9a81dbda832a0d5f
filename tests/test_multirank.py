"""The N > 1 bench path on CPU: two gloo ranks (replicas only, no data-path collective).

The bench times each rank, takes the slowest rank's time (all_reduce MAX) and reports the
whole job's site updates over it; the reference arm runs on rank 0 only.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(local_ms, world, "cpu")
        value = bench.job_glups(world, 1_000_000, 100, slowest * 1e-3)
        w, r, _ = bench.dist_setup()
        ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 3, "ref_budget": 1.0})()) if r != 0 else None
        out.put((rank, slowest, value, w, r, ref))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value, w, r, ref in res:
        assert w == 2 and r == rank
        assert slowest == pytest.approx(15.0)  # both ranks see the slowest rank's time
        # 2 ranks x 1e6 sites x 100 steps / 15 ms
        assert value == pytest.approx(2 * 1e6 * 100 / 15e-3 / 1e9)
    assert res[1][5] is None  # the reference arm does no work on rank 1
