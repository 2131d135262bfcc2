"""Multi-rank logic of bench.py on CPU ranks (gloo, world size 2): every rank runs
its own problem, the reported time is the slowest rank's, the whole-job rate
counts all ranks' bytes, and only rank 0 prints.  No GPU is used."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_info()
    assert (ws, r, local) == (world, rank, rank)
    # each rank's own "step time": the slowest must be reported everywhere
    ms = 10.0 + 5.0 * rank
    bench.rank_barrier()
    slowest = bench.max_over_ranks(ms)
    rate = bench.whole_job_rate(1e9, 4, ws, slowest)
    out[rank] = (slowest, rate)
    dist.destroy_process_group()


def test_two_gloo_ranks_report_slowest_and_whole_job_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        slowest, rate = out[r]
        assert slowest == 15.0
        # 2 ranks x 1 GB x 4 steps in 15 ms
        assert abs(rate - 2 * 1e9 * 4 / 15e-3 / 1e9) < 1e-9


def test_single_process_without_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    bench.rank_barrier()
    assert bench.whole_job_rate(2e9, 10, 1, 1000.0) == 20.0
