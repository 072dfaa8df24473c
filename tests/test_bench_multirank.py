"""The multi-rank path of bench.py (replicas, max over ranks) with world_size 2 on CPU (gloo)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank 1 is slower: the job time is the max over ranks, the bytes are the sum over ranks
    total_ms = 100.0 if rank == 0 else 250.0
    v, ms = bench.job_value(1e9, total_ms, 10, world, dist, "cpu")
    out[rank] = (v, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_job_value_takes_max_time_and_sums_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        v, ms = out[r]
        assert ms == pytest.approx(25.0)           # 250 ms / 10 steps on the slowest rank
        assert v == pytest.approx(2 * 1e9 / 25e-3 / 1e9)
