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


def test_bench_names_the_single_rhs_kernels_and_their_traffic_evidence():
    """The roofline line names the kernels the autotuner chose and reports a DRAM-traffic ratio only
    for a kernel whose ncu capture it comes from."""
    import bench

    names, ratio, _ = bench.single_rhs_kernels([8, 5, 5, 4])
    assert names == "stage1_kernel<4>" and ratio == bench.TRAFFIC_RATIO
    names, ratio, _ = bench.single_rhs_kernels([4, 10, 16])
    assert set(names.split(" + ")) == {"stage1_kernel<4>", "stage1_bulk_kernel", "stage1_kernel<8>"}
    assert ratio is None
    assert bench.single_rhs_kernels([9, 11])[1] == bench.BULK_TRAFFIC_RATIO
