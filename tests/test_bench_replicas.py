"""The multi-GPU path of bench.py runs independent replicas (the method is not partitioned here):
each rank times its own V-cycles, the job time is the largest over the ranks and the value counts
the cells of every replica.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    ms = 100.0 + 25.0 * rank  # rank 1 is the slower replica
    ms_max = bench.reduce_max(ms, w, "cpu")
    out[rank] = (r, w, lr, ms_max, bench.job_rate(1000, 10, ms_max, w))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_all_cells():
    ctx = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for rank in (0, 1):
        r, w, lr, ms_max, rate = res[rank]
        assert (r, w, lr) == (rank, 2, rank)
        assert ms_max == 125.0
        assert rate == pytest.approx(2 * 1000 * 10 / 0.125 / 1e6)
