"""The bench's multi-rank aggregation on CPU with the gloo backend, world size 2: every rank
runs an independent replica; the job's throughput is all ranks' units over the slowest rank's
time (max over ranks)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
    value, ms = bench.job_throughput(ms_local, 1000, dist, "cpu")
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_uses_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        value, ms = res[r]
        assert ms == 150.0
        assert value == pytest.approx(2 * 1000 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    value, ms = bench.job_throughput(200.0, 500)
    assert ms == 200.0 and value == pytest.approx(500 / 0.2)
