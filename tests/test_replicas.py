"""Multi-GPU runs are replicas (independent k-point sequences, one per GPU, no collective on
the data path).  The host-side aggregation bench.py uses -- problems summed over ranks,
time the maximum over ranks -- checked with world_size 2 over gloo on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def worker(rank, world, port, out):
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [1500.0, 2500.0][rank]          # rank 1 is the slowest
    problems_local = [40, 40][rank]
    ms, problems, value = bench.aggregate_replicas(ms_local, problems_local, "cpu")
    out.put((rank, ms, problems, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, problems, value in res:
        assert ms == 2500.0 and problems == 80
        assert value == pytest.approx(80 / 2.5)


def test_single_process_aggregation():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ms, problems, value = bench.aggregate_replicas(1000.0, 20, "cpu")
    assert (ms, problems) == (1000.0, 20) and value == pytest.approx(20.0)
