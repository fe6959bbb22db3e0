"""The multi-GPU path is replicas only (one independent coarsening per GPU;
the method has no exchange step to shard): bench.py's whole-job value is
every rank's units over the slowest rank's time.  That host-side reduction
runs here with the gloo backend, world size 2, on CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r took 1 + r seconds for 100 units: the job did 200 units in 2 s
        value = bench.replica_value(100, 1.0 + rank, ws)
        slowest = bench.max_over_ranks(0.5 * (rank + 1), ws)
        dist.barrier()
        out.put((rank, value, slowest))
    finally:
        dist.destroy_process_group()


def test_replica_value_takes_the_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(out.get(timeout=10) for _ in range(2))
    for rank, value, slowest in got:
        assert value == pytest.approx(100.0)  # 2 * 100 units / 2.0 s
        assert slowest == pytest.approx(1.0)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_value(50, 2.0, 1) == pytest.approx(25.0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
