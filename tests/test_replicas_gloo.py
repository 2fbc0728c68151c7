"""The multi-GPU form of the bench is replicas: every rank steps its own
lattice, the ranks meet at a barrier around the timed region, the job's time
is the slowest rank's and the whole-job rate counts the units of all ranks.
Two gloo ranks on the CPU run that logic with bench.py's own helpers."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        dist.barrier()
        local_ms = 10.0 * (rank + 1)           # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, dist, device="cpu")
        rate = bench.whole_job_rate(1000.0, ms * 1e-3, world)
        q.put((rank, local_ms, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_the_whole_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [10.0, 20.0]
    for rank, local, ms, rate in got:
        assert ms == 20.0                            # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 1000.0 / 0.020)  # both ranks' units over that time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, None, device="cpu") == 3.5
    assert bench.whole_job_rate(100.0, 2.0, 1) == 50.0
