"""The multi-GPU path is replicas only (one independent frame per rank); its host logic runs
here as world-size-2 gloo process groups on the CPU: the slowest rank's time decides, the
job rate counts every rank's frames, and the reference arm runs on rank 0 alone."""
import io
import os
import socket
from contextlib import redirect_stdout
from types import SimpleNamespace

import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, world, "cpu")   # rank 1 is the slow one
    rate = bench.job_rate(world, 20, ms)
    buf = io.StringIO()
    with redirect_stdout(buf):
        if rank != 0:   # the reference arm: ranks other than 0 return without work or output
            bench.run_reference(SimpleNamespace(ref_tiles=1, warmup=0, steps=1), rank, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, rate, buf.getvalue()))


def test_replica_timing_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, printed in out:
        assert ms == 150.0                         # max over ranks
        assert abs(rate - 2 * 20 / 0.150) < 1e-9   # frames of both ranks over the slowest time
    assert out[1][3] == ""


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_rate(1, 10, 500.0) == 20.0
