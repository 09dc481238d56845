"""The replicas path of bench.py (one independent grid per rank, no
data-path collective) across processes: world size 2 over gloo on the host.
The ranks' timings are combined by the slowest rank, the whole-job
throughput counts every rank's cells, and the reference arm runs on rank 0
only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier_ranks()
        ms = bench.max_over_ranks(torch, 10.0 + 5.0 * rank)  # rank 1 is slower
        value = bench.replica_throughput(world, 1000, 2, 4, ms)
        ref = bench.reference_arm(bench.argparse.Namespace(scheme="cgks5", steps=1, warmup=0,
                                                           gpus=world), rank) if rank else None
        q.put((rank, ms, value, ref))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_every_rank():
    torch = pytest.importorskip("torch")
    import torch.distributed as dist
    if not dist.is_available():
        pytest.skip("torch.distributed not built")
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    for rank, ms, value, ref in out:
        assert ms == 15.0                      # max over the ranks
        assert value == 2 * 1000 * 2 * 4 / 15e-3
        assert ref is None                     # only rank 0 runs the reference arm
