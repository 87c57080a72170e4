"""The N > 1 host path of bench.py on CPU ranks (gloo, world size 2):
replicas only - no data-path collective; the job time is the slowest rank's
and the value sums the units of every rank; the reference arm runs on rank 0
only while the other ranks exit without work."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        times = [100.0 + 50.0 * rank, 300.0 - 10.0 * rank]  # rank 1 is the slow one on the first
        out, value = bench.aggregate_replicas(times, 1_000_000, 10, world)
        q.put(("agg", rank, out, value))
        args = type("A", (), dict(ref_sample=3000, warmup=3, steps=1))()
        res = bench.run_reference(args, rank, world)
        q.put(("ref", rank, None if res is None else res["value"], None))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = [q.get(timeout=10) for _ in range(4)]
    agg = {r: (o, v) for k, r, o, v in got if k == "agg"}
    ref = {r: o for k, r, o, _ in got if k == "ref"}
    for r in (0, 1):
        out, value = agg[r]
        assert out == [150.0, 300.0]                       # max over ranks, per timing
        assert value == pytest.approx(2 * 1_000_000 / (150.0 / 10 / 1e3))
    assert ref[1] is None and ref[0] is not None and ref[0] > 0
