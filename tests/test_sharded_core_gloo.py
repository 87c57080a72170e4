"""Host logic of the sharded core phase on CPU ranks (gloo, world size 2).

Each rank takes its shard of Omega with shard_range, computes the shard's
core gradient (here with the FP64 oracle, standing in for ft_core_grad on a
GPU), and the ranks sum them with allreduce_core_grad.  Every rank must end
with the gradient over all of Omega, and a core step taken from it with
|Omega| must equal the oracle's core epoch over all of Omega - the identity
that lets Algorithm 5 run on shards (its gradient is a plain sum over the
nonzeros, taken from one fixed A and B).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2404_10087_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from paper_2404_10087_gb300 import synth
    I, J, R, nnz = (9, 11, 13), (3, 4, 2), 3, 257
    idx, x, A, B = synth.random_problem(31, I, J, R, nnz)
    return (idx.numpy(), x.double().numpy(), [a.double().numpy() for a in A],
            [b.double().numpy() for b in B])


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        idx, x, A, B = _problem()
        lo, hi = shard.shard_range(x.size, rank, world)
        Gs = oracle.core_grad(A, B, idx[:, lo:hi], x[lo:hi])
        G = torch.from_numpy(np.concatenate([g.ravel() for g in Gs]))
        shard.allreduce_core_grad(G)
        q.put((rank, lo, hi, G.numpy().copy()))
    finally:
        dist.destroy_process_group()


def test_shard_ranges_cover_once():
    for nnz in (0, 1, 2, 3, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            ranges = [shard.shard_range(nnz, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == nnz
            for (lo, hi), (lo2, _) in zip(ranges, ranges[1:]):
                assert hi == lo2
            sizes = [hi - lo for lo, hi in ranges]
            assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1
    for bad in ((5, 2, 2), (5, -1, 2), (5, 0, 0), (-1, 0, 1)):
        with pytest.raises(ValueError):
            shard.shard_range(*bad)


def test_allreduce_without_a_group_leaves_the_gradient():
    G = torch.arange(6, dtype=torch.float32)
    assert torch.equal(shard.allreduce_core_grad(G.clone()), G)


def test_two_cpu_ranks_sum_to_the_full_gradient():
    import oracle
    oracle.build()  # once, before the ranks load it
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    idx, x, A, B = _problem()
    full = np.concatenate([g.ravel() for g in oracle.core_grad(A, B, idx, x)])
    assert got[0][1:3] == (0, 128) and got[1][1:3] == (128, 257)
    for _, _, _, G in got:
        np.testing.assert_allclose(G, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    # the step from the summed gradient is the core epoch over all of Omega
    lr, lam = 0.4, 0.03
    ref = oracle.core_epoch(A, B, idx, x, lr, lam)
    off = 0
    for n, b in enumerate(B):
        g = got[0][3][off:off + b.size].reshape(b.shape)
        off += b.size
        np.testing.assert_allclose(b - lr * (g / x.size + lam * b), ref[n], rtol=1e-12, atol=1e-14)
