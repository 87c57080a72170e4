"""Algorithm 5 in two halves - the gradient (ft_core_grad) and the step
(ft_core_apply) - and over shards of Omega, through the C ABI.

* gradient then step on one context equals ft_epoch_core bit for bit (the
  step is the finalize's arithmetic on the same float32 gradient);
* the shards' gradients, summed, equal the FP64 oracle's gradient over all
  of Omega, and the step from that sum with |Omega| equals the oracle's core
  epoch, at the core-gradient tolerances of the parity tests (FP32 1e-5,
  BF16 2e-2, Frobenius, on the step B_new - B_old);
* shard_range splits ragged sizes, empty shards included;
* epoch_core_sharded without a process group is ft_epoch_core.
The sum over processes is the collective's job; here, on one GPU, the
shards' gradients are added in the test, and the collective itself is
covered by the two-process CPU test of the same helpers.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2404_10087_gb300 import ft, shard, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL_GRAD = {"fp32": 1e-5, "bf16": 2e-2}
SHAPE = ((60, 70, 80), (16, 16, 16), 16)


def f64(ts):
    return [t.detach().double().cpu().numpy() for t in ts]


def rel_fro(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / d) if d > 0 else float(np.linalg.norm(got))


def dev_copy(idx, x, A, B, lo=0, hi=None):
    hi = int(x.numel()) if hi is None else hi
    return ([idx[n][lo:hi].contiguous().to(DEV) for n in range(idx.shape[0])],
            x[lo:hi].contiguous().to(DEV), [a.clone().to(DEV) for a in A],
            [b.clone().to(DEV) for b in B])


def flat_grad(m):
    return torch.cat([g.reshape(-1) for g in m.core_grad()])


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_grad_then_apply_is_the_core_epoch_bitwise(precision):
    I, J, R = SHAPE
    idx, x, A, B = synth.random_problem(21, I, J, R, 5003)
    lr, lam = 0.5, 0.01
    a = ft.FastTuckerPlus(*dev_copy(idx, x, A, B), precision=precision)
    a.epoch_core(lr, lam)
    b = ft.FastTuckerPlus(*dev_copy(idx, x, A, B), precision=precision)
    b.core_apply(flat_grad(b), b.nnz, lr, lam)
    torch.cuda.synchronize()
    for n in range(3):
        assert torch.equal(a.B[n], b.B[n]), n


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("nnz,world", [(5003, 2), (5003, 3), (1, 2)])
def test_shard_gradients_sum_to_the_full_core_step(precision, nnz, world):
    I, J, R = SHAPE
    idx, x, A, B = synth.random_problem(22, I, J, R, nnz)
    lr, lam = 0.5, 0.01
    gA = [a.clone().to(DEV) for a in A]
    gB = [b.clone().to(DEV) for b in B]
    models, G = [], None
    for r in range(world):
        lo, hi = shard.shard_range(nnz, r, world)
        sidx, sx, _, _ = dev_copy(idx, x, A, B, lo, hi)
        m = ft.FastTuckerPlus(sidx, sx, gA, gB, precision=precision)  # shared A, B: read only
        g = flat_grad(m)
        G = g if G is None else G + g
        models.append(m)
    torch.cuda.synchronize()
    ref_G = oracle.core_grad(f64(A), f64(B), idx.numpy(), x.double().numpy())
    off = 0
    for n in range(3):
        got = G[off:off + J[n] * R].view(J[n], R).double().cpu().numpy()
        off += J[n] * R
        assert rel_fro(got, ref_G[n]) <= TOL_GRAD[precision], n
    models[0].core_apply(G, nnz, lr, lam)
    ref_B = oracle.core_epoch(f64(A), f64(B), idx.numpy(), x.double().numpy(), lr, lam)
    got_B, B0 = f64(gB), f64(B)
    for n in range(3):
        assert rel_fro(got_B[n] - B0[n], ref_B[n] - B0[n]) <= TOL_GRAD[precision], n
    for m in models:
        m.check()


def test_sharded_epoch_without_a_group_is_the_core_epoch():
    I, J, R = SHAPE
    idx, x, A, B = synth.random_problem(23, I, J, R, 777)
    a = ft.FastTuckerPlus(*dev_copy(idx, x, A, B), precision="fp32")
    a.epoch_core(0.3, 0.02)
    b = ft.FastTuckerPlus(*dev_copy(idx, x, A, B), precision="fp32")
    s = torch.cuda.Stream()
    shard.epoch_core_sharded(b, 0.3, 0.02, b.nnz, stream=s)
    s.synchronize()
    torch.cuda.synchronize()
    for n in range(3):
        assert torch.equal(a.B[n], b.B[n]), n


def test_apply_rejects_bad_arguments():
    I, J, R = SHAPE
    idx, x, A, B = synth.random_problem(24, I, J, R, 50)
    m = ft.FastTuckerPlus(*dev_copy(idx, x, A, B))
    G = torch.zeros(sum(J) * R, dtype=torch.float32, device=DEV)
    with pytest.raises(ft.FtError):
        ft.ft_core_apply(m.ctx, G, -1, 0.1, 0.1)
    with pytest.raises(ft.FtError):
        ft.ft_core_apply(m.ctx, G, 50, math.inf, 0.1)
    with pytest.raises(ValueError):
        m.core_apply(G[:-1], 50, 0.1, 0.1)
    B0 = [b.clone() for b in m.B]
    m.core_apply(G, 0, 0.1, 0.5)          # zero gradient, no data: only the decay acts
    for b, b0 in zip(m.B, B0):
        torch.testing.assert_close(b, b0 * (1 - 0.1 * 0.5), rtol=1e-6, atol=1e-7)
