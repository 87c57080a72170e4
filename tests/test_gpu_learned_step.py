"""Learned per-row step sizes on the GPU against the FP64 oracle, and the
A/B test of the learned step against the plain method.

Tolerances: row features <= 1e-4 and line-search labels <= 1e-3 relative
(FP32 with atomic accumulation); network outputs <= 1e-4 and gradients
<= 1e-4 (Frobenius) relative to the oracle evaluated on the same BF16
weights (FP32 accumulation on the GPU).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_10087_gb300 import ft, learned_step, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def f64(ts):
    return [t.detach().double().cpu().numpy() for t in ts]


def test_row_stats_match_oracle():
    I, J, R, nnz = (50, 60, 70), (16, 12, 16), 16, 3000
    idx, x, A, B = synth.random_problem(31, I, J, R, nnz)
    gidx = [idx[n].contiguous().to(DEV) for n in range(3)]
    gA = [a.to(DEV) for a in A]
    gB = [b.to(DEV) for b in B]
    m = ft.FastTuckerPlus(gidx, x.to(DEV), gA, gB)
    rows = sum(I)
    g = torch.Generator().manual_seed(3)
    ema0 = torch.rand(rows, generator=g)
    ema = ema0.clone().to(DEV)
    feat = torch.empty(rows, 3, device=DEV)
    lab = torch.empty(rows, device=DEV)
    lam, lr, beta = 0.05, 0.02, 0.7
    ft.ft_row_stats(m.ctx, lam, lr, beta, ema, feat, lab)
    of, ol = oracle.row_stats(f64(A), f64(B), idx.numpy(), x.double().numpy(), lam, lr, beta,
                              ema0.double().numpy())
    gf = feat.double().cpu().numpy()
    assert np.allclose(gf[:, 0], of[:, 0], rtol=1e-6, atol=0)
    assert np.allclose(gf[:, 1], of[:, 1], rtol=1e-4, atol=1e-6)
    assert np.allclose(gf[:, 2], of[:, 2], rtol=1e-4, atol=1e-5)
    assert np.allclose(lab.double().cpu().numpy(), ol, rtol=1e-3, atol=0)
    # the running average is updated in place: ema = beta ema0 + (1 - beta) |g| / count
    assert np.allclose(ema.double().cpu().numpy(), np.expm1(of[:, 1]), rtol=1e-4, atol=1e-6)


def test_stepnet_forward_and_gradient_match_oracle():
    net = ft.new_stepnet(DEV, seed=11)
    g = torch.Generator().manual_seed(5)
    X = torch.randn(1000, 3, generator=g) * torch.tensor([1.5, 0.8, 1.0]) + torch.tensor([2.0, 0.3, 0.0])
    y = torch.rand(1000, generator=g) * 3.75 + 0.25
    Xd, yd = X.contiguous().to(DEV), y.contiguous().to(DEV)
    P = ft.ft_stepnet_get(net, 1).astype(np.float64)       # the BF16 weights the kernels use
    s = torch.empty(1000, device=DEV)
    ft.ft_stepnet_forward(net, Xd, s)
    want = oracle.mlp_forward(P, X.double().numpy())
    np.testing.assert_allclose(s.double().cpu().numpy(), want, rtol=1e-4)
    loss = ft.ft_stepnet_train(net, Xd, yd, lr=0.0, steps=1)   # lr 0: only the gradient
    G = ft.ft_stepnet_get(net, 2).astype(np.float64)
    OG, oloss = oracle.mlp_grad(P, X.double().numpy(), y.double().numpy())
    assert abs(loss - oloss) <= 1e-5 * oloss
    assert np.linalg.norm(G - OG) <= 1e-4 * np.linalg.norm(OG)
    np.testing.assert_array_equal(ft.ft_stepnet_get(net, 1), P.astype(np.float32))


def test_stepnet_training_reduces_loss():
    net = ft.new_stepnet(DEV, seed=12)
    g = torch.Generator().manual_seed(6)
    X = torch.randn(4096, 3, generator=g)
    y = torch.clamp(1.0 + 0.8 * X[:, 0] - 0.5 * X[:, 2], 0.25, 4.0)
    curve = learned_step.train(net, X.contiguous().to(DEV), y.contiguous().to(DEV), steps=300, lr=3e-3)
    assert curve[-1] < 0.25 * curve[0], curve


def planted():
    w = synth.WORKLOADS["planted_uniform_1e5"]
    d = synth.draw_workload(w)
    pl = oracle.predict(f64(d.planted_A), f64(d.planted_B), d.idx.numpy())
    x = (torch.from_numpy(pl) + d.noise.double()).float()
    tri = [d.idx[n, d.train].contiguous().to(DEV) for n in range(3)]
    tei = [d.idx[n, d.test].contiguous().to(DEV) for n in range(3)]
    return w, tri, tei, x[d.train].contiguous().to(DEV), x[d.test].contiguous().to(DEV)


def test_learned_step_reaches_plain_rmse_sooner():
    """The planted 3-order workload (1e5 uniform coordinates, planted J = R = 4,
    noise 0.1) with eta = lambda = 0.01 for factors and cores: the learned
    step (network trained on traces of a plain run from another start) must
    reach the plain FP32 method's 20-epoch test RMSE in fewer epochs and less
    wall time, its own statistics and network passes included."""
    w, tri, tei, xtr, xte = planted()
    LR = LAM = 0.01

    def start(off):
        A, B = synth.initial_factors(w, seed_offset=off)
        return [a.to(DEV) for a in A], [b.to(DEV) for b in B]

    def timed(model_epoch, model, epochs, target=None):
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for ep in range(epochs):
            model_epoch()
            r = model.rmse(tei, xte)[0]
            if target is not None and r <= target:
                t1 = torch.cuda.Event(enable_timing=True)
                t1.record()
                t1.synchronize()
                return ep + 1, t0.elapsed_time(t1), r
        t1 = torch.cuda.Event(enable_timing=True)
        t1.record()
        t1.synchronize()
        return epochs, t0.elapsed_time(t1), r

    A, B = start(1)
    plain = ft.FastTuckerPlus(tri, xtr, A, B)
    ep_p, t_p, target = timed(lambda: (plain.epoch_factors(LR, LAM), plain.epoch_core(LR, LAM)), plain, 20)
    A2, B2 = start(7)
    tracer = ft.FastTuckerPlus(tri, xtr, A2, B2)
    F, Y = learned_step.collect_traces(tracer, 10, LR, LAM, LR, LAM)
    net = ft.new_stepnet(DEV, seed=0)
    learned_step.train(net, F, Y, steps=400, lr=3e-3)
    A3, B3 = start(1)
    model = ft.FastTuckerPlus(tri, xtr, A3, B3)
    ls = learned_step.LearnedStep(model, net, LR, LAM)
    ep_l, t_l, r_l = timed(lambda: ls.epoch(LR, LAM), model, 20, target)
    assert r_l <= target, (r_l, target)
    assert ep_l < ep_p and t_l < t_p, (ep_l, t_l, ep_p, t_p)
