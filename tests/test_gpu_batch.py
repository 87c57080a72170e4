"""Batched persistent epoch (many tensors, one graph) against the oracle."""
import numpy as np
import pytest
import torch

import errmodel
import oracle
from paper_2404_10087_gb300 import ft, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"

# (I, J, R, nnz): uneven orders and ranks over both padded ranks K = 16, 32;
# rows read as 16-byte groups (J_n a multiple of 4, full width or narrower than
# K: the branch-free tile) and element by element (J_n = 5, 6, 7: the generic
# tile) in one kernel class
SHAPES = [((40, 50, 60), (16, 16, 16), 16, 16 * 40 + 3),
          ((30, 35, 40), (5, 6, 7), 9, 16 * 28 + 5),
          ((30, 40), (4, 8), 8, 333),
          ((20, 21, 22, 23), (8, 8, 8, 8), 32, 500),
          ((25, 26, 27, 28, 29), (16, 16, 16, 16, 16), 8, 600),
          ((25, 26, 27, 28, 29), (8, 8, 8, 8, 8), 32, 400),
          ((60, 70, 80), (16, 16, 16), 16, 0)]


def f64(ts):
    return [t.detach().double().cpu().numpy() for t in ts]


def rel_fro(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / d) if d > 0 else float(np.linalg.norm(got))


def make(seed, disjoint):
    out = []
    for k, (I, J, R, nnz) in enumerate(SHAPES):
        idx, x, A, B = synth.random_problem(seed + k, I, J, R, nnz)
        if disjoint and nnz:
            nnz = min(nnz, min(I))
            g = torch.Generator().manual_seed(seed + 100 + k)
            idx = torch.stack([torch.randperm(In, generator=g)[:nnz] for In in I]).to(torch.int32)
            x = x[:nnz].contiguous()
        out.append(dict(idx=idx, x=x, A=A, B=B))
    return out


def to_batch(probs):
    dev = []
    for p in probs:
        dev.append(([p["idx"][n].contiguous().to(DEV) for n in range(p["idx"].shape[0])], p["x"].to(DEV),
                    [a.clone().to(DEV) for a in p["A"]], [b.clone().to(DEV) for b in p["B"]]))
    return dev


@pytest.mark.parametrize("tune", [False, True])
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("bf16", 2e-2)])
def test_batch_epoch_without_collisions_matches_oracle(precision, tol, tune):
    """Rows shared by no two nonzeros: every tensor's factor pass equals the
    sequential epoch - element by element, against the absolute-value error
    model (FP32 1e-5, BF16 2e-2) and relative to max(|step|, RMS step) within
    the same bound or 10 times the step change that rounding A, B to the
    precision's inputs causes in the oracle, untouched rows bit for bit - and
    its core step the oracle's on those factors, element by element against
    lr_b / nnz times the absolute-value model of the core gradient (same
    bounds)."""
    tol_model = {"fp32": 1e-5, "bf16": 2e-2}[precision]
    u = errmodel.UNIT_ROUNDOFF[precision]
    probs = make(10, disjoint=True)
    dev = to_batch(probs)
    b = ft.FastTuckerBatch(dev, precision=precision, tune=tune)
    lr_a, lam_a, lr_b, lam_b = 0.03, 0.02, 0.5, 0.01
    b.epoch(lr_a, lam_a, lr_b, lam_b)
    torch.cuda.synchronize()
    for p, (idx, x, A, B) in zip(probs, dev):
        i64, x64 = p["idx"].numpy(), p["x"].double().numpy()
        A0, B0 = f64(p["A"]), f64(p["B"])
        nnz = max(1, x64.shape[0])
        oA, sc, touches = errmodel.epoch_step_model(A0, B0, i64, x64, nnz, lr_a, lam_a)
        A1 = f64(A)
        for a0, a1, t in zip(A0, A1, touches):
            assert np.array_equal(a1[t == 0], a0[t == 0])
        assert errmodel.step_errors(A0, A1, oA, sc, touches) <= tol_model
        sens = errmodel.rounding_sensitivity(A0, B0, i64, x64, nnz, lr_a, lam_a, u)
        assert errmodel.step_errors_floor(A0, A1, oA, touches, 1.0) <= max(tol_model, 10 * sens)
        oB = oracle.core_epoch(oA, B0, i64, x64, lr_b, lam_b)
        # the core step, element by element against lr_b / nnz times the
        # absolute-value model of the core gradient, plus the float32
        # rounding of the stored B
        if x64.shape[0]:
            e = x64 - oracle.predict(oA, B0, i64)
            Aa, Ba = [np.abs(a) for a in oA], [np.abs(b) for b in B0]
            Gs = oracle.core_grad(Aa, Ba, i64, oracle.predict(Aa, Ba, i64) - np.abs(e))
            for n in range(len(A0)):
                B1 = f64(B)[n]
                err = np.abs(B1 - oB[n]) - 2.0 ** -24 * np.abs(oB[n])
                assert np.max(err / (lr_b / x64.shape[0] * Gs[n] + 1e-300)) <= tol_model, n


def test_batch_core_step_matches_oracle_with_collisions():
    """With lr_a = 0 the factor pass leaves A unchanged, so the batched core
    pass and finalize can be checked exactly on tensors with collisions."""
    probs = make(20, disjoint=False)
    dev = to_batch(probs)
    b = ft.FastTuckerBatch(dev, precision="fp32")
    b.epoch(0.0, 0.0, 0.7, 0.05)
    torch.cuda.synchronize()
    for p, (idx, x, A, B) in zip(probs, dev):
        A0, B0 = f64(p["A"]), f64(p["B"])
        for n in range(len(A0)):
            assert np.array_equal(f64(A)[n], A0[n])
        oB = oracle.core_epoch(A0, B0, p["idx"].numpy(), p["x"].double().numpy(), 0.7, 0.05)
        for n in range(len(B0)):
            assert rel_fro(f64(B)[n] - B0[n], oB[n] - B0[n]) <= 1e-5


def test_batch_rmse_and_classes():
    probs = make(30, disjoint=False)
    dev = to_batch(probs)
    b = ft.FastTuckerBatch(dev, precision="bf16", tune=True)
    cls = b.classes()
    assert sum(c["tensors"] for c in cls) == len(probs)
    for c in cls:
        assert c["unit_tiles"] in (64, 256, 1024) and c["ctas_per_sm"] >= 1 and c["units"] >= c["tensors"]
    for t, (p, (idx, x, A, B)) in enumerate(zip(probs, dev)):
        r = b.rmse(t, idx, x)
        o = oracle.errors(f64(p["A"]), f64(p["B"]), p["idx"].numpy(), p["x"].double().numpy())
        assert abs(r[0] - o[0]) <= 1e-5 * max(o[0], 1e-30)
    n0 = b.launches
    b.epoch(0.01, 0.01)
    assert b.launches - n0 == 1 + 2 * len(cls) + 1


def test_batch_rejects_bad_coordinates():
    probs = make(40, disjoint=False)
    dev = to_batch(probs)
    dev[1][0][0][3] = 10_000
    with pytest.raises(ft.FtError) as e:
        ft.FastTuckerBatch(dev)
    assert e.value.status == -2
