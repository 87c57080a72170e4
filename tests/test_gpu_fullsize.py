"""Parity at the benchmark's full size and launch configuration.

The Netflix-shaped Zipf tensor (1e8 distinct coordinates, 9e7 training and
1e7 test nonzeros, J = R = 16) is drawn on the device; its planted ratings
are computed by the FP64 oracle (never by the CUDA path).  Against the
oracle:
  * predictions on a 2e5-nonzero sample (FP32, bound-relative 1e-5);
  * the core gradient over all 9e7 training nonzeros (FP32 <= 1e-5 and BF16
    <= 2e-2 in Frobenius norm), and the core epoch's B (its step to the same
    tolerance, plus the float32 rounding of the stored B);
  * the test-set RMSE and MAE (<= 1e-5);
  * the Hogwild factor pass in the benchmark's configuration (BF16, hot-row
    cache): properties that hold at any size - rows of no training nonzero are
    bitwise unchanged, every row stays finite, and the training error on a
    1e6-nonzero sample (oracle) drops.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_10087_gb300 import ft, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
THREADS = oracle.default_threads()


def rel_fro(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def full():
    w = synth.WORKLOADS["netflix_shaped_zipf_1e8"]
    d = synth.draw_workload(w, device=DEV)
    idx_h = d.idx.cpu().numpy()
    pred = oracle.predict([a.double().cpu().numpy() for a in d.planted_A],
                          [b.double().cpu().numpy() for b in d.planted_B], idx_h, nthreads=THREADS)
    vals = synth.to_ratings(torch.from_numpy(pred))
    del pred
    tr, te = d.train.cpu(), d.test.cpu()
    tr_h = np.ascontiguousarray(idx_h[:, tr.numpy()])
    te_h = np.ascontiguousarray(idx_h[:, te.numpy()])
    _, x_tr, x_te = synth.centre(vals[tr].contiguous(), vals[te].contiguous())
    A0, B0 = synth.initial_factors(w)
    return dict(w=w, tr_h=tr_h, te_h=te_h, x_tr=x_tr, x_te=x_te, A0=A0, B0=B0,
                tri=[torch.from_numpy(tr_h[n]).to(DEV) for n in range(3)],
                tei=[torch.from_numpy(te_h[n]).to(DEV) for n in range(3)],
                gx_tr=x_tr.to(DEV), gx_te=x_te.to(DEV))


def context(full, precision):
    gA = [a.clone().to(DEV) for a in full["A0"]]
    gB = [b.clone().to(DEV) for b in full["B0"]]
    return ft.FastTuckerPlus(full["tri"], full["gx_tr"], gA, gB, precision=precision), gA, gB


def test_fullsize_predict_sample(full):
    m, gA, gB = context(full, "bf16")
    pred = m.predict(full["tri"])
    g = torch.Generator().manual_seed(5)
    pick = torch.randint(0, pred.numel(), (200_000,), generator=g)
    got = pred.cpu()[pick].double().numpy()
    sub = full["tr_h"][:, pick.numpy()]
    A64 = [a.double().numpy() for a in full["A0"]]
    B64 = [b.double().numpy() for b in full["B0"]]
    ref = oracle.predict(A64, B64, sub, nthreads=THREADS)
    scale = oracle.predict([np.abs(a) for a in A64], [np.abs(b) for b in B64], sub, nthreads=THREADS)
    assert float(np.max(np.abs(got - ref) / scale)) <= 1e-5


@pytest.fixture(scope="module")
def oracle_grad(full):
    A64 = [a.double().numpy() for a in full["A0"]]
    B64 = [b.double().numpy() for b in full["B0"]]
    return oracle.core_grad(A64, B64, full["tr_h"], full["x_tr"].double().numpy(), nthreads=THREADS)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16", 2e-2)])
def test_fullsize_core_gradient_and_epoch(full, oracle_grad, precision, tol):
    m, gA, gB = context(full, precision)
    G = [g.double().cpu().numpy() for g in m.core_grad()]
    for n in range(3):
        assert rel_fro(G[n], oracle_grad[n]) <= tol, n
    lr, lam = 0.01, 0.01
    m.epoch_core(lr, lam)
    nnz = full["x_tr"].numel()
    for n in range(3):
        b0 = full["B0"][n].double().numpy()
        want = b0 - lr * (oracle_grad[n] / nnz + lam * b0)
        got = gB[n].double().cpu().numpy()
        # the step (~1e-4 of B) is compared up to tol plus the float32 rounding
        # of the stored B (a few ulps of |B|)
        err = np.linalg.norm(got - want)
        assert err <= tol * np.linalg.norm(want - b0) + 4 * 2.0 ** -24 * np.linalg.norm(want), n


def test_fullsize_errors(full):
    m, gA, gB = context(full, "bf16")
    r = m.rmse(full["tei"], full["gx_te"])
    A64 = [a.double().numpy() for a in full["A0"]]
    B64 = [b.double().numpy() for b in full["B0"]]
    o = oracle.errors(A64, B64, full["te_h"], full["x_te"].double().numpy(), nthreads=THREADS)
    assert abs(r[0] - o[0]) <= 1e-5 * o[0]
    assert abs(r[1] - o[1]) <= 1e-5 * o[1]


def test_fullsize_hogwild_epoch_properties(full):
    m, gA, gB = context(full, "bf16")   # the benchmark's configuration
    m.epoch_factors(0.01, 0.01)
    m.check()
    touched = [np.zeros(I, dtype=bool) for I in full["w"].I]
    for n in range(3):
        touched[n][full["tr_h"][n]] = True
    for n in range(3):
        a = gA[n].cpu()
        assert torch.isfinite(a).all()
        assert torch.equal(a[~torch.from_numpy(touched[n])], full["A0"][n][~torch.from_numpy(touched[n])])
        assert not torch.equal(a[torch.from_numpy(touched[n])], full["A0"][n][torch.from_numpy(touched[n])])
    g = torch.Generator().manual_seed(6)
    pick = torch.randint(0, full["x_tr"].numel(), (1_000_000,), generator=g).numpy()
    sub, xs = full["tr_h"][:, pick], full["x_tr"].double().numpy()[pick]
    B64 = [b.double().numpy() for b in full["B0"]]
    before = oracle.errors([a.double().numpy() for a in full["A0"]], B64, sub, xs, nthreads=THREADS)[0]
    after = oracle.errors([a.double().cpu().numpy() for a in gA], B64, sub, xs, nthreads=THREADS)[0]
    assert after < before, (before, after)
