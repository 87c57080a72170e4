"""The tcgen05 factor pass (FT_ENGINE_TCGEN05: 128-nonzero warpgroup tiles,
products on tcgen05.mma with TMEM accumulators) against the FP64 oracle,
through the C ABI.  With the hot-row cache on, every row full width and one
step size (the full-width shapes below with a cache), the rows of the next
tile arrive by bulk copies (cp.async.bulk on an mbarrier) while the current
tile computes; the other shapes and the row-scale test run the pass that
gathers through registers.

Tolerances as for the BF16 warp-tile pass: one epoch's step A_new - A_old
element by element within 2e-2 of the oracle's against the absolute-value
error model of tests/errmodel.py, and relative to max(|step|, RMS step)
within 2e-2 or 10 times the step change that rounding A, B to BF16 causes in
the oracle, when no two nonzeros share a row (no races, so the Hogwild
pass equals the sequential epoch); untouched rows bit for bit.  Sizes
span several 128-nonzero tiles, several CTAs and a ragged tail.
"""
import numpy as np
import pytest
import torch

import errmodel
import oracle
from paper_2404_10087_gb300 import ft, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = 2e-2


def f64(ts):
    return [t.detach().double().cpu().numpy() for t in ts]


def rel_fro(got, ref):
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / d) if d > 0 else float(np.linalg.norm(got))


def check_step(A0, B, idx, x, lr, lam, A1, row_scale=None):
    nnz = max(1, x.shape[0])
    ref, sc, touches = errmodel.epoch_step_model(A0, B, idx, x, nnz, lr, lam, row_scale=row_scale)
    for a0, a1, t in zip(A0, A1, touches):
        assert np.array_equal(a1[t == 0], a0[t == 0])
    assert errmodel.step_errors(A0, A1, ref, sc, touches) <= TOL
    sens = errmodel.rounding_sensitivity(A0, B, idx, x, nnz, lr, lam, errmodel.UNIT_ROUNDOFF["bf16"])
    assert errmodel.step_errors_floor(A0, A1, ref, touches, 1.0) <= max(TOL, 10 * sens)


def distinct_rows_problem(seed, nnz, J, R, extra=7):
    """nnz nonzeros whose rows are distinct in every mode."""
    N = len(J)
    I = tuple(nnz + extra * (n + 1) for n in range(N))
    g = torch.Generator().manual_seed(seed)
    idx = torch.stack([torch.randperm(In, generator=g)[:nnz] for In in I]).to(torch.int32)
    _, x, A, B = synth.random_problem(seed, I, J, R, nnz)
    return I, idx, x, A, B


SHAPES = [
    ((16, 16, 16), 16, 128 * 40 + 77),       # the Netflix-shaped ranks, ragged tail
    ((16, 16, 16), 16, 128 * 4 * 152 * 2 + 5),  # more tiles than one pass of the grid
    ((4, 12, 9), 13, 1000),                  # J, R below 16 (zero padding, scalar rows)
    ((16, 8), 16, 700),
    ((16,), 11, 300),
    ((16, 16, 12, 8), 16, 2000),
]
IDS = [f"N{len(s[0])}_J{max(s[0])}_R{s[1]}_nnz{s[2]}" for s in SHAPES]


@pytest.mark.parametrize("cache", [dict(hot_rows=0), dict(hot_min_count=1), dict(hot_min_count=1, hot_window=1)],
                         ids=["no_cache", "all_rows_cacheable", "window_1"])
@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_collision_free_epoch_matches_oracle(shape, cache):
    J, R, nnz = shape
    I, idx, x, A, B = distinct_rows_problem(11, nnz, J, R)
    gidx = [idx[n].contiguous().to(DEV) for n in range(len(J))]
    gA = [a.clone().to(DEV) for a in A]
    gB = [b.clone().to(DEV) for b in B]
    m = ft.FastTuckerPlus(gidx, x.to(DEV), gA, gB, precision="bf16", engine="tcgen05", **cache)
    m.epoch_factors(0.03, 0.02)
    m.check()
    check_step(f64(A), f64(B), idx.numpy(), x.double().numpy(), 0.03, 0.02, f64(gA))
    # B is not touched by the factor pass
    for b0, b in zip(B, gB):
        assert torch.equal(b0, b.cpu())


def test_row_step_scale():
    J, R, nnz = (16, 16, 16), 16, 3000
    I, idx, x, A, B = distinct_rows_problem(12, nnz, J, R)
    g = torch.Generator().manual_seed(4)
    scales = [torch.rand(In, generator=g) * 3.75 + 0.25 for In in I]
    gidx = [idx[n].contiguous().to(DEV) for n in range(3)]
    gA = [a.clone().to(DEV) for a in A]
    m = ft.FastTuckerPlus(gidx, x.to(DEV), gA, [b.to(DEV) for b in B], precision="bf16", engine="tcgen05")
    m.epoch_factors(0.02, 0.01, [s.to(DEV) for s in scales])
    m.check()
    check_step(f64(A), f64(B), idx.numpy(), x.double().numpy(), 0.02, 0.01, f64(gA),
               row_scale=[s.double().numpy() for s in scales])


def test_agrees_with_warp_engine():
    """Both engines compute the same BF16 products with FP32 accumulation:
    on a collision-free epoch they agree far inside the oracle tolerance."""
    J, R, nnz = (16, 16, 16), 16, 5000
    I, idx, x, A, B = distinct_rows_problem(13, nnz, J, R)
    outs = []
    for engine in ("warp", "tcgen05"):
        gA = [a.clone().to(DEV) for a in A]
        m = ft.FastTuckerPlus([idx[n].contiguous().to(DEV) for n in range(3)], x.to(DEV), gA,
                              [b.to(DEV) for b in B], precision="bf16", engine=engine, hot_rows=0)
        m.epoch_factors(0.03, 0.02)
        m.check()
        outs.append(f64(gA))
    for n in range(3):
        step_w, step_t = outs[0][n] - f64(A)[n], outs[1][n] - f64(A)[n]
        assert rel_fro(step_t, step_w) <= 2e-3, n
        # element by element, relative to max(|step|, RMS step)
        rms = np.sqrt(np.mean(step_w * step_w))
        assert np.max(np.abs(step_t - step_w) / np.maximum(np.abs(step_w), rms)) <= 2e-2, n


def test_hogwild_training_converges():
    """Ten Hogwild epochs on the planted 3-order workload (1e5 uniform
    coordinates on 1000 rows per mode, so many updates collide inside a
    128-nonzero tile): the test RMSE falls and stays within 35% of the
    sequential FP64 oracle's."""
    w = synth.WORKLOADS["planted_uniform_1e5"]
    d = synth.draw_workload(w)
    planted = oracle.predict(f64(d.planted_A), f64(d.planted_B), d.idx.numpy())
    x = (torch.from_numpy(planted) + d.noise.double()).float()
    A0, B0 = synth.initial_factors(w)
    tr, te = d.train, d.test
    gA = [a.clone().to(DEV) for a in A0]
    gB = [b.clone().to(DEV) for b in B0]
    tri = [d.idx[n, tr].contiguous().to(DEV) for n in range(3)]
    tei = [d.idx[n, te].contiguous().to(DEV) for n in range(3)]
    m = ft.FastTuckerPlus(tri, x[tr].contiguous().to(DEV), gA, gB, precision="bf16", engine="tcgen05")
    lr = lam = 0.01
    oA, oB = f64(A0), f64(B0)
    itr, ite = d.idx[:, tr].numpy(), d.idx[:, te].numpy()
    xtr, xte = x[tr].double().numpy(), x[te].double().numpy()
    r0 = oracle.errors(oA, oB, ite, xte)[0]
    for _ in range(10):
        m.epoch_factors(lr, lam)
        m.epoch_core(lr, lam)
        oA = oracle.factor_epoch(oA, oB, itr, xtr, 1, lr, lam)
        oB = oracle.core_epoch(oA, oB, itr, xtr, lr, lam, nthreads=oracle.default_threads())
    g = m.rmse(tei, x[te].contiguous().to(DEV))[0]
    o = oracle.errors(oA, oB, ite, xte)[0]
    assert g < r0, (g, r0)
    assert g <= 1.35 * o, (g, o)


def test_bad_index_is_reported_and_masked():
    J, R, nnz = (16, 16, 16), 16, 600
    I, idx, x, A, B = distinct_rows_problem(14, nnz, J, R)
    gidx = [idx[n].contiguous().to(DEV) for n in range(3)]
    gA = [a.clone().to(DEV) for a in A]
    m = ft.FastTuckerPlus(gidx, x.to(DEV), gA, [b.to(DEV) for b in B], precision="bf16", engine="tcgen05",
                          hot_rows=0)
    gidx[1][17] = I[1] + 3      # out of range after ft_init validated the tensor
    m.epoch_factors(0.03, 0.02)
    with pytest.raises(ft.FtError) as e:
        m.check()
    assert e.value.status == -2
    m.close()


def test_bad_index_is_reported_and_masked_async():
    """The same with the hot-row cache on and full-width rows, where the rows
    arrive by bulk copies: the masked nonzero's rows are neither copied nor
    written."""
    J, R, nnz = (16, 16, 16), 16, 600
    I, idx, x, A, B = distinct_rows_problem(16, nnz, J, R)
    gidx = [idx[n].contiguous().to(DEV) for n in range(3)]
    gA = [a.clone().to(DEV) for a in A]
    m = ft.FastTuckerPlus(gidx, x.to(DEV), gA, [b.to(DEV) for b in B], precision="bf16", engine="tcgen05",
                          hot_min_count=1)
    bad = [t.clone() for t in gidx]
    bad[1][17] = I[1] + 3
    m.rebind(bad, x.to(DEV))
    before = [a.clone() for a in gA]
    m.epoch_factors(0.03, 0.02)
    with pytest.raises(ft.FtError) as e:
        m.check()
    assert e.value.status == -2
    for n in (0, 2):
        r = int(idx[n, 17])
        assert torch.equal(gA[n][r], before[n][r])
    m.close()


def test_empty_and_single_nonzero():
    for nnz in (0, 1):
        J, R = (16, 16, 16), 16
        I, idx, x, A, B = distinct_rows_problem(15, nnz, J, R)
        gA = [a.clone().to(DEV) for a in A]
        m = ft.FastTuckerPlus([idx[n].contiguous().to(DEV) for n in range(3)], x.to(DEV), gA,
                              [b.to(DEV) for b in B], precision="bf16", engine="tcgen05")
        m.epoch_factors(0.03, 0.02)
        m.check()
        ref = oracle.factor_epoch(f64(A), f64(B), idx.numpy(), x.double().numpy(), 1, 0.03, 0.02)
        for n in range(3):
            np.testing.assert_allclose(f64(gA)[n], ref[n], rtol=0, atol=2e-2 * max(1e-30, np.abs(ref[n]).max()))
