"""GPU path against the FP64 oracle, through the C ABI.

Tolerances (relative; denominators as stated), the same at every order N:
  * FP32 path: predictions <= 1e-5 relative to the same model evaluated on
    |A|, |B| (the scale of the FP32 rounding bound, so cancellation does not
    count against the kernel) and <= 1e-5 in Frobenius norm; per-nonzero
    factor gradients and factor steps <= 1e-5 elementwise against the
    absolute-value error model of tests/errmodel.py, and <= 1e-5 elementwise
    relative to max(|step|, RMS step of the mode) (or 10 times the step
    change that rounding A, B to the precision's inputs causes in the
    oracle, if larger: see TOL_ELEM_RMS); core gradients <= 1e-5
    elementwise relative to the absolute-value model of the gradient and in
    Frobenius norm; one deterministic factor epoch's factors <= 1e-4
    (Frobenius per matrix); one core epoch's B <= 1e-5.
  * TF32 path: the elementwise factor bounds at 5e-3, gradients
    (absolute-value model) <= 5e-3.
  * BF16 path: the same at 2e-2; trained test RMSE within 1% of the FP64
    oracle's.
Factors and cores are zero-mean draws at every order.  Sizes span several
16-nonzero tiles with a ragged tail.
"""
import math

import numpy as np
import pytest
import torch

import errmodel
import oracle
from paper_2404_10087_gb300 import ft, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL_STEP = {"fp32": 1e-4, "tf32": 5e-3, "bf16": 2e-2}
TOL_GRAD = {"fp32": 1e-5, "tf32": 5e-3, "bf16": 2e-2}
# elementwise factor steps: against the absolute-value error model (the
# stated bounds), and relative to max(|step|, RMS step of the mode) within
# the larger of TOL_ELEM_RMS and 10 times the change that a rounding of A and
# B to the precision's inputs causes in the FP64 oracle's own step (the
# error the inputs' precision implies by itself; on zero-mean factors of
# high order it exceeds any fixed bound, since d^(n) multiplies N - 1
# products that can cancel)
TOL_ELEM_MODEL = {"fp32": 1e-5, "tf32": 5e-3, "bf16": 2e-2}
TOL_ELEM_RMS = {"fp32": 1e-5, "tf32": 5e-3, "bf16": 2e-2}


def to_dev(idx, x, A, B):
    return ([idx[n].contiguous().to(DEV) for n in range(idx.shape[0])], x.to(DEV),
            [a.clone().to(DEV) for a in A], [b.clone().to(DEV) for b in B])


def f64(ts):
    return [t.detach().double().cpu().numpy() for t in ts]


def rel_elem(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    rms = math.sqrt(float(np.mean(ref * ref))) if ref.size else 0.0
    den = np.maximum(np.abs(ref), 1e-3 * rms + 1e-300)
    return float(np.max(np.abs(got - ref) / den)) if ref.size else 0.0


def rel_bound(got, ref, scale):
    """Forward error relative to the absolute-value model: |got - ref| over
    the same computation on |A|, |B| (the scale a rounding-error bound of
    sums of products is proportional to)."""
    got, ref, scale = (np.asarray(v, np.float64) for v in (got, ref, scale))
    return float(np.max(np.abs(got - ref) / np.maximum(scale, 1e-300))) if ref.size else 0.0


def core_grad_scale(A, B, idx, x):
    """sum_m |e_m| |a^(n)|^T prod_{k != n} |a^(k)| |B^(k)| - the absolute-value
    model of the core gradient, obtained from the oracle by evaluating it on
    |A|, |B| with values shifted so that every residual equals |e_m|."""
    e = x - oracle.predict(A, B, idx)
    Aa, Ba = [np.abs(a) for a in A], [np.abs(b) for b in B]
    shifted = oracle.predict(Aa, Ba, idx) - np.abs(e)
    return oracle.core_grad(Aa, Ba, idx, shifted)


def rel_fro(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / d) if d > 0 else float(np.linalg.norm(got))


SHAPES = [
    # (I, J, R, nnz)
    ((50, 60, 70), (16, 16, 16), 16, 16 * 37 + 5),
    ((40, 50, 60), (4, 5, 6), 7, 1000),
    ((30, 20), (3, 9), 11, 333),
    ((25,), (8,), 5, 77),
    ((20, 21, 22, 23), (32, 32, 32, 32), 32, 16 * 20 + 9),
    ((20, 21, 22, 23, 24), (16, 12, 10, 8, 16), 16, 400),
    ((40, 41, 42, 43, 44, 45, 46, 47), (4, 4, 4, 4, 4, 4, 4, 4), 4, 300),
    ((40, 40, 40), (20, 24, 17), 29, 700),
    ((20, 21, 22, 23, 24), (32, 17, 24, 20, 28), 24, 16 * 19 + 3),
    ((12, 13, 14, 15, 16, 17, 18, 19, 20), (8, 16, 4, 12, 16, 8, 16, 4, 16), 16, 16 * 23 + 7),
    (tuple(range(10, 20)), (16,) * 10, 16, 16 * 25 + 11),
]
SHAPE_IDS = [f"N{len(s[0])}_J{max(s[1])}_R{s[2]}_nnz{s[3]}" for s in SHAPES]


@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
def test_predict_fp32(shape):
    I, J, R, nnz = shape
    idx, x, A, B = synth.random_problem(1, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    m = ft.FastTuckerPlus(gidx, gx, gA, gB)
    got = m.predict(gidx).double().cpu().numpy()
    ref = oracle.predict(f64(A), f64(B), idx.numpy())
    scale = oracle.predict([np.abs(a) for a in f64(A)], [np.abs(b) for b in f64(B)], idx.numpy())
    assert rel_bound(got, ref, scale) <= 1e-5
    assert rel_fro(got, ref) <= 1e-5


def check_factor_step(A0, B, idx, x, S, lr, lam, A1, precision):
    """Elementwise check of one factor epoch's step A1 - A0 against the
    oracle's batch-synchronous epoch (batch S): against the absolute-value
    error model and relative to max(|step|, RMS step of the mode); rows no
    nonzero touches are unchanged bit for bit.  Returns both errors."""
    ref, scales, touches = errmodel.epoch_step_model(A0, B, idx, x, S, lr, lam)
    for a0, a1, t in zip(A0, A1, touches):
        assert np.array_equal(a1[t == 0], a0[t == 0])
    em = errmodel.step_errors(A0, A1, ref, scales, touches)
    er = errmodel.step_errors_floor(A0, A1, ref, touches, 1.0)
    sens = errmodel.rounding_sensitivity(A0, B, idx, x, S, lr, lam, errmodel.UNIT_ROUNDOFF[precision])
    assert em <= TOL_ELEM_MODEL[precision], em
    assert er <= max(TOL_ELEM_RMS[precision], 10 * sens), (er, sens)
    return em, er


def collision_free(shape, seed):
    """The shape's ranks and nonzero count with mode sizes of at least nnz and
    rows that no two nonzeros share in any mode."""
    I, J, R, nnz = shape
    I2 = tuple(max(In, nnz + 3) for In in I)
    _, x, A, B = synth.random_problem(seed, I2, J, R, nnz)
    g = torch.Generator().manual_seed(seed + 1000)
    idx = torch.stack([torch.randperm(In, generator=g)[:nnz] for In in I2]).to(torch.int32)
    return idx, x, A, B


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
def test_per_nonzero_gradients(shape, precision):
    """Eq. "Gradient_low_rank_cp" per nonzero, element by element: with rows
    that no two nonzeros share and one batch of all nonzeros, the
    deterministic epoch at step 1 moves every row by exactly -g of its one
    nonzero, computed from the starting factors."""
    idx, x, A, B = collision_free(shape, 21)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    nnz = shape[3]
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision=precision, scatter="deterministic", det_batch=nnz)
    m.epoch_factors(1.0, 0.05)
    m.check()
    check_factor_step(f64(A), f64(B), idx.numpy(), x.double().numpy(), nnz, 1.0, 0.05, f64(gA), precision)


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
def test_deterministic_factor_epoch(shape, precision):
    """One batch-synchronous epoch (batch 128, rows shared by many nonzeros):
    the step element by element, and at FP32 the factors in Frobenius norm."""
    I, J, R, nnz = shape
    idx, x, A, B = synth.random_problem(2, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    S = 128
    lr, lam = 0.02, 0.05
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision=precision, scatter="deterministic", det_batch=S)
    m.epoch_factors(lr, lam)
    m.check()
    got = f64(gA)
    check_factor_step(f64(A), f64(B), idx.numpy(), x.double().numpy(), S, lr, lam, got, precision)
    if precision == "fp32":
        ref = oracle.factor_epoch(f64(A), f64(B), idx.numpy(), x.double().numpy(), S, lr, lam)
        for n in range(len(I)):
            assert rel_fro(got[n], ref[n]) <= 1e-4


@pytest.mark.parametrize("scheme", ["calc", "store"])
@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
def test_core_gradient(shape, precision, scheme):
    """Both core schemes of Sec. 5.6: rows of C formed per nonzero
    (calculation) or gathered from C = A B computed once in FP32 (storage)."""
    I, J, R, nnz = shape
    idx, x, A, B = synth.random_problem(3, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision=precision, core_scheme=scheme)
    G = f64(m.core_grad())
    A64, B64, i64, x64 = f64(A), f64(B), idx.numpy(), x.double().numpy()
    ref = oracle.core_grad(A64, B64, i64, x64)
    scale = core_grad_scale(A64, B64, i64, x64)
    for n in range(len(I)):
        assert rel_bound(G[n], ref[n], scale[n]) <= TOL_GRAD[precision], n
        if precision == "fp32":
            assert rel_fro(G[n], ref[n]) <= 1e-5, n


@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
def test_bf16_row_copies_change_nothing(shape):
    """The BF16 core pass of a context reads BF16 copies of the factor rows
    (rounded to nearest even, zero past J_n); the pass without a workspace
    gathers the float32 rows and rounds them itself.  Same grid, same order,
    same roundings: the gradients must be equal bit for bit."""
    I, J, R, nnz = shape
    idx, x, A, B = synth.random_problem(13, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision="bf16")
    G = torch.cat([g.reshape(-1) for g in m.core_grad()])
    G2 = torch.empty_like(G)
    ft.ft_core_grad_noalloc(gidx, gx, gA, gB, G2, precision="bf16")
    torch.cuda.synchronize()
    assert torch.equal(G, G2)


@pytest.mark.parametrize("precision,scheme", [("fp32", "calc"), ("bf16", "calc"), ("fp32", "store"),
                                              ("bf16", "store")])
def test_core_epoch_and_errors(precision, scheme):
    I, J, R, nnz = (60, 70, 80), (16, 16, 16), 16, 5000
    idx, x, A, B = synth.random_problem(4, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision=precision, core_scheme=scheme)
    lr, lam = 0.5, 0.01
    m.epoch_core(lr, lam)
    ref = oracle.core_epoch(f64(A), f64(B), idx.numpy(), x.double().numpy(), lr, lam)
    got = f64(gB)
    B0 = f64(B)
    for n in range(3):
        assert rel_fro(got[n] - B0[n], ref[n] - B0[n]) <= TOL_GRAD[precision]
    r = m.rmse(gidx, gx)
    ro = oracle.errors(f64(gA), f64(gB), idx.numpy(), x.double().numpy())
    assert abs(r[0] - ro[0]) <= 1e-5 * ro[0]
    assert abs(r[1] - ro[1]) <= 1e-5 * ro[1]
    assert abs(r[2] - ro[2]) <= 2e-5 * ro[2]


@pytest.mark.parametrize("scheme", ["calc", "store"])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[4], SHAPES[1]], ids=[SHAPE_IDS[0], SHAPE_IDS[4], SHAPE_IDS[1]])
def test_core_sgd_sets_match_oracle(shape, precision, scheme):
    """Per-set core SGD (Algorithm 3's core loop): consecutive sets of S
    nonzeros, a ragged last one, each an averaged core step from the core
    matrices the previous set left."""
    I, J, R, nnz = shape
    idx, x, A, B = synth.random_problem(7, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision=precision, core_scheme=scheme)
    S = max(1, nnz // 5 + 3)
    lr, lam = 0.5, 0.01
    m.epoch_core_sgd(lr, lam, S)
    m.check()
    ref = oracle.core_epoch_sgd(f64(A), f64(B), idx.numpy(), x.double().numpy(), S, lr, lam)
    got, B0 = f64(gB), f64(B)
    for n in range(len(I)):
        assert rel_fro(got[n] - B0[n], ref[n] - B0[n]) <= TOL_GRAD[precision], n


def test_core_sgd_one_set_is_the_core_epoch():
    """A set size of at least nnz is exactly Algorithm 5's step (bit for bit)."""
    I, J, R, nnz = (40, 50, 60), (16, 16, 16), 16, 3000
    idx, x, A, B = synth.random_problem(8, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    gB2 = [b.clone() for b in gB]
    m1 = ft.FastTuckerPlus(gidx, gx, gA, gB, precision="bf16")
    m2 = ft.FastTuckerPlus(gidx, gx, gA, gB2, precision="bf16")
    m1.epoch_core(0.3, 0.01)
    m2.epoch_core_sgd(0.3, 0.01, nnz + 5)
    torch.cuda.synchronize()
    for a, b in zip(gB, gB2):
        assert torch.equal(a, b)
    with pytest.raises(ft.FtError):
        m2.epoch_core_sgd(0.3, 0.01, 0)


def test_row_step_scale_deterministic():
    I, J, R, nnz = (30, 40, 50), (16, 16, 16), 16, 900
    idx, x, A, B = synth.random_problem(5, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    g = torch.Generator().manual_seed(9)
    scales = [torch.rand(In, generator=g, dtype=torch.float64).float() * 3.75 + 0.25 for In in I]
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, scatter="deterministic", det_batch=64)
    m.epoch_factors(0.02, 0.05, [s.to(DEV) for s in scales])
    m.check()
    rs = [s.double().numpy() for s in scales]
    A0 = f64(A)
    ref, sc, touches = errmodel.epoch_step_model(A0, f64(B), idx.numpy(), x.double().numpy(), 64, 0.02, 0.05,
                                                 row_scale=rs)
    assert errmodel.step_errors(A0, f64(gA), ref, sc, touches) <= TOL_ELEM_MODEL["fp32"]
    assert errmodel.step_errors_floor(A0, f64(gA), ref, touches, 1.0) <= 1e-4


@pytest.mark.parametrize("cache", [dict(hot_rows=0), dict(hot_min_count=1)], ids=["no_cache", "all_rows_cacheable"])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("shape", SHAPES, ids=SHAPE_IDS)
def test_hogwild_without_collisions_every_shape(shape, precision, cache):
    """The Hogwild pass on every parity shape - rows narrower than the padded
    rank K among them (read and written as 16-byte groups where J_n is a
    multiple of 4, element by element elsewhere), K = 32 with FP32-accurate
    three-pass TF32 products - equals the sequential epoch when no two
    nonzeros share a row, with the hot-row cache off and with every row
    cacheable."""
    idx, x, A, B = collision_free(shape, 31)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    nnz = shape[3]
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision=precision, **cache)
    m.epoch_factors(0.03, 0.02)
    m.check()
    check_factor_step(f64(A), f64(B), idx.numpy(), x.double().numpy(), nnz, 0.03, 0.02, f64(gA), precision)


@pytest.mark.parametrize("cache", [dict(hot_rows=0), dict(hot_min_count=1), dict(hot_min_count=1, hot_window=1)],
                         ids=["no_cache", "all_rows_cacheable", "window_1"])
@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("nnz", [16 * 50 + 3, 16 * 50], ids=["ragged", "multiple_of_4"])
def test_hogwild_without_collisions_is_exact(precision, cache, nnz):
    """When no two nonzeros share a row in any mode, the Hogwild pass has no
    races and equals the sequential epoch - with or without the shared-memory
    cache of hot rows (hot_min_count = 1 lets every row be cached; a nonzero
    count that is a multiple of 4 takes the vector path of the coordinate
    remap)."""
    I, J, R = (nnz + 5, nnz + 9, nnz), (16, 16, 16), 16
    g = torch.Generator().manual_seed(6)
    idx = torch.stack([torch.randperm(In, generator=g)[:nnz] for In in I]).to(torch.int32)
    _, x, A, B = synth.random_problem(6, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision=precision, **cache)
    m.epoch_factors(0.03, 0.02)
    m.check()
    # no shared rows: the sequential epoch equals one batch of all nonzeros
    check_factor_step(f64(A), f64(B), idx.numpy(), x.double().numpy(), nnz, 0.03, 0.02, f64(gA), precision)


def test_permute_reorders_the_epoch():
    """ft_permute (a reshuffle of Omega between iterations, Algorithm 3):
    after reordering, the Hogwild pass (hot-row cache on, no row collisions,
    so the result is exact) equals a fresh context built on the reordered
    arrays bit for bit, and the oracle's sequential epoch in that order; a
    second reshuffle writes into the other buffer and still matches."""
    nnz = 16 * 40 + 7
    I, J, R = (nnz + 3, nnz + 11, nnz + 2), (16, 16, 16), 16
    g = torch.Generator().manual_seed(9)
    idx = torch.stack([torch.randperm(In, generator=g)[:nnz] for In in I]).to(torch.int32)
    _, x, A, B = synth.random_problem(9, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision="fp32", hot_min_count=1)
    order = torch.arange(nnz)
    for k in range(2):
        perm = torch.randperm(nnz, generator=g).to(torch.int32)
        order = order[perm.long()]
        m.permute(perm.to(DEV))
        A_before = [a.clone() for a in gA]
        m.epoch_factors(0.03, 0.02)
        m.check()
        pidx = idx[:, order]
        px = x[order]
        fresh_A = [a.clone() for a in A_before]
        m2 = ft.FastTuckerPlus([t.contiguous().to(DEV) for t in pidx], px.contiguous().to(DEV), fresh_A,
                               [b.clone() for b in gB], precision="fp32", hot_min_count=1)
        m2.epoch_factors(0.03, 0.02)
        torch.cuda.synchronize()
        for a, b in zip(gA, fresh_A):
            assert torch.equal(a, b), k
        ref = oracle.factor_epoch(f64(A_before), f64(gB), pidx.numpy(), px.double().numpy(), 1, 0.03, 0.02)
        for n in range(3):
            assert rel_fro(f64(gA)[n], ref[n]) <= 1e-5
    assert torch.equal(m.idx[0].cpu(), idx[0, order])


def test_rebind_to_another_copy():
    """ft_rebind: after pointing the context at a copy of its nonzeros (and
    spoiling the old arrays) the Hogwild pass (hot-row cache on, no row
    collisions) equals a fresh context on the copy bit for bit; a bad
    coordinate in a rebound array is masked and reported."""
    nnz = 16 * 30 + 5
    I, J, R = (nnz + 3, nnz + 7, nnz + 1), (16, 16, 16), 16
    g = torch.Generator().manual_seed(11)
    idx = torch.stack([torch.randperm(In, generator=g)[:nnz] for In in I]).to(torch.int32)
    _, x, A, B = synth.random_problem(11, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision="bf16", hot_min_count=1)
    cidx, cx = [t.clone() for t in gidx], gx.clone()
    m.rebind(cidx, cx)
    for t in gidx:
        t.fill_(-1)
    gx.fill_(float("nan"))
    fresh = [a.clone() for a in gA]
    m.epoch_factors(0.03, 0.02)
    m.check()
    m2 = ft.FastTuckerPlus(cidx, cx, fresh, [b.clone() for b in gB], precision="bf16", hot_min_count=1)
    m2.epoch_factors(0.03, 0.02)
    torch.cuda.synchronize()
    for a, b in zip(gA, fresh):
        assert torch.equal(a, b)
    # a rebind enqueued on a second stream while this context's epoch is still
    # queued on the current one (the rebuild goes to the idle remapped copy)
    cidx2, cx2 = [t.clone() for t in cidx], cx.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    m.epoch_factors(0.03, 0.02)
    m.rebind(cidx2, cx2, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    m.epoch_factors(0.03, 0.02)
    m.check()
    m2.epoch_factors(0.03, 0.02)
    m2.epoch_factors(0.03, 0.02)
    torch.cuda.synchronize()
    for a, b in zip(gA, fresh):
        assert torch.equal(a, b)
    bad = [t.clone() for t in cidx]
    bad[1][3] = I[1]
    m.rebind(bad, cx)
    m.epoch_factors(0.03, 0.02)
    with pytest.raises(ft.FtError) as e:
        m.check()
    assert e.value.status == -2


def test_permute_deterministic_mode_and_bad_entries():
    I, J, R, nnz = (30, 40, 50), (8, 16, 12), 10, 2000
    idx, x, A, B = synth.random_problem(10, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision="fp32", scatter="deterministic", det_batch=128)
    g = torch.Generator().manual_seed(10)
    perm = torch.randperm(nnz, generator=g).to(torch.int32)
    m.permute(perm.to(DEV))
    m.epoch_factors(0.02, 0.05)
    m.check()
    ref = oracle.factor_epoch(f64(A), f64(B), idx[:, perm.long()].numpy(), x[perm.long()].double().numpy(),
                              128, 0.02, 0.05)
    for n in range(3):
        assert rel_fro(f64(gA)[n], ref[n]) <= 1e-4
    bad = perm.clone()
    bad[17] = nnz
    m.permute(bad.to(DEV))
    with pytest.raises(ft.FtError) as e:
        m.check()
    assert e.value.status == -2
    with pytest.raises(ft.FtError) as e:
        ft.ft_permute(m.ctx, perm.to(DEV), m.idx, m.vals)   # aliases the current arrays
    assert e.value.status == -1


def test_l2_persist_is_only_a_cache_hint():
    """With the factor matrices marked persisting in L2 (one allocation, so
    the window covers only them) the deterministic epoch and the core
    gradient are bit for bit those of the same context without the hint."""
    I, J, R, nnz = (90, 80, 70), (16, 16, 16), 16, 3000
    idx, x, A, B = synth.random_problem(12, I, J, R, nnz)
    gidx, gx, _, gB = to_dev(idx, x, A, B)
    flat = torch.cat([a.reshape(-1) for a in A]).to(DEV)
    views, off = [], 0
    for a in A:
        views.append(flat[off:off + a.numel()].view(a.shape))
        off += a.numel()
    plain = [a.clone().to(DEV) for a in A]
    got = []
    for mats, l2 in ((views, True), (plain, False)):
        m = ft.FastTuckerPlus(gidx, gx, mats, [b.clone() for b in gB], precision="bf16",
                              scatter="deterministic", det_batch=256, l2_persist=l2)
        m.epoch_factors(0.02, 0.01)
        G = torch.cat([g.reshape(-1) for g in m.core_grad()])
        m.check()
        got.append(([t.clone() for t in mats], G.clone()))
    for a, b in zip(got[0][0], got[1][0]):
        assert torch.equal(a, b)
    assert torch.equal(got[0][1], got[1][1])


def test_deterministic_mode_is_bitwise_reproducible():
    I, J, R, nnz = (100, 20, 10), (16, 16, 16), 16, 4000
    idx, x, A, B = synth.random_problem(7, I, J, R, nnz)
    outs = []
    for _ in range(2):
        gidx, gx, gA, gB = to_dev(idx, x, A, B)
        m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision="bf16", scatter="deterministic", det_batch=512)
        for _ in range(2):
            m.epoch_factors(0.01, 0.01)
            m.epoch_core(0.01, 0.01)
        torch.cuda.synchronize()
        outs.append([t.cpu() for t in gA + gB])
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def planted_setup():
    w = synth.WORKLOADS["planted_uniform_1e5"]
    d = synth.draw_workload(w)
    planted = oracle.predict(f64(d.planted_A), f64(d.planted_B), d.idx.numpy())
    x = (torch.from_numpy(planted) + d.noise.double()).float()
    A0, B0 = synth.initial_factors(w)
    return w, d, x, A0, B0


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("tf32", 1e-2), ("bf16", 1e-2)])
def test_planted_training_matches_oracle(precision, tol):
    """Ten deterministic epochs (batch 256) on the planted 3-order workload
    (1e5 uniform coordinates, planted J = R = 4, noise 0.1): test RMSE of the
    GPU run within `tol` (relative) of the FP64 oracle's run."""
    w, d, x, A0, B0 = planted_setup()
    tr, te = d.train, d.test
    gA = [a.clone().to(DEV) for a in A0]
    gB = [b.clone().to(DEV) for b in B0]
    tri = [d.idx[n, tr].contiguous().to(DEV) for n in range(3)]
    tei = [d.idx[n, te].contiguous().to(DEV) for n in range(3)]
    S = 256
    m = ft.FastTuckerPlus(tri, x[tr].contiguous().to(DEV), gA, gB, precision=precision,
                          scatter="deterministic", det_batch=S)
    lr = lam = 0.01
    oA, oB = f64(A0), f64(B0)
    itr, ite = d.idx[:, tr].numpy(), d.idx[:, te].numpy()
    xtr, xte = x[tr].double().numpy(), x[te].double().numpy()
    r0 = oracle.errors(oA, oB, ite, xte)[0]
    for _ in range(10):
        m.epoch_factors(lr, lam)
        m.epoch_core(lr, lam)
        oA = oracle.factor_epoch(oA, oB, itr, xtr, S, lr, lam)
        oB = oracle.core_epoch(oA, oB, itr, xtr, lr, lam, nthreads=oracle.default_threads())
    g = m.rmse(tei, x[te].contiguous().to(DEV))[0]
    o = oracle.errors(oA, oB, ite, xte)[0]
    assert o < 0.9 * r0
    assert abs(g - o) <= tol * o, (g, o)


@pytest.mark.parametrize("cache,band", [(dict(hot_rows=3000, hot_min_count=1), 0.02), (dict(hot_rows=1500), 0.10),
                                        (dict(hot_rows=-1), 0.10), (dict(hot_rows=0), 0.35)],
                         ids=["all_rows_cached", "half_rows_cached", "default_cache", "no_cache"])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_hogwild_training_converges(precision, cache, band):
    """The Hogwild pass on a tensor whose rows collide constantly (9e4
    nonzeros on 1000 rows per mode, tens of thousands of updates in flight):
    ten epochs lower the test RMSE, and end near the sequential FP64 oracle's.
    With every row in the shared-memory cache no update is lost (each CTA's
    change is added to the row at write-back), and the run ends within 2% of
    the sequential oracle; with half of the rows cached, or the default
    cache (the 3024 most frequent rows with two or more nonzeros at K = 16,
    N = 3), within 10%; without the cache, where concurrent plain stores of
    a row lose updates as in the paper's kernel, within 35%."""
    w, d, x, A0, B0 = planted_setup()
    tr, te = d.train, d.test
    gA = [a.clone().to(DEV) for a in A0]
    gB = [b.clone().to(DEV) for b in B0]
    tri = [d.idx[n, tr].contiguous().to(DEV) for n in range(3)]
    tei = [d.idx[n, te].contiguous().to(DEV) for n in range(3)]
    m = ft.FastTuckerPlus(tri, x[tr].contiguous().to(DEV), gA, gB, precision=precision, **cache)
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
    assert abs(g - o) <= band * o, (g, o)


# ------------------------------------------------------------ edge cases
def test_empty_tensor():
    I, J, R = (5, 6, 7), (4, 4, 4), 4
    idx, x, A, B = synth.random_problem(8, I, J, R, 0)
    gidx = [torch.empty(0, dtype=torch.int32, device=DEV) for _ in range(3)]
    gx = torch.empty(0, dtype=torch.float32, device=DEV)
    gA = [a.clone().to(DEV) for a in A]
    gB = [b.clone().to(DEV) for b in B]
    for scatter in ("hogwild", "deterministic"):
        m = ft.FastTuckerPlus(gidx, gx, gA, gB, scatter=scatter)
        m.epoch_factors(0.1, 0.1)
        m.check()
        assert all(torch.equal(a.cpu(), b) for a, b in zip(gA, A))
    m.epoch_core(0.1, 0.5)  # no data: only the regulariser acts
    for b, b0 in zip(gB, B):
        torch.testing.assert_close(b.cpu(), b0 * (1 - 0.1 * 0.5), rtol=1e-6, atol=1e-7)
    assert m.rmse(gidx, gx) == (0.0, 0.0, 0.0)


@pytest.mark.parametrize("nnz", [1, 15, 16, 17])
def test_tiny_tensors(nnz):
    I, J, R = (3, 4, 5), (16, 16, 16), 16
    idx, x, A, B = synth.random_problem(9, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, scatter="deterministic", det_batch=4)
    m.epoch_factors(0.05, 0.1)
    ref = oracle.factor_epoch(f64(A), f64(B), idx.numpy(), x.double().numpy(), 4, 0.05, 0.1)
    for n in range(3):
        assert rel_fro(f64(gA)[n], ref[n]) <= 1e-5


def test_bad_inputs_are_rejected():
    I, J, R, nnz = (10, 11, 12), (4, 4, 4), 4, 100
    idx, x, A, B = synth.random_problem(10, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    bad = [t.clone() for t in gidx]
    bad[1][17] = 11  # == I_2
    with pytest.raises(ft.FtError) as e:
        ft.FastTuckerPlus(bad, gx, gA, gB)
    assert e.value.status == -2
    bad[1][17] = -1
    with pytest.raises(ft.FtError) as e:
        ft.FastTuckerPlus(bad, gx, gA, gB)
    assert e.value.status == -2
    gx2 = gx.clone()
    gx2[3] = float("nan")
    with pytest.raises(ft.FtError) as e:
        ft.FastTuckerPlus(gidx, gx2, gA, gB)
    assert e.value.status == -5
    cfg = ft.make_config()
    ws = torch.empty(256, dtype=torch.uint8, device=DEV)
    with pytest.raises(ft.FtError) as e:
        ft.ft_init(I, J, R, gidx, gx, gA, gB, ws, cfg)
    assert e.value.status == -7


def test_nonfinite_residual_is_latched():
    I, J, R, nnz = (10, 11, 12), (4, 4, 4), 4, 100
    idx, x, A, B = synth.random_problem(11, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    m = ft.FastTuckerPlus(gidx, gx, gA, gB)
    gB[0][0, 0] = float("inf")  # poisons every prediction that uses row 0 of B^(1)
    m.epoch_factors(0.01, 0.01)
    with pytest.raises(ft.FtError) as e:
        m.check()
    assert e.value.status == -5
    m.check()  # the latch was cleared


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("J", [(16, 16, 16), (8, 12, 4)], ids=["full_width", "narrow"])
def test_fast_tile_reports_bad_coordinates_and_nonfinite(precision, J):
    """The branch-free Hogwild tile (every mode full width, or every mode's
    rows a multiple of 4 wide and some narrower than K; hot-row cache on, one
    step size) masks a coordinate outside its range (FT_ERR_INDEX) and
    latches a non-finite residual (FT_ERR_NONFINITE); rows of the masked
    nonzero are not written, and the next clean epoch clears the latch."""
    nnz = 16 * 30 + 7
    I, R = (nnz + 3, nnz + 5, nnz + 1), 16
    g = torch.Generator().manual_seed(17)
    idx = torch.stack([torch.randperm(In, generator=g)[:nnz] for In in I]).to(torch.int32)
    _, x, A, B = synth.random_problem(17, I, J, R, nnz)
    gidx, gx, gA, gB = to_dev(idx, x, A, B)
    m = ft.FastTuckerPlus(gidx, gx, gA, gB, precision=precision, hot_min_count=1)
    bad = [t.clone() for t in gidx]
    bad[0][40] = I[0] + 2
    m.rebind(bad, gx)
    before = [a.clone() for a in gA]
    m.epoch_factors(0.03, 0.02)
    with pytest.raises(ft.FtError) as e:
        m.check()
    assert e.value.status == -2
    for n in (1, 2):   # the masked nonzero's other rows are untouched
        r = int(idx[n, 40])
        assert torch.equal(gA[n][r], before[n][r])
    m.rebind(gidx, gx)
    m.epoch_factors(0.03, 0.02)
    m.check()
    gB[0][0, 0] = float("inf")
    m.epoch_factors(0.03, 0.02)
    with pytest.raises(ft.FtError) as e:
        m.check()
    assert e.value.status == -5
