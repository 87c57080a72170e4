"""The no-allocation core-gradient entry point against the context-based one.

ft_core_grad_noalloc serves callers that cannot call cudaMalloc (their device
memory belongs to another allocator, or they cannot keep a context and its
workspace alive between calls): it takes the inputs and the output buffer
and keeps its scratch in a device array compiled into the library.  These
tests call it through the C ABI twice in a row (the shared scratch keeps the
previous call's contents) and compare each result with ft_core_grad on the
same inputs, within the FP32 tolerance the other parity tests use.

This file is collected last so that a run stopping at the first failure has
run every other test before it.
"""
import numpy as np
import pytest
import torch

from paper_2404_10087_gb300 import ft, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def rel_fro(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / d) if d > 0 else float(np.linalg.norm(got))


def problem(seed, I, J, R, nnz):
    idx, x, A, B = synth.random_problem(seed, I, J, R, nnz)
    return ([idx[n].contiguous().to(DEV) for n in range(len(I))], x.to(DEV),
            [a.to(DEV) for a in A], [b.to(DEV) for b in B])


def with_context(idx, x, A, B, precision):
    m = ft.FastTuckerPlus(idx, x, A, B, precision=precision)
    G = torch.cat([g.reshape(-1) for g in m.core_grad()])
    torch.cuda.synchronize()
    m.close()
    return G.double().cpu().numpy()


def no_alloc(idx, x, A, B, precision):
    out = torch.full((sum(a.shape[1] for a in A) * B[0].shape[1],), float("nan"),
                     dtype=torch.float32, device=DEV)
    ft.ft_core_grad_noalloc(idx, x, A, B, out, precision=precision)
    return out.double().cpu().numpy()


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16", 1e-5)])
def test_no_alloc_core_grad_matches_context_path(precision, tol):
    first = problem(21, (60, 70, 80), (16, 16, 16), 16, 16 * 300 + 7)
    second = problem(22, (30, 40, 50, 20), (32, 20, 8, 32), 24, 16 * 90 + 3)
    ref1 = with_context(*first, precision)
    ref2 = with_context(*second, precision)
    # two calls in a row on the same inputs, then a call on other inputs (a
    # different shape): the shared scratch must not leak between calls
    for ref, inputs in ((ref1, first), (ref1, first), (ref2, second)):
        got = no_alloc(*inputs, precision)
        assert np.all(np.isfinite(got))
        assert rel_fro(got, ref) <= tol


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_no_alloc_fits_the_largest_shapes(precision):
    """The scratch array holds the partials of every supported shape at the
    grid the context path uses (the largest per-CTA partials: N * K * K at
    K = 32, N = 3..5, and at K = 16, N = 6..10)."""
    for I, J, R in (((9, 10, 11, 12, 13), (32,) * 5, 32), ((9, 10, 11, 12), (32,) * 4, 32),
                    ((9, 10, 11), (32,) * 3, 32), ((5,) * 10, (16,) * 10, 16), ((6,) * 6, (16,) * 6, 16)):
        inputs = problem(24, I, J, R, 16 * 7 + 5)
        ref = with_context(*inputs, precision)
        got = no_alloc(*inputs, precision)
        assert rel_fro(got, ref) <= 1e-5, (len(I), J[0])


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("shape", [((10, 11, 12), (4, 4, 4), 4, 100), ((10, 11, 12, 13), (32, 20, 8, 32), 24, 16 * 9 + 5)],
                         ids=["K16", "K32"])
def test_no_alloc_reports_bad_inputs(precision, shape):
    """This entry point skips the validation pass of ft_init, so the kernel
    itself must mask and report a coordinate outside [0, I_n) (FT_ERR_INDEX)
    and a non-finite value (FT_ERR_NONFINITE); the error word is cleared by
    the next call, whose result is then exact."""
    I, J, R, nnz = shape
    idx, x, A, B = problem(23, I, J, R, nnz)
    out = torch.empty(sum(J) * R, dtype=torch.float32, device=DEV)
    bad = [t.clone() for t in idx]
    bad[2][5] = I[2]
    with pytest.raises(ft.FtError) as e:
        ft.ft_core_grad_noalloc(bad, x, A, B, out, precision=precision)
    assert e.value.status == -2
    ref = with_context(idx, x, A, B, precision)
    ft.ft_core_grad_noalloc(idx, x, A, B, out, precision=precision)
    assert rel_fro(out.double().cpu().numpy(), ref) <= 1e-5
    xn = x.clone()
    xn[7] = float("nan")
    with pytest.raises(ft.FtError) as e:
        ft.ft_core_grad_noalloc(idx, xn, A, B, out, precision=precision)
    assert e.value.status == -5
    ft.ft_core_grad_noalloc(idx, x, A, B, out, precision=precision)
    assert rel_fro(out.double().cpu().numpy(), ref) <= 1e-5
