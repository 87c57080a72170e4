"""Absolute-value error models of the factor step, for elementwise parity.

A floating-point evaluation of the per-nonzero factor gradient
(Eq. "Gradient_low_rank_cp")
    g^(n)_j = -(x - xhat) p^(n)_j + lambda a^(n)_j,   p^(n) = d^(n) B^(n)T
has a forward error bounded, to first order, by a multiple of the unit
roundoff times the same expression evaluated on absolute values:
    scale^(n)_j = (|x - xhat| + xhat_abs) pabs^(n)_j + lambda |a^(n)_j|,
where xhat_abs and pabs are xhat and p computed from |A|, |B| (the residual
carries the rounding error of xhat, whose scale is xhat_abs).  Elementwise
tolerances are stated relative to this scale, so cancellation in the exact
value does not count against the kernel (it would make any relative test
on an entry near zero meaningless).

Every number here comes from the FP64 oracle; nothing from the CUDA path.
"""
from __future__ import annotations

import numpy as np

import oracle


def nonzero_scales(A, B, idx, x, lam):
    """Per nonzero and mode, the vector scale^(n) above: list over modes of
    [nnz, J_n] arrays (float64), at the factors A, B."""
    N = len(A)
    nnz = idx.shape[1]
    Aa = [np.abs(a) for a in A]
    Ba = [np.abs(b) for b in B]
    e = np.abs(np.asarray(x, np.float64) - oracle.predict(A, B, idx)) if nnz else np.zeros(0)
    out = [np.zeros((nnz, a.shape[1])) for a in A]
    for m in range(nnz):
        _, _, pabs, xabs = oracle.nonzero_terms(Aa, Ba, idx, m)
        for n in range(N):
            out[n][m] = (e[m] + xabs) * pabs[n] + lam * Aa[n][idx[n, m]]
    return out


def epoch_step_model(A0, B, idx, x, S, lr, lam, row_scale=None):
    """The batch-synchronous factor epoch of the oracle (batch size S) with,
    for every row, the error scale of its total step and the number of
    batches that touched it.  Returns (A_final, scales, touches): scales[n]
    is lr times the sum, over the row's nonzeros, of their scale^(n) taken
    at the factors of their batch's start (times the row's step multiplier
    when row_scale is given)."""
    A = [np.array(a, np.float64, copy=True) for a in A0]
    N = len(A)
    nnz = idx.shape[1]
    scales = [np.zeros_like(a) for a in A]
    touches = [np.zeros(a.shape[0], np.int64) for a in A]
    x = np.asarray(x, np.float64)
    for lo in range(0, nnz, S):
        hi = min(nnz, lo + S)
        sub = np.ascontiguousarray(idx[:, lo:hi])
        sc = nonzero_scales(A, B, sub, x[lo:hi], lam)
        for n in range(N):
            mult = lr if row_scale is None else lr * np.asarray(row_scale[n], np.float64)[sub[n]][:, None]
            np.add.at(scales[n], sub[n], mult * sc[n])
            touches[n][np.unique(sub[n])] += 1
        A = oracle.factor_epoch(A, B, sub, x[lo:hi], S, lr, lam, row_scale=row_scale)
    return A, scales, touches


def step_errors(A0, A1, ref, scales, touches):
    """Elementwise forward error of the step A1 - A0 against the oracle's
    ref - A0, relative to the error scale.  Each batch that touched a row
    stores it once in float32 (a rounding of up to 2^-24 |a|), which is
    subtracted from the difference first.  Returns the max over all
    touched entries of every mode (0 if none)."""
    worst = 0.0
    for a0, a1, r, s, t in zip(A0, A1, ref, scales, touches):
        a0, a1, r = (np.asarray(v, np.float64) for v in (a0, a1, r))
        store = 2.0 ** -24 * t[:, None] * np.maximum(np.abs(a1), np.abs(r))
        diff = np.maximum(np.abs((a1 - a0) - (r - a0)) - store, 0.0)
        rows = t > 0
        if rows.any():
            worst = max(worst, float(np.max(diff[rows] / np.maximum(s[rows], 1e-300))))
    return worst


def step_errors_floor(A0, A1, ref, touches, floor):
    """Elementwise error of the step A1 - A0 against ref - A0 relative to
    max(|ref step|, floor * RMS of the mode's ref step over touched rows),
    after the float32 storage allowance of step_errors."""
    worst = 0.0
    for a0, a1, r, t in zip(A0, A1, ref, touches):
        a0, a1, r = (np.asarray(v, np.float64) for v in (a0, a1, r))
        rows = t > 0
        if not rows.any():
            continue
        store = 2.0 ** -24 * t[:, None] * np.maximum(np.abs(a1), np.abs(r))
        diff = np.maximum(np.abs((a1 - a0) - (r - a0)) - store, 0.0)[rows]
        st = np.abs(r - a0)[rows]
        rms = float(np.sqrt(np.mean(st * st)))
        worst = max(worst, float(np.max(diff / np.maximum(st, max(floor * rms, 1e-300)))))
    return worst


# Unit roundoff of the inputs of the products in each precision of the path
# (round to nearest: half an ulp of 1): FP32 2^-24, TF32 (10 stored mantissa
# bits) 2^-11, BF16 (7 stored bits) 2^-8.
UNIT_ROUNDOFF = {"fp32": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8}


def rounding_sensitivity(A0, B, idx, x, S, lr, lam, u, seed=0):
    """How far the FP64 oracle's own step moves (the measure of
    step_errors_floor with floor 1: elementwise, relative to max(|step|, RMS
    step of the mode)) when every entry of A and B is perturbed by a relative
    amount of at most u - the error that rounding the inputs to a precision
    of unit roundoff u implies by itself, whatever the arithmetic after it."""
    rng = np.random.default_rng(seed)
    ref = oracle.factor_epoch(A0, B, idx, x, S, lr, lam)
    Ap = [a * (1 + u * rng.uniform(-1, 1, a.shape)) for a in A0]
    Bp = [b * (1 + u * rng.uniform(-1, 1, b.shape)) for b in B]
    got = oracle.factor_epoch(Ap, Bp, idx, x, S, lr, lam)
    worst = 0.0
    for a0, ap, r, g in zip(A0, Ap, ref, got):
        st, sp = r - a0, g - ap
        moved = np.any(st != 0, axis=1)
        if not moved.any():
            continue
        rms = float(np.sqrt(np.mean(st[moved] ** 2)))
        worst = max(worst, float(np.max(np.abs(sp - st)[moved] / np.maximum(np.abs(st[moved]), max(rms, 1e-300)))))
    return worst
