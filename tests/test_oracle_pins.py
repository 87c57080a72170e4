"""Pins of the FP64 CPU oracle against things other than itself.

Each pin ties one part of the oracle to a fact the paper or the mathematics
fixes independently of the oracle's code:

* the prediction of Eq. "fasttucker" equals a brute-force dense Tucker
  reconstruction (Eq. "tucker" with the R-Kruskal core of Eq.
  "fasttucker_core_tensor") built with numpy outer products and contractions;
* the per-nonzero factor and core gradients (Eqs. "Gradient_low_rank_cp",
  "Gradient_core_tensor_cp") equal central finite differences of
  1/2 (x - xhat)^2 + 1/2 lambda ||.||^2 evaluated through that dense model;
* with B^(n) = I and J = R the factor epoch is textbook CP-SGD, and with N = 2
  textbook matrix-factorisation SGD (coded here from their own definitions);
* a batch of S = nnz equals one step along the sum of finite-difference
  gradients, taken from the batch-start factors (Algorithm 3/4 snapshot);
* invariants: batch size does not matter when no two nonzeros share a row; a
  duplicated nonzero doubles the batch step; at an exact planted model with
  lambda = 0 nothing moves and with lambda > 0 rows only shrink;
* the intermediates of one nonzero (c^(n), d^(n), p^(n) = d^(n) B^(n)T, xhat)
  equal dense predictions of reduced models, and p^(n) equals the finite-
  difference gradient of xhat with respect to a^(n);
* hand-worked scalar examples (tests/golden/hand_worked.json);
* RMSE/MAE by their definitions with math.fsum;
* planted-model recovery.

A final test plants mistakes in copies of the oracle source and checks that
each one breaks at least one pin.
"""
import json
import math
import os
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


# --------------------------------------------------------------- independent
def dense_core(B):
    """G = sum_r b^(1)_r o ... o b^(N)_r (Def. "R Kruskal Product")."""
    R = B[0].shape[1]
    G = np.zeros([b.shape[0] for b in B])
    for r in range(R):
        t = B[0][:, r]
        for b in B[1:]:
            t = np.multiply.outer(t, b[:, r])
        G = G + t
    return G


def dense_predict(A, B, coord):
    """G x_1 a^(1)_{i1} ... x_N a^(N)_{iN} (Eq. "tucker")."""
    v = dense_core(B)
    for n, a in enumerate(A):
        v = np.tensordot(a[coord[n]], v, axes=([0], [0]))
    return float(v)


def rand_problem(rng, N, I, J, R, nnz, scale=0.7):
    A = [rng.normal(0, scale, (I[n], J[n])) for n in range(N)]
    B = [rng.normal(0, scale, (J[n], R)) for n in range(N)]
    idx = np.stack([rng.integers(0, I[n], nnz) for n in range(N)]).astype(np.int32)
    x = rng.normal(0, 1, nnz)
    return A, B, idx, x


# ---------------------------------------------------------------------- pins
def pin_predict_dense(seed=0):
    rng = np.random.default_rng(seed)
    for N, J, R in [(2, (3, 2), 4), (3, (2, 3, 4), 3), (4, (2, 2, 3, 2), 5), (3, (1, 1, 1), 1)]:
        I = [5 + n for n in range(N)]
        A, B, idx, _ = rand_problem(rng, N, I, J, R, 12)
        got = oracle.predict(A, B, idx)
        want = [dense_predict(A, B, idx[:, m]) for m in range(idx.shape[1])]
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def pin_factor_grad_fd(seed=1):
    rng = np.random.default_rng(seed)
    h = 1e-6
    for N, J, R in [(3, (2, 3, 2), 3), (4, (2, 2, 2, 3), 2), (2, (3, 4), 5)]:
        I = [4] * N
        A, B, idx, x = rand_problem(rng, N, I, J, R, 5)
        lam = 0.3
        for m in range(idx.shape[1]):
            g = oracle.factor_grads(A, B, idx, m, x[m], lam)
            for n in range(N):
                row = idx[n, m]
                fd = np.empty(J[n])
                for j in range(J[n]):
                    vals = []
                    for sgn in (+1, -1):
                        Ap = [a.copy() for a in A]
                        Ap[n][row, j] += sgn * h
                        e = x[m] - dense_predict(Ap, B, idx[:, m])
                        vals.append(0.5 * e * e + 0.5 * lam * np.dot(Ap[n][row], Ap[n][row]))
                    fd[j] = (vals[0] - vals[1]) / (2 * h)
                np.testing.assert_allclose(g[n], fd, rtol=1e-6, atol=1e-7)


def pin_nonzero_terms_dense(seed=13):
    """Every intermediate of one nonzero against the dense model (Eq. "tucker"
    with the Kruskal core), never against the oracle's own formulas:
      * c^(n)_r is the dense prediction of a model that keeps column r of
        B^(n) and replaces every other mode by the scalar 1 (J_k = R = 1);
      * d^(n)_r is the dense prediction of the rank-1 model made of column r
        of every B^(k), with mode n replaced by the scalar 1;
      * p^(n) = d^(n) B^(n)T is the gradient of xhat with respect to a^(n)
        (central differences through the dense model);
      * xhat = a^(n) . p^(n) for every n (xhat is linear in each a^(n)) and
        equals the dense prediction."""
    rng = np.random.default_rng(seed)
    h = 1e-6
    one_a, one_b = np.ones((1, 1)), np.ones((1, 1))
    for N, J, R in [(3, (2, 3, 4), 3), (4, (2, 2, 3, 2), 4), (2, (3, 1), 2), (1, (3,), 2)]:
        I = [4 + n for n in range(N)]
        A, B, idx, _ = rand_problem(rng, N, I, J, R, 4)
        for m in range(idx.shape[1]):
            c, d, p, xhat = oracle.nonzero_terms(A, B, idx, m)
            coord = idx[:, m]
            assert math.isclose(xhat, dense_predict(A, B, coord), rel_tol=1e-12, abs_tol=1e-13)
            for n in range(N):
                for r in range(R):
                    As = [A[k] if k == n else one_a for k in range(N)]
                    Bs = [B[k][:, [r]] if k == n else one_b for k in range(N)]
                    cs = [coord[k] if k == n else 0 for k in range(N)]
                    assert math.isclose(c[n, r], dense_predict(As, Bs, cs), rel_tol=1e-12, abs_tol=1e-13)
                    As = [one_a if k == n else A[k] for k in range(N)]
                    Bs = [one_b if k == n else B[k][:, [r]] for k in range(N)]
                    cs = [0 if k == n else coord[k] for k in range(N)]
                    assert math.isclose(d[n, r], dense_predict(As, Bs, cs), rel_tol=1e-12, abs_tol=1e-13)
                fd = np.empty(J[n])
                for j in range(J[n]):
                    vals = []
                    for sgn in (+1, -1):
                        Ap = [a.copy() for a in A]
                        Ap[n][coord[n], j] += sgn * h
                        vals.append(dense_predict(Ap, B, coord))
                    fd[j] = (vals[0] - vals[1]) / (2 * h)
                np.testing.assert_allclose(p[n], fd, rtol=1e-6, atol=1e-8)
                assert math.isclose(float(np.dot(A[n][coord[n]], p[n])), xhat, rel_tol=1e-12, abs_tol=1e-13)


def pin_core_grad_fd(seed=2):
    rng = np.random.default_rng(seed)
    h = 1e-6
    N, J, R = 3, (2, 3, 2), 3
    A, B, idx, x = rand_problem(rng, N, [4, 5, 3], J, R, 9)

    def loss(Bs):
        return sum(0.5 * (x[m] - dense_predict(A, Bs, idx[:, m])) ** 2 for m in range(len(x)))

    G = oracle.core_grad(A, B, idx, x)
    for n in range(N):
        fd = np.empty((J[n], R))
        for j in range(J[n]):
            for r in range(R):
                Bp = [b.copy() for b in B]
                Bm = [b.copy() for b in B]
                Bp[n][j, r] += h
                Bm[n][j, r] -= h
                fd[j, r] = (loss(Bp) - loss(Bm)) / (2 * h)
        np.testing.assert_allclose(G[n], fd, rtol=1e-6, atol=1e-7)


def pin_core_epoch_step(seed=3):
    """Algorithm 5's step is gradient descent on sum(1/2 e^2)/|Omega| + 1/2 lambda||B||^2."""
    rng = np.random.default_rng(seed)
    h = 1e-6
    N, J, R = 3, (2, 2, 3), 2
    A, B, idx, x = rand_problem(rng, N, [3, 4, 5], J, R, 7)
    gamma, lam = 0.05, 0.2
    nnz = len(x)

    def obj(Bs):
        s = sum(0.5 * (x[m] - dense_predict(A, Bs, idx[:, m])) ** 2 for m in range(nnz))
        return s / nnz + 0.5 * lam * sum(float((b * b).sum()) for b in Bs)

    Bn = oracle.core_epoch(A, B, idx, x, gamma, lam)
    for n in range(N):
        fd = np.empty((J[n], R))
        for j in range(J[n]):
            for r in range(R):
                Bp = [b.copy() for b in B]
                Bm = [b.copy() for b in B]
                Bp[n][j, r] += h
                Bm[n][j, r] -= h
                fd[j, r] = (obj(Bp) - obj(Bm)) / (2 * h)
        np.testing.assert_allclose(Bn[n], B[n] - gamma * fd, rtol=1e-7, atol=1e-8)


def pin_core_sgd_sets(seed=12):
    """Per-set core SGD (Algorithm 3's core loop): each consecutive set of S
    nonzeros is a gradient step on its own averaged objective
    sum_Psi(1/2 e^2)/|Psi| + 1/2 lambda ||B||^2, by central differences
    through the dense model, taken from the core matrices left by the
    previous set (S = 1: one rule-"Update_FastTuckerPlus_core" step per
    nonzero; a ragged last set)."""
    rng = np.random.default_rng(seed)
    h = 1e-6
    N, J, R = 3, (2, 3, 2), 2
    A, B, idx, x = rand_problem(rng, N, [3, 4, 3], J, R, 7)
    gamma, lam = 0.1, 0.15
    for S in (1, 3):
        want = [b.copy() for b in B]
        for lo in range(0, len(x), S):
            ms = range(lo, min(lo + S, len(x)))

            def obj(Bs):
                s = sum(0.5 * (x[m] - dense_predict(A, Bs, idx[:, m])) ** 2 for m in ms)
                return s / len(ms) + 0.5 * lam * sum(float((b * b).sum()) for b in Bs)

            step = []
            for n in range(N):
                fd = np.empty((J[n], R))
                for j in range(J[n]):
                    for r in range(R):
                        Bp = [b.copy() for b in want]
                        Bm = [b.copy() for b in want]
                        Bp[n][j, r] += h
                        Bm[n][j, r] -= h
                        fd[j, r] = (obj(Bp) - obj(Bm)) / (2 * h)
                step.append(gamma * fd)
            want = [b - st for b, st in zip(want, step)]
        got = oracle.core_epoch_sgd(A, B, idx, x, S, gamma, lam)
        for n in range(N):
            np.testing.assert_allclose(got[n], want[n], rtol=1e-7, atol=1e-8)


def pin_cp_special_case(seed=4):
    """B = I, J = R: one sequential epoch is CP-SGD on x ~ sum_r prod_n a^(n)_r."""
    rng = np.random.default_rng(seed)
    N, R = 3, 3
    I = [6, 5, 4]
    A = [rng.normal(0, 0.6, (I[n], R)) for n in range(N)]
    B = [np.eye(R) for _ in range(N)]
    nnz = 40
    idx = np.stack([rng.integers(0, I[n], nnz) for n in range(N)]).astype(np.int32)
    x = rng.normal(0, 1, nnz)
    gamma, lam = 0.05, 0.1
    got = oracle.factor_epoch(A, B, idx, x, 1, gamma, lam)
    W = [a.copy() for a in A]
    for m in range(nnz):
        rows = [W[n][idx[n, m]].copy() for n in range(N)]
        e = x[m] - float(np.sum(np.prod(np.stack(rows), axis=0)))
        for n in range(N):
            others = np.prod(np.stack([rows[k] for k in range(N) if k != n]), axis=0)
            W[n][idx[n, m]] = rows[n] + gamma * (e * others - lam * rows[n])
    for n in range(N):
        np.testing.assert_allclose(got[n], W[n], rtol=1e-12, atol=1e-13)


def pin_mf_special_case(seed=5):
    """N = 2, B = I: one sequential epoch is matrix-factorisation SGD (x ~ u.v)."""
    rng = np.random.default_rng(seed)
    R = 4
    U = rng.normal(0, 0.5, (7, R))
    V = rng.normal(0, 0.5, (9, R))
    nnz = 50
    iu = rng.integers(0, 7, nnz)
    iv = rng.integers(0, 9, nnz)
    x = rng.normal(0, 1, nnz)
    gamma, lam = 0.07, 0.02
    got = oracle.factor_epoch([U, V], [np.eye(R), np.eye(R)], np.stack([iu, iv]).astype(np.int32),
                              x, 1, gamma, lam)
    U2, V2 = U.copy(), V.copy()
    for m in range(nnz):
        u, v = U2[iu[m]].copy(), V2[iv[m]].copy()
        e = x[m] - u @ v
        U2[iu[m]] = u + gamma * (e * v - lam * u)
        V2[iv[m]] = v + gamma * (e * u - lam * v)
    np.testing.assert_allclose(got[0], U2, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(got[1], V2, rtol=1e-12, atol=1e-13)


def pin_full_batch_is_sum_of_fd_grads(seed=6):
    """S = nnz: A_new = A - gamma * sum_m g_m, every g_m a finite difference
    taken at the batch-start factors."""
    rng = np.random.default_rng(seed)
    h = 1e-6
    N, J, R = 3, (2, 3, 2), 2
    I = [3, 3, 4]
    A, B, idx, x = rand_problem(rng, N, I, J, R, 8)
    gamma, lam = 0.1, 0.05
    got = oracle.factor_epoch(A, B, idx, x, len(x), gamma, lam)
    want = [a.copy() for a in A]
    for m in range(len(x)):
        for n in range(N):
            row = idx[n, m]
            for j in range(J[n]):
                vals = []
                for sgn in (+1, -1):
                    Ap = [a.copy() for a in A]
                    Ap[n][row, j] += sgn * h
                    e = x[m] - dense_predict(Ap, B, idx[:, m])
                    vals.append(0.5 * e * e + 0.5 * lam * np.dot(Ap[n][row], Ap[n][row]))
                want[n][row, j] -= gamma * (vals[0] - vals[1]) / (2 * h)
    for n in range(N):
        np.testing.assert_allclose(got[n], want[n], rtol=1e-6, atol=1e-8)


def pin_disjoint_rows_batch_invariance(seed=7):
    rng = np.random.default_rng(seed)
    N, J, R = 3, (3, 2, 4), 3
    nnz = 10
    I = [nnz, nnz + 2, nnz + 5]
    A = [rng.normal(0, 0.5, (I[n], J[n])) for n in range(N)]
    B = [rng.normal(0, 0.5, (J[n], R)) for n in range(N)]
    idx = np.stack([rng.permutation(I[n])[:nnz] for n in range(N)]).astype(np.int32)
    x = rng.normal(0, 1, nnz)
    ref = oracle.factor_epoch(A, B, idx, x, 1, 0.1, 0.05)
    for S in (2, 3, nnz, 10 * nnz):
        got = oracle.factor_epoch(A, B, idx, x, S, 0.1, 0.05)
        for n in range(N):
            np.testing.assert_array_equal(got[n], ref[n])


def pin_duplicate_doubles_step(seed=8):
    rng = np.random.default_rng(seed)
    N, J, R = 3, (2, 2, 3), 2
    A, B, idx, x = rand_problem(rng, N, [3, 3, 3], J, R, 1)
    one = oracle.factor_epoch(A, B, idx, x, 2, 0.1, 0.3)
    two = oracle.factor_epoch(A, B, np.concatenate([idx, idx], axis=1), np.concatenate([x, x]),
                              2, 0.1, 0.3)
    for n in range(N):
        np.testing.assert_allclose(two[n] - A[n], 2 * (one[n] - A[n]), rtol=1e-12, atol=1e-14)


def pin_planted_fixed_point(seed=9):
    rng = np.random.default_rng(seed)
    N, J, R = 3, (3, 2, 2), 3
    A, B, idx, _ = rand_problem(rng, N, [5, 6, 7], J, R, 30)
    x = np.array([dense_predict(A, B, idx[:, m]) for m in range(idx.shape[1])])
    # lambda = 0: the error is zero up to rounding, so nothing moves
    got = oracle.factor_epoch(A, B, idx, x, 4, 0.2, 0.0)
    for n in range(N):
        np.testing.assert_allclose(got[n], A[n], rtol=0, atol=1e-12)
    Bn = oracle.core_epoch(A, B, idx, x, 0.2, 0.0)
    for n in range(N):
        np.testing.assert_allclose(Bn[n], B[n], rtol=0, atol=1e-12)
    # lambda > 0, one nonzero per batch touching each row once: each row
    # shrinks by exactly (1 - gamma lambda) in its first batch
    gamma, lam = 0.2, 0.5
    idx1 = idx[:, :1]
    got = oracle.factor_epoch(A, B, idx1, x[:1], 1, gamma, lam)
    for n in range(N):
        want = A[n].copy()
        want[idx1[n, 0]] *= (1 - gamma * lam)
        np.testing.assert_allclose(got[n], want, rtol=1e-12, atol=1e-12)
    Bn = oracle.core_epoch(A, B, idx, x, gamma, lam)
    for n in range(N):
        np.testing.assert_allclose(Bn[n], B[n] * (1 - gamma * lam), rtol=1e-10, atol=1e-12)


def pin_hand_worked():
    with open(os.path.join(HERE, "golden", "hand_worked.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        A = [np.array(a, dtype=np.float64) for a in c["A"]]
        B = [np.array(b, dtype=np.float64) for b in c["B"]]
        idx = np.array(c["coords"], dtype=np.int32)
        x = np.array(c["x"], dtype=np.float64)
        if "xhat" in c:
            np.testing.assert_allclose(oracle.predict(A, B, idx), c["xhat"], rtol=1e-15)
        if "A_after" in c:
            got = oracle.factor_epoch(A, B, idx, x, c["S"], c["gamma"], c["lambda"])
            for n, want in enumerate(c["A_after"]):
                np.testing.assert_allclose(got[n], np.array(want), rtol=1e-13, err_msg=c["name"])
        if "G" in c:
            G = oracle.core_grad(A, B, idx, x)
            for n, want in enumerate(c["G"]):
                np.testing.assert_allclose(G[n], np.array(want), rtol=1e-15, err_msg=c["name"])
        if "B_after" in c:
            got = oracle.core_epoch(A, B, idx, x, c["gamma"], c["lambda"])
            for n, want in enumerate(c["B_after"]):
                np.testing.assert_allclose(got[n], np.array(want), rtol=1e-13, err_msg=c["name"])


def pin_errors_definition(seed=10):
    rng = np.random.default_rng(seed)
    N, J, R = 3, (2, 3, 2), 2
    A, B, idx, x = rand_problem(rng, N, [4, 4, 4], J, R, 25)
    rmse, mae, sse = oracle.errors(A, B, idx, x)
    e = [x[m] - dense_predict(A, B, idx[:, m]) for m in range(len(x))]
    assert math.isclose(sse, math.fsum(v * v for v in e), rel_tol=1e-12)
    assert math.isclose(rmse, math.sqrt(math.fsum(v * v for v in e) / len(e)), rel_tol=1e-12)
    assert math.isclose(mae, math.fsum(abs(v) for v in e) / len(e), rel_tol=1e-12)
    lam_a, lam_b = 0.3, 0.7
    obj = oracle.objective(A, B, idx, x, lam_a, lam_b)
    want = (math.fsum(v * v for v in e) + lam_a * sum(float((a * a).sum()) for a in A)
            + lam_b * sum(float((b * b).sum()) for b in B))
    assert math.isclose(obj, want, rel_tol=1e-12)
    # threaded reductions agree with the single-thread order up to rounding
    r4 = oracle.errors(A, B, idx, x, nthreads=4)
    assert math.isclose(r4[2], sse, rel_tol=1e-13)
    G1 = oracle.core_grad(A, B, idx, x, nthreads=1)
    G3 = oracle.core_grad(A, B, idx, x, nthreads=3)
    for g1, g3 in zip(G1, G3):
        np.testing.assert_allclose(g3, g1, rtol=1e-12, atol=1e-14)


def pin_planted_recovery(seed=11):
    """Training on noiseless data of a planted model from a nearby start drives
    the test RMSE down by orders of magnitude."""
    rng = np.random.default_rng(seed)
    N, J, R = 3, (2, 2, 2), 2
    I = [12, 12, 12]
    At = [rng.normal(0, 0.8, (I[n], J[n])) for n in range(N)]
    Bt = [rng.normal(0, 0.8, (J[n], R)) for n in range(N)]
    nnz = 1500
    idx = np.stack([rng.integers(0, I[n], nnz) for n in range(N)]).astype(np.int32)
    x = oracle.predict(At, Bt, idx)
    A = [a + rng.normal(0, 0.05, a.shape) for a in At]
    B = [b.copy() for b in Bt]
    r0 = oracle.errors(A, B, idx, x)[0]
    for _ in range(30):
        A = oracle.factor_epoch(A, B, idx, x, 1, 0.05, 0.0)
        B = oracle.core_epoch(A, B, idx, x, 0.05, 0.0)
    r1 = oracle.errors(A, B, idx, x)[0]
    assert r1 < 0.05 * r0, (r0, r1)


PINS = [pin_predict_dense, pin_nonzero_terms_dense, pin_factor_grad_fd, pin_core_grad_fd, pin_core_epoch_step, pin_core_sgd_sets,
        pin_cp_special_case, pin_mf_special_case, pin_full_batch_is_sum_of_fd_grads,
        pin_disjoint_rows_batch_invariance, pin_duplicate_doubles_step,
        pin_planted_fixed_point, pin_hand_worked, pin_errors_definition, pin_planted_recovery]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


# Mistakes planted in copies of the oracle source: (name, exact text, replacement).
MUTANTS = [
    ("dropped_lambda_in_factor_update", "g[j] += -e * dbt + lambda * a[j];", "g[j] += -e * dbt;"),
    ("flipped_error_sign", "double e = x[m] - orc_xhat(N, R, c);\n      for (int n = 0; n < N; ++n) {\n        int64_t row",
     "double e = orc_xhat(N, R, c) - x[m];\n      for (int n = 0; n < N; ++n) {\n        int64_t row"),
    ("leave_one_out_keeps_own_mode", "if (k != n) p *= c[k * R + r];", "p *= c[k * R + r];"),
    ("transposed_core_in_c", "s += a[j] * B[n][(int64_t)j * R + r];", "s += a[j] * B[n][(int64_t)r * J[n] + j];"),
    ("core_grad_wrong_mode_row", "gp[off + (int64_t)j * R + r] += ne * a[j] * d[n * R + r];",
     "gp[off + (int64_t)j * R + r] += ne * a[j] * d[((n + 1) % N) * R + r];"),
    ("core_step_missing_mean", "double gq = nnz > 0 ? G[n][q] / (double)nnz : 0.0;", "double gq = G[n][q];"),
    ("batch_overwrites_instead_of_summing", "g[j] += -e * dbt + lambda * a[j];",
     "g[j] = -e * dbt + lambda * a[j];"),
    ("update_sign_flipped", "a[j] -= gamma * s * g[j];", "a[j] += gamma * s * g[j];"),
    ("mae_squared", "ae += fabs(e);", "ae += e * e;"),
    ("core_sgd_values_of_first_set", "x + lo, gamma, lambda, nthreads);", "x, gamma, lambda, nthreads);"),
    ("back_projection_uses_c_not_d",
     "for (int r = 0; r < R; ++r) s += d[n * R + r] * B[n][(int64_t)j * R + r];\n      p[off + j] = s;",
     "for (int r = 0; r < R; ++r) s += c[n * R + r] * B[n][(int64_t)j * R + r];\n      p[off + j] = s;"),
    ("core_sgd_first_set_only", "for (int64_t lo = 0; lo < nnz; lo += S) {",
     "for (int64_t lo = 0; lo < nnz && lo < S; lo += S) {"),
]


def test_planted_mistakes_break_a_pin(tmp_path):
    src = open(oracle._SRC).read()
    survivors = []
    for name, old, new in MUTANTS:
        assert src.count(old) >= 1, f"mutation anchor for {name} not found"
        msrc = tmp_path / f"{name}.c"
        msrc.write_text(src.replace(old, new, 1))
        so = tmp_path / f"{name}.so"
        subprocess.run(["gcc", *oracle.CFLAGS, str(msrc), "-o", str(so), "-lm"], check=True)
        caught = False
        with oracle.use_library(str(so)):
            for pin in PINS:
                try:
                    pin()
                except AssertionError:
                    caught = True
                    break
        if not caught:
            survivors.append(name)
    assert not survivors, f"planted mistakes no pin caught: {survivors}"


def test_hogwild_timing_epoch_is_the_sequential_epoch():
    """The host Hogwild epoch (timing of the CPU baseline only) runs the same
    rule: on one thread it is the sequential epoch (S = 1) bit for bit, also
    with rows shared by many nonzeros; on several threads, when no two
    nonzeros share a row, it is again the sequential epoch bit for bit."""
    rng = np.random.default_rng(14)
    N, J, R = 3, (3, 4, 2), 3
    A, B, idx, x = rand_problem(rng, N, [6, 5, 7], J, R, 60)
    one = oracle.factor_epoch_hogwild(A, B, idx, x, 0.05, 0.1, nthreads=1)
    seq = oracle.factor_epoch(A, B, idx, x, 1, 0.05, 0.1)
    for n in range(N):
        np.testing.assert_array_equal(one[n], seq[n])
    nnz = 40
    I = [nnz + 3, nnz + 1, nnz + 8]
    A = [rng.normal(0, 0.5, (I[n], J[n])) for n in range(N)]
    idx = np.stack([rng.permutation(I[n])[:nnz] for n in range(N)]).astype(np.int32)
    x = rng.normal(0, 1, nnz)
    many = oracle.factor_epoch_hogwild(A, B, idx, x, 0.05, 0.1, nthreads=4)
    seq = oracle.factor_epoch(A, B, idx, x, 1, 0.05, 0.1)
    for n in range(N):
        np.testing.assert_array_equal(many[n], seq[n])
