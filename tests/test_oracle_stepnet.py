"""Pins of the oracle's learned-step parts (row statistics, line-search
labels, step-size network) against independent computations:

* counts by np.bincount, residuals and row gradients by central finite
  differences of the row's subproblem loss through the dense Tucker model;
* the label is the log of the exact minimiser along -g of that (quadratic)
  subproblem, recovered from three loss evaluations, over N times the step
  size; and on a tensor whose rows each hold one nonzero, the N rows of a
  nonzero stepping together by their labels remove its residual to first
  order (without the 1/N they would flip its sign: e -> (1 - N) e);
* the network's forward pass equals the textbook MLP written with numpy
  matrix products (linear output u, multiplier exp(clamp(u))), and its
  gradient equals central finite differences of mean 1/2 (u - y)^2 computed
  through that numpy network.
"""
import numpy as np

import oracle
from test_oracle_pins import dense_predict, rand_problem


def row_loss(A, B, idx, x, lam, n, row, a_row):
    """F_r(a) = sum over the row's nonzeros of 1/2 (x - xhat)^2 + 1/2 lam |a|^2."""
    A2 = [a.copy() for a in A]
    A2[n][row] = a_row
    tot = 0.0
    for m in np.nonzero(idx[n] == row)[0]:
        e = x[m] - dense_predict(A2, B, idx[:, m])
        tot += 0.5 * e * e + 0.5 * lam * float(a_row @ a_row)
    return tot


def test_row_stats_against_definitions():
    rng = np.random.default_rng(3)
    N, J, R = 3, (2, 3, 2), 3
    I = [4, 5, 3]
    A, B, idx, x = rand_problem(rng, N, I, J, R, 30, scale=0.6)
    lam, gamma, beta = 0.1, 1.0, 0.3
    ema_in = rng.uniform(0, 1, sum(I))
    feat, lab = oracle.row_stats(A, B, idx, x, lam, gamma, beta, ema_in)
    # most labels inside the clip range, so the formula itself is exercised
    lo, hi = np.log(1 / 16), np.log(16)
    assert np.mean((lab > lo) & (lab < hi)) > 0.8
    xhat = np.array([dense_predict(A, B, idx[:, m]) for m in range(len(x))])
    e = x - xhat
    off = 0
    h = 1e-6
    for n in range(N):
        cnt = np.bincount(idx[n], minlength=I[n])
        for r in range(I[n]):
            q = off + r
            assert np.isclose(feat[q, 0], np.log1p(cnt[r]), rtol=1e-14)
            mean_e = e[idx[n] == r].mean() if cnt[r] else 0.0
            assert np.isclose(feat[q, 2], mean_e, rtol=1e-10, atol=1e-12)
            # row gradient by central differences
            g = np.zeros(J[n])
            for j in range(J[n]):
                ap, am = A[n][r].copy(), A[n][r].copy()
                ap[j] += h
                am[j] -= h
                g[j] = (row_loss(A, B, idx, x, lam, n, r, ap) - row_loss(A, B, idx, x, lam, n, r, am)) / (2 * h)
            gnorm = np.linalg.norm(g) / max(cnt[r], 1)
            ema = beta * ema_in[q] + (1 - beta) * gnorm
            assert np.isclose(feat[q, 1], np.log1p(ema), rtol=1e-6, atol=1e-9)
            # exact line search along -g from three loss values (F is quadratic in t)
            if cnt[r] == 0 or np.linalg.norm(g) < 1e-12:
                assert lab[q] == 0.0
                continue
            dlt = 1e-3
            f0 = row_loss(A, B, idx, x, lam, n, r, A[n][r])
            fp = row_loss(A, B, idx, x, lam, n, r, A[n][r] - dlt * g)
            fm = row_loss(A, B, idx, x, lam, n, r, A[n][r] + dlt * g)
            t_star = dlt * (fm - fp) / (2 * (fp - 2 * f0 + fm))
            want = float(np.log(np.clip(t_star / (N * gamma), 1 / 16, 16)))
            assert np.isclose(lab[q], want, rtol=1e-5, atol=1e-6), (n, r, lab[q], want)
        off += I[n]


def test_labels_share_the_step_among_the_modes():
    """Every row holds one nonzero and lambda = 0, so each row's exact step
    alone would remove its nonzero's residual.  The N rows of a nonzero
    stepping together by gamma exp(label) g (g by central differences of the
    dense model) leave a residual of second order in e; the same steps
    without the 1/N leave (1 - N) e."""
    rng = np.random.default_rng(11)
    for N, J, R in [(3, (2, 3, 2), 3), (4, (2, 2, 3, 2), 2)]:
        M = 12
        I = [M] * N
        A = [rng.normal(0, 0.8, (M, J[n])) for n in range(N)]
        B = [rng.normal(0, 0.8, (J[n], R)) for n in range(N)]
        idx = np.stack([rng.permutation(M) for _ in range(N)]).astype(np.int32)
        xhat = np.array([dense_predict(A, B, idx[:, m]) for m in range(M)])
        e = 1e-3 * rng.choice([-1.0, 1.0], M) * (1 + rng.uniform(0, 1, M))
        x = xhat + e
        gamma = 1.0
        _, lab = oracle.row_stats(A, B, idx, x, 0.0, gamma, 0.0, None)
        lo, hi = np.log(1 / 16), np.log(16)
        checked = 0
        h = 1e-6
        for m in range(M):
            q = [n * M + idx[n, m] for n in range(N)]
            if not all(lo + 1e-9 < lab[v] < hi - 1e-9 for v in q):
                continue
            steps = []
            for n in range(N):
                r = idx[n, m]
                dx = np.zeros(J[n])
                for j in range(J[n]):
                    Ap = [a.copy() for a in A]
                    Am = [a.copy() for a in A]
                    Ap[n][r, j] += h
                    Am[n][r, j] -= h
                    dx[j] = (dense_predict(Ap, B, idx[:, m]) - dense_predict(Am, B, idx[:, m])) / (2 * h)
                g = -e[m] * dx
                steps.append(gamma * np.exp(lab[q[n]]) * g)
            # second-order terms grow with the step: 2% of e for the shared
            # steps, 10% for the N times larger ones (both far from the
            # other case's value, |(1 - N) e| >= 2 |e|)
            for mult, want, tol in ((1.0, 0.0, 2e-2), (float(N), (1 - N) * e[m], 1e-1)):
                A2 = [a.copy() for a in A]
                for n in range(N):
                    A2[n][idx[n, m]] -= mult * steps[n]
                e2 = x[m] - dense_predict(A2, B, idx[:, m])
                assert abs(e2 - want) <= tol * abs(e[m]), (N, m, mult, e2, want, e[m])
            checked += 1
        assert checked >= M // 2, checked


def mlp_numpy_raw(P, X):
    """The textbook 3 -> 64 -> 64 -> 1 ReLU network with a linear output."""
    H = 64
    W1 = P[:H * 3].reshape(H, 3)
    b1 = P[H * 3:H * 4]
    W2 = P[H * 4:H * 4 + H * H].reshape(H, H)
    b2 = P[H * 4 + H * H:H * 5 + H * H]
    w3 = P[H * 5 + H * H:H * 6 + H * H]
    b3 = P[H * 6 + H * H]
    h1 = np.maximum(0.0, X @ W1.T + b1)
    h2 = np.maximum(0.0, h1 @ W2.T + b2)
    return h2 @ w3 + b3


def test_mlp_forward_is_the_textbook_network():
    rng = np.random.default_rng(4)
    P = rng.normal(0, 0.3, oracle.mlp_nparams())
    X = rng.normal(0, 1, (50, 3))
    u = mlp_numpy_raw(P, X)
    # both sides of the clamp are exercised
    assert np.any(np.abs(u) < np.log(16)) and np.any(np.abs(u) > np.log(16))
    want = np.exp(np.clip(u, np.log(1 / 16), np.log(16)))
    np.testing.assert_allclose(oracle.mlp_forward(P, X), want, rtol=1e-12)


def test_mlp_gradient_by_central_differences():
    rng = np.random.default_rng(5)
    n_par = oracle.mlp_nparams()
    P = rng.normal(0, 0.3, n_par)
    X = rng.normal(0, 1, (20, 3))
    y = rng.uniform(np.log(1 / 16), np.log(16), 20)

    def loss(Pv):
        return float(np.mean(0.5 * (mlp_numpy_raw(Pv, X) - y) ** 2))

    G, L = oracle.mlp_grad(P, X, y)
    assert np.isclose(L, loss(P), rtol=1e-12)
    h = 1e-6
    pick = np.concatenate([np.arange(0, 192, 17), np.arange(192, 256, 7), np.arange(256, 4352, 97),
                           np.arange(4352, 4481, 11), [4480]])
    for q in pick:
        Pp, Pm = P.copy(), P.copy()
        Pp[q] += h
        Pm[q] -= h
        fd = (loss(Pp) - loss(Pm)) / (2 * h)
        assert np.isclose(G[q], fd, rtol=1e-5, atol=1e-9), q


STEPNET_PINS = [test_row_stats_against_definitions, test_mlp_forward_is_the_textbook_network,
                test_mlp_gradient_by_central_differences,
                test_labels_share_the_step_among_the_modes]
STEPNET_MUTANTS = [
    ("label_without_regulariser_curvature", "double den = hsum[q] + lambda * k * gg;", "double den = hsum[q];"),
    ("relu_derivative_dropped", "double dh2 = h2[i] > 0.0 ? dz * w3[i] : 0.0;", "double dh2 = dz * w3[i];"),
    ("output_clamp_wrong", "if (u > log(ORC_SMAX)) u = log(ORC_SMAX);", "if (u > log(4.0)) u = log(4.0);"),
    ("loss_gradient_halved", "double dz = r / (double)n;", "double dz = 0.5 * r / (double)n;"),
    ("row_gradient_sign", "g[goff[n] + row * J[n] + j] += -e * pj + lambda * a[j];",
     "g[goff[n] + row * J[n] + j] += e * pj + lambda * a[j];"),
    ("mean_residual_not_divided", "feat[3 * q + 2] = k > 0.0 ? esum[q] / k : 0.0;", "feat[3 * q + 2] = esum[q];"),
    ("label_step_not_shared", "s = gg / den / ((double)N * gamma);", "s = gg / den / gamma;"),
]


def test_planted_mistakes_break_a_stepnet_pin(tmp_path):
    import subprocess
    src = open(oracle._SRC).read()
    survivors = []
    for name, old, new in STEPNET_MUTANTS:
        assert src.count(old) == 1, f"mutation anchor for {name} not found"
        msrc = tmp_path / f"{name}.c"
        msrc.write_text(src.replace(old, new, 1))
        so = tmp_path / f"{name}.so"
        subprocess.run(["gcc", *oracle.CFLAGS, str(msrc), "-o", str(so), "-lm"], check=True)
        caught = False
        with oracle.use_library(str(so)):
            for pin in STEPNET_PINS:
                try:
                    pin()
                except AssertionError:
                    caught = True
                    break
        if not caught:
            survivors.append(name)
    assert not survivors, survivors
