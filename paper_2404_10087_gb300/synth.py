"""Seeded synthetic inputs for sparse FastTucker workloads.

This module only draws random data: coordinates (uniform or Zipf-skewed per
mode), planted factor and core matrices, noise, train/test splits and the
rating map for integer-valued tensors.  It holds none of the method's
arithmetic: the values of a planted tensor are the planted model's
predictions, and those are computed by whoever consumes the draw (the CPU
oracle in the tests, the library's own predict call in the benchmark).

Workload shapes follow the paper's experiments (Sec. 5.1, Table "Datasets"):
a Netflix-shaped 3-order tensor (480,189 x 17,770 x 2,182 users x movies x
days, about 1e8 ratings in 1..5), a Yahoo!Music-shaped tensor, and the
synthetic order-3..10 tensors.  The real datasets are not available, so
skewed (Zipf) index popularity stands in for their structure.

Everything is driven by torch generators so that the large draws run on the
device; the small ones run on the CPU with the same code.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch


def generator(seed: int, device="cpu") -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def zipf_cdf(I: int, s: float, device="cpu") -> torch.Tensor:
    """Cumulative distribution of a Zipf law truncated to ranks 1..I (float64)."""
    k = torch.arange(1, I + 1, dtype=torch.float64, device=device)
    p = k.pow(-float(s))
    c = torch.cumsum(p, 0)
    return c / c[-1]


def draw_mode_indices(gen: torch.Generator, I: int, nnz: int, dist: str = "uniform",
                      s: float = 1.1, device="cpu") -> torch.Tensor:
    """Draw nnz row indices in [0, I) for one mode (int64).

    ``uniform``: i.i.d. uniform rows.  ``zipf``: the rank of each draw follows
    a truncated Zipf(s) law (inverse CDF on the precomputed table) and ranks
    are mapped to row ids through a seeded random permutation, so that hot rows
    are scattered over the matrix rather than packed at its top.
    """
    if dist == "uniform":
        return torch.randint(0, I, (nnz,), generator=gen, device=device, dtype=torch.int64)
    if dist != "zipf":
        raise ValueError(f"unknown index distribution {dist!r}")
    cdf = zipf_cdf(I, s, device=device)
    u = torch.rand(nnz, generator=gen, device=device, dtype=torch.float64)
    rank = torch.searchsorted(cdf, u).clamp_(max=I - 1)
    ids = torch.randperm(I, generator=gen, device=device)
    return ids[rank]


def dedup_coords(idx: torch.Tensor) -> torch.Tensor:
    """Drop repeated coordinates, keeping the first occurrence of each.

    idx: [N, nnz] int64.  The surviving columns keep their original order
    (which is random, so the result is still a random sample order).
    Uses N stable sorts (lexicographic order by mode N, ..., 1) so that no
    linearised key can overflow for large mode sizes.
    """
    N, nnz = idx.shape
    if nnz == 0:
        return idx
    order = torch.arange(nnz, device=idx.device)
    for n in reversed(range(N)):
        _, o = torch.sort(idx[n, order], stable=True)
        order = order[o]
    srt = idx[:, order]
    same = torch.ones(nnz, dtype=torch.bool, device=idx.device)
    same[0] = False
    same[1:] = (srt[:, 1:] == srt[:, :-1]).all(dim=0)
    keep_pos = order[~same]
    keep_pos, _ = torch.sort(keep_pos)
    return idx[:, keep_pos]


def draw_unique_coords(gen: torch.Generator, I, target: int, dist: str, s: float, device="cpu",
                       max_rounds: int = 12) -> torch.Tensor:
    """``target`` distinct coordinates ([N, target] int64, random order).

    Skewed laws repeat popular coordinates, so coordinates are drawn in rounds
    until ``target`` distinct ones exist; each round's size follows the
    fraction of new coordinates the previous round produced.  Earlier draws
    keep their place, so a smaller target is a prefix-like sample of the same
    recipe."""
    idx = torch.empty((len(I), 0), dtype=torch.int64, device=device)
    want = target
    for _ in range(max_rounds):
        if want <= 0:
            break
        cols = torch.stack([draw_mode_indices(gen, In, want, dist, s, device) for In in I])
        before = idx.shape[1]
        idx = dedup_coords(torch.cat([idx, cols], dim=1))
        gained = idx.shape[1] - before
        if idx.shape[1] >= target:
            break
        frac = max(gained / max(want, 1), 0.02)
        want = int(min((target - idx.shape[1]) / frac * 1.15 + 1024, 3 * target + 1024))
    if idx.shape[1] < target:
        raise RuntimeError(f"could not draw {target} distinct coordinates")
    return idx[:, :target].contiguous()


def normal_matrices(gen: torch.Generator, shapes, std: float, device="cpu",
                    dtype=torch.float32):
    """One N(0, std^2) matrix per shape (std is the standard deviation)."""
    return [
        (torch.randn(tuple(sh), generator=gen, device=device, dtype=torch.float64) * std).to(dtype)
        for sh in shapes
    ]


def start_std(J: int, R: int, N: int, pred_std: float = 0.2) -> float:
    """Standard deviation s of an N(0, s^2) start for every entry of A^(n) and
    B^(n) whose predictions have standard deviation ``pred_std``: each
    a^(n) B^(n) entry has variance J s^4 and the prediction sums R products of
    N of them, so pred_std^2 = R (J s^4)^N.  A small random start: at much
    smaller ones plain SGD stalls near the saddle point at zero."""
    return (pred_std * pred_std / R) ** (1.0 / (4 * N)) / J ** 0.25


def centre(train_x: torch.Tensor, *others: torch.Tensor):
    """Values minus the training mean (computed in float64): the mean and the
    centred training values, then every other tensor centred by the same
    mean.  Ratings tensors are trained centred, since the model
    sum_r prod_n c^(n)_r has no offset term."""
    mu = float(train_x.double().mean()) if train_x.numel() else 0.0
    return (mu, (train_x.double() - mu).to(torch.float32),
            *[(t.double() - mu).to(torch.float32) for t in others])


def to_ratings(pred: torch.Tensor, centre: float = 3.0, spread: float = 1.1,
               lo: float = 1.0, hi: float = 5.0) -> torch.Tensor:
    """Map planted predictions to integer ratings lo..hi: standardise, scale,
    round, clip (float32 output)."""
    p = pred.to(torch.float64)
    z = (p - p.mean()) / p.std().clamp_min(1e-30)
    return torch.clamp(torch.round(centre + spread * z), lo, hi).to(torch.float32)


def split_train_test(gen: torch.Generator, nnz: int, test_frac: float, device="cpu"):
    """Random split of positions 0..nnz-1 (both parts keep a random order)."""
    perm = torch.randperm(nnz, generator=gen, device=device)
    n_test = int(round(nnz * test_frac))
    return perm[n_test:], perm[:n_test]


@dataclass
class Workload:
    """A named synthetic tensor recipe (sizes, index law, planted model)."""
    name: str
    I: tuple
    nnz: int
    J: tuple
    R: int
    dist: str = "uniform"
    zipf_s: float = 1.1
    planted_std: float | None = None    # None: 1/sqrt(J)
    noise_std: float = 0.0
    ratings: bool = False
    test_frac: float = 0.1
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return len(self.I)


# Named recipes.  Mode sizes of the Netflix-shaped tensor follow the paper's
# dataset table (Sec. 5.1); the Zipf skew stands in for the popularity
# structure of real ratings.
WORKLOADS = {
    "planted_uniform_1e5": Workload(
        name="planted_uniform_1e5", I=(1000, 1000, 1000), nnz=100_000, J=(4, 4, 4), R=4,
        dist="uniform", planted_std=0.5, noise_std=0.1),
    # the same planted model on Zipf-skewed coordinates (row counts spread
    # over orders of magnitude)
    "planted_zipf_1e5": Workload(
        name="planted_zipf_1e5", I=(1000, 1000, 1000), nnz=100_000, J=(4, 4, 4), R=4,
        dist="zipf", zipf_s=1.1, planted_std=0.5, noise_std=0.1),
    "netflix_shaped_zipf_1e8": Workload(
        name="netflix_shaped_zipf_1e8", I=(480_000, 18_000, 2_200), nnz=100_000_000,
        J=(16, 16, 16), R=16, dist="zipf", zipf_s=1.1, planted_std=0.25, ratings=True),
    # the same shape and size without popularity skew (no hot rows)
    "netflix_shaped_uniform_1e8": Workload(
        name="netflix_shaped_uniform_1e8", I=(480_000, 18_000, 2_200), nnz=100_000_000,
        J=(16, 16, 16), R=16, dist="uniform", planted_std=0.25, ratings=True),
    "order4_zipf_2e8": Workload(
        name="order4_zipf_2e8", I=(1_000_000, 1_000_000, 100_000, 1_000), nnz=200_000_000,
        J=(32, 32, 32, 32), R=32, dist="zipf", zipf_s=1.05, noise_std=0.05),
}



def synthetic_order(N: int, nnz: int = 100_000_000) -> Workload:
    """The paper's synthetic family (Sec. 5.1, synthetic dataset table):
    order N in 3..10, every mode of size 10,000, 1e8 uniform coordinates,
    integer values 1..5 (here: a planted J = R = 16 model mapped to ratings)."""
    return Workload(name=f"synthetic_order{N}_1e8", I=(10_000,) * N, nnz=nnz, J=(16,) * N, R=16,
                    dist="uniform", planted_std=0.25, ratings=True)

@dataclass
class Draw:
    """The random part of a workload: coordinates, planted model, noise, split."""
    idx: torch.Tensor            # [N, nnz] int32, deduplicated, random order
    planted_A: list
    planted_B: list
    noise: torch.Tensor          # [nnz] float32 (zeros when noise_std == 0)
    train: torch.Tensor          # positions of the training nonzeros
    test: torch.Tensor           # positions of the test nonzeros


def draw_workload(w: Workload, device="cpu", nnz: int | None = None) -> Draw:
    """Draw coordinates, the planted model, noise and the split of ``w``.

    ``nnz`` overrides the coordinate count (a prefix-sized sample of the
    same recipe)."""
    gen = generator(w.seed, device)
    target = int(w.nnz if nnz is None else nnz)
    idx = draw_unique_coords(gen, w.I, target, w.dist, w.zipf_s, device)
    nnz_u = idx.shape[1]
    std_of = (lambda J: w.planted_std) if w.planted_std is not None else (lambda J: 1.0 / math.sqrt(J))
    A = [normal_matrices(gen, [(I, J)], std_of(J), device)[0] for I, J in zip(w.I, w.J)]
    B = [normal_matrices(gen, [(J, w.R)], std_of(J), device)[0] for J in w.J]
    if w.noise_std > 0:
        noise = (torch.randn(nnz_u, generator=gen, device=device, dtype=torch.float64)
                 * w.noise_std).to(torch.float32)
    else:
        noise = torch.zeros(nnz_u, dtype=torch.float32, device=device)
    train, test = split_train_test(gen, nnz_u, w.test_frac, device)
    return Draw(idx=idx.to(torch.int32), planted_A=A, planted_B=B, noise=noise,
                train=train, test=test)


def initial_factors(w: Workload, device="cpu", seed_offset: int = 1):
    """Starting point of training, N(0, s^2) entries: s = 1/sqrt(J) for
    planted real-valued tensors; for ratings tensors (trained centred, unit
    scale) the s of ``start_std``, whose predictions have standard deviation
    0.2."""
    gen = generator(w.seed + seed_offset, device)
    if w.ratings:
        sd = [start_std(max(w.J), w.R, w.N)] * w.N
    else:
        sd = [1.0 / math.sqrt(J) for J in w.J]
    A = [normal_matrices(gen, [(I, J)], s, device)[0] for I, J, s in zip(w.I, w.J, sd)]
    B = [normal_matrices(gen, [(J, w.R)], s, device)[0] for J, s in zip(w.J, sd)]
    return A, B


def random_problem(seed: int, I, J, R, nnz, device="cpu", std=None, value_std=1.0, positive=False):
    """A small unstructured problem for parity tests: uniform coordinates
    (duplicates allowed), N(0, s_n^2) factors and cores, N(0, value_std^2)
    values.  By default s_n = (R^(-1/N) / J_n)^(1/4), which makes every
    a^(n) B^(n) entry of variance R^(-1/N) and the prediction of variance
    about 1, so SGD steps stay well scaled for any N, J, R.  positive=True
    takes the absolute values of the factor and core draws (no cancellation
    in the products a.B)."""
    gen = generator(seed, device)
    N = len(I)
    idx = torch.stack([torch.randint(0, int(In), (nnz,), generator=gen, device=device)
                       for In in I]).to(torch.int32)
    if positive:   # |N(0, s^2)| has mean s sqrt(2/pi): mean of every a.B entry R^(-1/N)
        sd = [std if std is not None else math.sqrt(math.pi / 2 * R ** (-1.0 / N) / Jn) for Jn in J]
    else:
        sd = [std if std is not None else (R ** (-1.0 / N) / Jn) ** 0.25 for Jn in J]
    A = [normal_matrices(gen, [(In, Jn)], s, device)[0] for In, Jn, s in zip(I, J, sd)]
    B = [normal_matrices(gen, [(Jn, R)], s, device)[0] for Jn, s in zip(J, sd)]
    if positive:
        A = [a.abs() for a in A]
        B = [b.abs() for b in B]
    x = (torch.randn(nnz, generator=gen, device=device, dtype=torch.float64) * value_std).to(torch.float32)
    return idx, x, A, B


# ------------------------------------------------------------ batches
def batched_recipe(count: int = 64, seed: int = 0):
    """Shapes of a batch of independent tensors of uneven order and size:
    N uniform in {3, 4, 5}, nnz log-uniform in [1e4, 1e6], every I_n
    log-uniform in [1e3, 1e5], J_n uniform in {4, 8, 16} (one J per tensor),
    R uniform in {8, 16, 32}."""
    gen = generator(seed)
    out = []
    for k in range(count):
        u = torch.rand(4 + 5, generator=gen, dtype=torch.float64)
        N = 3 + int(u[0] * 3)
        nnz = int(round(10 ** (4 + 2 * float(u[1]))))
        J = (4, 8, 16)[int(u[2] * 3)]
        R = (8, 16, 32)[int(u[3] * 3)]
        I = tuple(int(round(10 ** (3 + 2 * float(u[4 + n])))) for n in range(N))
        out.append(Workload(name=f"batch{count}_{k}", I=I, nnz=nnz, J=(J,) * N, R=R, dist="uniform",
                            noise_std=0.1, seed=seed * 1000 + k + 1))
    return out
