"""Learned per-row step sizes on top of the FastTuckerPlus factor update.

The paper uses one step size gamma_A for every row (Eq.
"Update_FastTuckerPlus_factor"); this module scales it per row by a small
network (3 -> 64 -> 64 -> 1, BF16 weights, FP32 accumulation) that maps row
statistics - nonzeros in the row, a running average of the row-gradient
norm, the mean residual - to a multiplier in (1/4, 4).  The network is
trained on traces of plain runs, with the exact line-search step of every
row's subproblem as the label (see ft_row_stats in include/ft.h).

Every step runs in the CUDA library (ft_row_stats, ft_stepnet_*,
ft_epoch_factors with row_step_scale); this module only sequences calls.
"""
from __future__ import annotations

import torch

from . import ft


def _rows(model: ft.FastTuckerPlus) -> int:
    return sum(model.I)


def split_rows(model: ft.FastTuckerPlus, t: torch.Tensor):
    """Per-mode views of a tensor over the concatenated rows."""
    out, off = [], 0
    for I in model.I:
        out.append(t[off:off + I])
        off += I
    return out


def collect_traces(model: ft.FastTuckerPlus, epochs: int, lr_a: float, lam_a: float, lr_b: float,
                   lam_b: float, beta: float = 0.9):
    """Run `epochs` plain epochs and record, before each, every row's features
    and line-search label.  Returns (features [epochs * rows, 3], labels)."""
    dev = model.vals.device
    rows = _rows(model)
    ema = torch.zeros(rows, dtype=torch.float32, device=dev)
    feats, labs = [], []
    for _ in range(epochs):
        f = torch.empty(rows, 3, dtype=torch.float32, device=dev)
        y = torch.empty(rows, dtype=torch.float32, device=dev)
        ft.ft_row_stats(model.ctx, lam_a, lr_a, beta, ema, f, y)
        feats.append(f)
        labs.append(y)
        model.epoch_factors(lr_a, lam_a)
        model.epoch_core(lr_b, lam_b)
    return torch.cat(feats), torch.cat(labs)


def train(net: torch.Tensor, features: torch.Tensor, labels: torch.Tensor, steps: int = 300,
          lr: float = 3e-3, chunk: int = 50):
    """Full-batch Adam on mean 1/2 (s - label)^2; returns the loss curve."""
    curve = []
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        curve.append(ft.ft_stepnet_train(net, features.contiguous(), labels.contiguous(), lr, k))
        done += k
    return curve


class LearnedStep:
    """Per-row multipliers for one model, refreshed from its statistics."""

    def __init__(self, model: ft.FastTuckerPlus, net: torch.Tensor, lr_a: float, lam_a: float,
                 beta: float = 0.9):
        dev = model.vals.device
        self.model, self.net = model, net
        self.lr_a, self.lam_a, self.beta = lr_a, lam_a, beta
        rows = _rows(model)
        self.ema = torch.zeros(rows, dtype=torch.float32, device=dev)
        self.feat = torch.empty(rows, 3, dtype=torch.float32, device=dev)
        self.scale = torch.ones(rows, dtype=torch.float32, device=dev)
        self.per_mode = split_rows(model, self.scale)

    def refresh(self):
        ft.ft_row_stats(self.model.ctx, self.lam_a, self.lr_a, self.beta, self.ema, self.feat, None)
        ft.ft_stepnet_forward(self.net, self.feat, self.scale)

    def epoch(self, lr_b: float, lam_b: float):
        """Refresh the multipliers, then one factor epoch with them and one core epoch."""
        self.refresh()
        self.model.epoch_factors(self.lr_a, self.lam_a, self.per_mode)
        self.model.epoch_core(lr_b, lam_b)
