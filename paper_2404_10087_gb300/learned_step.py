"""Learned per-row step sizes on top of the FastTuckerPlus factor update.

The paper uses one step size gamma_A for every row (Eq.
"Update_FastTuckerPlus_factor"); this module scales it per row by a small
network (3 -> 64 -> 64 -> 1, BF16 weights, FP32 accumulation) that maps row
statistics - nonzeros in the row, a running average of the row-gradient
norm, the mean residual - to a multiplier in [1/16, 16] (it predicts the
log-multiplier).  The network is trained on traces of plain runs, with the
log of the exact line-search step of every row's subproblem, shared among
the N rows that each nonzero moves at once and relative to the step size, as
the label (see ft_row_stats in include/ft.h).

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
                   lam_b: float, beta: float = 0.9, label_step: float | None = None):
    """Run `epochs` plain epochs at factor step lr_a and record, before each,
    every row's features and line-search label (relative to label_step,
    default lr_a).  Returns (features [epochs * rows, 3], labels)."""
    label_step = lr_a if label_step is None else label_step
    dev = model.vals.device
    rows = _rows(model)
    ema = torch.zeros(rows, dtype=torch.float32, device=dev)
    feats, labs = [], []
    for _ in range(epochs):
        f = torch.empty(rows, 3, dtype=torch.float32, device=dev)
        y = torch.empty(rows, dtype=torch.float32, device=dev)
        ft.ft_row_stats(model.ctx, lam_a, label_step, beta, ema, f, y)
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
                 beta: float = 0.9, record: bool = False):
        dev = model.vals.device
        self.model, self.net = model, net
        self.lr_a, self.lam_a, self.beta = lr_a, lam_a, beta
        rows = _rows(model)
        self.ema = torch.zeros(rows, dtype=torch.float32, device=dev)
        self.feat = torch.empty(rows, 3, dtype=torch.float32, device=dev)
        self.scale = torch.ones(rows, dtype=torch.float32, device=dev)
        self.per_mode = split_rows(model, self.scale)
        self.used = [] if record else None   # the multipliers of every epoch, when recorded

    def refresh(self):
        ft.ft_row_stats(self.model.ctx, self.lam_a, self.lr_a, self.beta, self.ema, self.feat, None)
        ft.ft_stepnet_forward(self.net, self.feat, self.scale)
        if self.used is not None:
            self.used.append(self.scale.clone())

    def epoch(self, lr_b: float, lam_b: float):
        """Refresh the multipliers, then one factor epoch with them and one core epoch."""
        self.refresh()
        self.model.epoch_factors(self.lr_a, self.lam_a, self.per_mode)
        self.model.epoch_core(lr_b, lam_b)


def _timed_run(epoch, model, tei, xte, epochs, target=None):
    """Run up to `epochs` epochs (stopping once the test RMSE is at or below
    `target`, or once the run diverges: a non-finite residual ends it with
    RMSE inf); returns (epochs run, seconds by CUDA events, last test RMSE,
    the test-RMSE curve including the start)."""
    curve = [model.rmse(tei, xte)[0]]
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    ep, r = 0, curve[0]
    for ep in range(1, epochs + 1):
        epoch()
        try:
            r = model.rmse(tei, xte)[0]
        except ft.FtError as err:
            if err.status != ft.FT_ERR_NONFINITE:
                raise
            r = float("inf")
        curve.append(r)
        if (target is not None and r <= target) or r == float("inf"):
            break
    t1.record()
    t1.synchronize()
    return ep, t0.elapsed_time(t1) / 1e3, r, curve


def _epochs_to(curve, target):
    """Epochs until the curve (start included) first reaches target, or None."""
    for k, v in enumerate(curve):
        if v <= target:
            return k
    return None


def ab_study(make_model, tei, xte, lrs, lam, lr_b, lam_b, epochs=20, trace_epochs=10, train_steps=400,
             seed=0):
    """The learned step against fixed global steps.

    make_model(start) -> a fresh FastTuckerPlus context from start 1 (the
    evaluation start) or 7 (the start of the trace run).  For every step
    size in `lrs` plain SGD runs `epochs` epochs from start 1; eta* is the one
    with the lowest final test RMSE, which is the target.  A plain run at
    eta* from start 7 gives the traces (features, and labels relative to
    eta*; if that run diverges, the next smaller step of the grid runs the
    traces, labels still relative to eta*); the network trains on them.
    Then, from start 1, each run stops at the target:
      * learned: eta* times the per-row multipliers (refreshed every epoch;
        the statistics and network passes are timed with it);
      * constant: plain SGD at eta* times the learned run's mean multiplier
        over its rows and epochs (the same global scale without the per-row
        part).
    Reported with the plain sweep's own time to the target at every step
    size (the best fixed step is the fastest of the runs that did not
    diverge), the label distribution (share at the clip), the spread of the
    multipliers the learned run used (all its rows and epochs), and the
    trained network's loss against the best constant predictor's (the
    labels' variance)."""
    sweep = {}
    for lr in lrs:
        m = make_model(1)
        ep, t, r, curve = _timed_run(lambda: (m.epoch_factors(lr, lam), m.epoch_core(lr_b, lam_b)), m, tei, xte,
                                     epochs)
        sweep[lr] = {"final_test_rmse": r, "seconds": t, "epochs_run": ep, "curve": curve}
        m.close()
    finite = {lr: v for lr, v in sweep.items() if v["final_test_rmse"] < float("inf")}
    eta = min(finite, key=lambda lr: finite[lr]["final_test_rmse"])
    target = sweep[eta]["final_test_rmse"]
    for lr, v in sweep.items():
        k = _epochs_to(v["curve"], target)
        # seconds cover the epochs the run made (a diverged run stops early)
        v["seconds_to_target"] = (v["seconds"] * k / max(v["epochs_run"], 1)) if k is not None else None
        v["curve"] = [round(c, 5) if c < float("inf") else "diverged" for c in v["curve"]]
    # the best fixed step: the fastest to the target among the steps whose
    # run did not diverge
    best_fixed = min(v["seconds_to_target"] for lr, v in sweep.items()
                     if lr in finite and v["seconds_to_target"] is not None)
    # the trace run from another start; at a step on the edge of stability it
    # may diverge from there, and then the next smaller step of the grid
    # gives the traces (the labels stay relative to eta*, the learned run's
    # base step)
    base = eta
    for base in sorted([lr for lr in finite if lr <= eta], reverse=True):
        tracer = make_model(7)
        feats, labels = collect_traces(tracer, trace_epochs, base, lam, lr_b, lam_b, label_step=eta)
        ok = bool(torch.isfinite(feats).all()) and bool(torch.isfinite(labels).all())
        try:
            tracer.check()
        except ft.FtError:
            ok = False
        tracer.close()
        if ok:
            break
    lab = labels.double()
    const_loss = float(0.5 * ((lab - lab.mean()) ** 2).mean())
    net = ft.new_stepnet(feats.device, seed=seed)
    loss_curve = train(net, feats, labels, steps=train_steps)
    model = make_model(1)
    learned = LearnedStep(model, net, eta, lam, record=True)
    ep_l, t_l, r_l, curve_l = _timed_run(lambda: learned.epoch(lr_b, lam_b), model, tei, xte, epochs, target)
    # the multipliers the run used, over all its epochs and rows
    logs = torch.cat(learned.used).double().log()
    logs = logs[torch.isfinite(logs)]
    model.close()
    mean_mult = float(logs.exp().mean())
    cm = make_model(1)
    lr_c = eta * mean_mult
    ep_c, t_c, r_c, curve_c = _timed_run(lambda: (cm.epoch_factors(lr_c, lam), cm.epoch_core(lr_b, lam_b)), cm, tei,
                                         xte, epochs, target)
    cm.close()
    clip = float(torch.log(torch.tensor(16.0)))
    q = torch.tensor([0.05, 0.25, 0.5, 0.75, 0.95], dtype=torch.float64, device=lab.device)
    reached, reached_c = r_l <= target, r_c <= target
    return {
        "eta_grid": list(lrs), "eta_star": eta, "trace_step": base, "target_test_rmse": target,
        "plain_sweep": {str(k): v for k, v in sweep.items()},
        "plain_epochs": epochs, "plain_seconds": sweep[eta]["seconds"],
        "best_fixed_step_seconds_to_target": best_fixed,
        "learned_epochs": ep_l if reached else None, "learned_seconds": t_l if reached else None,
        "reached": reached, "learned_final_test_rmse": r_l,
        "learned_curve": [round(v, 5) for v in curve_l],
        "constant_step": lr_c, "constant_epochs": ep_c if reached_c else None,
        "constant_seconds": t_c if reached_c else None, "constant_reached": reached_c,
        "constant_curve": [round(v, 5) for v in curve_c],
        "speedup_vs_eta_star": (sweep[eta]["seconds"] / t_l) if reached else None,
        "speedup_vs_best_fixed_step": (best_fixed / t_l) if reached else None,
        "speedup_vs_constant_multiplier": (t_c / t_l) if (reached and reached_c) else None,
        "labels": {"rows": int(lab.numel()), "share_at_clip": float((lab.abs() >= clip - 1e-6).double().mean()),
                   "log_quantiles_5_25_50_75_95": [round(float(v), 4) for v in torch.quantile(lab, q)]},
        "net_loss": [round(v, 5) for v in loss_curve], "constant_predictor_loss": round(const_loss, 5),
        "multiplier": {"mean": mean_mult, "log_std": float(logs.std()),
                       "quantiles_5_25_50_75_95": [round(float(v), 4) for v in torch.quantile(logs.exp(), q)]},
    }
