#!/usr/bin/env python3
"""Throughput of the FastTuckerPlus SGD epoch on one GB300 (or N replicas).

A step is one pass of the whole hot path over the training nonzeros of the
Netflix-shaped synthetic tensor (N = 3, I = 480000 x 18000 x 2200, 1e8 Zipf
coordinates, J = R = 16, 90/10 split): the factor phase, the core phase
(gradient + finalize) and the test-set RMSE/MAE.  The metric is
nonzero-updates per second = |Omega_train| / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|tf32|bf16]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host

Prints one JSON line (rank 0).  Under torchrun every rank trains its own
replica (no data-path collective) and the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2404_10087_gb300 import ft, synth  # noqa: E402

METRIC = "SGD nonzero-updates/sec (factor+core) at J=R=16; time-to-RMSE vs plain FP32"
UNIT = "nnz-updates/s"
WORKLOAD = "netflix_shaped_zipf_1e8"
# Step sizes of the Netflix-shaped workload (the paper's are unstated): a
# sweep of the factor step on the full tensor (FP32, 20 epochs; test RMSE
# 0.005: 0.94, 0.01: 0.80, 0.02: 0.61, 0.03: 0.58, 0.04: 0.577, 0.06: 0.562,
# 0.08 and 0.12 diverged) - 0.04 keeps a factor of two to the first step that
# diverged; the core step is on the scale of a full-gradient step because
# Algorithm 5 divides the summed gradient by |Omega|.
LR = 0.04          # factor step gamma_A
LR_B = 0.3         # core step gamma_B
LR_ORDERS = 0.01   # factor step of the synthetic order sweep
LAM = 0.01
FALLBACK_HBM_GBS = 6800.0


def algorithmic_bytes_factor(N, J):
    """Per nonzero: N int32 coordinates + one float32 value read, N factor rows
    read and written (float32)."""
    return 4 * N + 4 + 2 * 4 * sum(J)


def peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def describe_data(w) -> str:
    """The "data" field of the JSON line: how the workload's inputs were drawn."""
    coords = f"Zipf({w.zipf_s}) coordinates" if w.dist == "zipf" else "uniform coordinates"
    values = ("planted-model ratings 1..5" if w.ratings
              else f"planted-model values + N(0, {w.noise_std}) noise")
    return f"synthetic (seeded {coords}, {values}; {w.name})"


def kernel_digest():
    h = hashlib.sha256()
    for name in ("ft_device.cuh",):
        with open(os.path.join(ROOT, "paper_2404_10087_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(precision, workload=WORKLOAD, nnz=None, engine="warp", hot_window=None):
    """DRAM bytes per factor launch from the committed ncu summary, if it was
    taken on the current kernel source and on this launch (the default
    workload at full size, warp-tile engine, the same hot-row write-back
    window); else None."""
    if workload != WORKLOAD or nnz is not None or engine != "warp":
        return None
    p = os.path.join(ROOT, "profiles", "ncu_factor_netflix_zipf.md")
    if not os.path.exists(p):
        return None
    text = open(p).read()
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    if not m or m.group(1) != kernel_digest():
        return None
    w = re.search(r"hot_window:\s*([0-9]+)", text)
    if hot_window is not None and (not w or int(w.group(1)) != int(hot_window)):
        return None
    m = re.search(rf"traffic_bytes_per_launch_{precision}:\s*([0-9.eE+]+)", text)
    return float(m.group(1)) if m else None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_replicas(times_ms, units_per_rank, steps, world, device="cpu"):
    """Replicas only: every rank trains its own tensor.  The job time is the
    slowest rank's (max over ranks of each timing) and the value is the units
    of all ranks over that time: world * units / (times_ms[0] / steps)."""
    t = torch.tensor([float(v) for v in times_ms], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    out = [float(v) for v in t.cpu()]
    value = world * units_per_rank / (out[0] / steps / 1e3)
    return out, value


def make_workload(device, nnz=None, name=WORKLOAD):
    """Draw the synthetic tensor on `device`; planted values are computed by the
    library's own predict call, then mapped to integer ratings 1..5 (ratings
    workloads) or given the workload's noise.  `name` is a recipe name or a
    synth.Workload."""
    w = synth.WORKLOADS[name] if isinstance(name, str) else name
    d = synth.draw_workload(w, device=device, nnz=nnz)
    N = w.N
    allidx = [d.idx[n].contiguous() for n in range(N)]
    zeros = torch.zeros(d.idx.shape[1], dtype=torch.float32, device=device)
    pm = ft.FastTuckerPlus(allidx, zeros, [a.contiguous() for a in d.planted_A],
                           [b.contiguous() for b in d.planted_B], hot_rows=0)
    pred = pm.predict(allidx)
    pm.close()
    del zeros
    vals = synth.to_ratings(pred) if w.ratings else pred + d.noise
    del pred
    tr, te = d.train, d.test
    train_idx = [d.idx[n, tr].contiguous() for n in range(N)]
    test_idx = [d.idx[n, te].contiguous() for n in range(N)]
    train_x = vals[tr].contiguous()
    test_x = vals[te].contiguous()
    if w.ratings:   # trained centred: the model has no offset term
        _, train_x, test_x = synth.centre(train_x, test_x)
    A, B = synth.initial_factors(w, device=device)
    return w, train_idx, train_x, test_idx, test_x, A, B


def one_allocation(mats):
    """The matrices copied into views of one device allocation (each view
    starting on a 256-byte boundary), so that one L2 access-policy window
    can cover all of them."""
    sizes = [(m.numel() + 63) // 64 * 64 for m in mats]
    flat = torch.empty(sum(sizes), dtype=mats[0].dtype, device=mats[0].device)
    out, off = [], 0
    for m, sz in zip(mats, sizes):
        v = flat[off:off + m.numel()].view(m.shape)
        v.copy_(m)
        out.append(v)
        off += sz
    return out


BATCHED = "batched_64"
# Step sizes of the batched workload (planted real-valued tensors; none are
# given for it): factor step 0.005 (at 0.01 one Hogwild epoch raised the
# training error of one of the 64 tensors), the Netflix-shaped workload's
# core step
LR_BATCH, LR_B_BATCH = 0.005, 0.3


def run_batched(args, rank, world, local_rank):
    """64 independent tensors (N in {3,4,5}, nnz log-uniform in [1e4, 1e6],
    I_n log-uniform in [1e3, 1e5], J in {4,8,16}, R in {8,16,32}, planted
    model + N(0, 0.1) noise) trained by the batched persistent epoch: one
    captured graph per epoch, launch shapes from the autotuner."""
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    ft.load()
    recipes = synth.batched_recipe(64, seed=0)
    train, test = [], []
    for w in recipes:
        d = synth.draw_workload(w, device=dev)
        allidx = [d.idx[n].contiguous() for n in range(w.N)]
        zeros = torch.zeros(d.idx.shape[1], dtype=torch.float32, device=dev)
        pm = ft.FastTuckerPlus(allidx, zeros, [a.contiguous() for a in d.planted_A],
                               [b.contiguous() for b in d.planted_B], hot_rows=0)
        vals = pm.predict(allidx) + d.noise
        pm.close()
        A, B = synth.initial_factors(w, device=dev)
        train.append(([d.idx[n, d.train].contiguous() for n in range(w.N)], vals[d.train].contiguous(), A, B))
        test.append(([d.idx[n, d.test].contiguous() for n in range(w.N)], vals[d.test].contiguous()))
    nnz_train = sum(int(t[1].numel()) for t in train)
    stream = torch.cuda.current_stream(dev)
    b = ft.FastTuckerBatch(train, precision=args.precision, tune=True)
    for _ in range(args.warmup):
        b.epoch(LR_BATCH, LAM, LR_B_BATCH, LAM)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    l0 = b.launches
    with ClockSampler(local_rank) as clk:
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            b.epoch(LR_BATCH, LAM, LR_B_BATCH, LAM)
        t1.record(stream)
        torch.cuda.synchronize()
    total_ms = t0.elapsed_time(t1)
    launches = b.launches - l0
    rm = [b.rmse(k, i, v)[0] for k, (i, v) in enumerate(test)]
    (total_ms,), value = aggregate_replicas([total_ms], nnz_train, args.steps, world, dev)
    if rank != 0:
        return None
    # algorithmic bytes of one epoch, summed over the tensors: the factor
    # phase (coordinates, value, N rows read and written) and the core phase
    # (coordinates, value, N rows read) of every training nonzero
    epoch_bytes = sum(int(t[1].numel()) * (algorithmic_bytes_factor(len(t[0]), [a.shape[1] for a in t[2]])
                                           + 4 * len(t[0]) + 4 + 4 * sum(a.shape[1] for a in t[2]))
                      for t in train)
    peak, peak_kind = peak_hbm()
    ms_per_step = total_ms / args.steps
    achieved = epoch_bytes / (ms_per_step / 1e3) / 1e9
    out = {
        "metric": METRIC + " (batched: 64 tensors, one graph per epoch)", "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "tf32", "bf16": "bf16"}[args.precision],
        "data": "synthetic (64 planted tensors of uneven order, size and rank, uniform coordinates)",
        "config": {"workload": BATCHED, "tensors": 64, "nnz_train": nnz_train, "precision": args.precision,
                   "classes": b.classes(), "lr_a": LR_BATCH, "lr_b": LR_B_BATCH, "lambda": LAM,
                   "l2": "inputs larger than L2 (training COO 216 MB per epoch)"},
        "mean_test_rmse": sum(rm) / len(rm),
        "roofline": {"bound": "hbm", "kernel": "the epoch graph (factor + core kernels of every class, "
                                                "finalize)", "scope": "epoch",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "bytes_per_epoch": epoch_bytes,
                     "launch_ms": ms_per_step},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_batched(train)
    return out


def cpu_baseline_batched(train, budget_s=10.0):
    """The FP64 oracle on every host core over the batch's tensors, one after
    another (Hogwild factor epoch + core epoch each), until about `budget_s`
    seconds of work; the rate over the tensors timed is taken as the batch's."""
    import oracle
    threads = oracle.default_threads()
    done, secs, ntens = 0, 0.0, 0
    for idx, x, A, B in train:
        i64 = np.ascontiguousarray(torch.stack([t.cpu() for t in idx]).numpy())
        x64 = x.double().cpu().numpy()
        A64 = [a.double().cpu().numpy() for a in A]
        B64 = [b.double().cpu().numpy() for b in B]
        t = time.perf_counter()
        A64 = oracle.factor_epoch_hogwild(A64, B64, i64, x64, LR_BATCH, LAM, nthreads=threads)
        oracle.core_epoch(A64, B64, i64, x64, LR_B_BATCH, LAM, nthreads=threads)
        secs += time.perf_counter() - t
        done += int(x.numel())
        ntens += 1
        if secs >= budget_s:
            break
    return {"value": done / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"the first {ntens} of {len(train)} tensors ({done} training nonzeros), one FP64 "
                      f"Hogwild factor epoch + core epoch each on {threads} host threads, {secs:.1f} s; "
                      f"rate taken as the batch's"}


def run_ours(args, rank, world, local_rank):
    if args.workload == BATCHED:
        return run_batched(args, rank, world, local_rank)
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    ft.load()
    w, tri, trx, tei, tex, A, B = make_workload(dev, args.nnz, args.workload)
    A = one_allocation(A)
    N, J, R = w.N, list(w.J), w.R
    nnz_train, nnz_test = int(trx.numel()), int(tex.numel())
    stream = torch.cuda.current_stream(dev)
    m = ft.FastTuckerPlus(tri, trx, A, B, precision=args.precision, scatter="hogwild",
                          hot_rows=args.hot_rows, hot_window=args.hot_window, engine=args.engine,
                          core_scheme=args.core_scheme, l2_persist=bool(args.l2_persist))

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(record=None, test=(tei, tex), after_core=None):
        e0, e1, e2, e3 = (ev(), ev(), ev(), ev()) if record is not None else (None,) * 4
        if record is not None:
            e0.record(stream)
        m.epoch_factors(LR, LAM)
        if record is not None:
            e1.record(stream)
        m.epoch_core(LR_B, LAM)
        if record is not None:
            e2.record(stream)
        if after_core is not None:
            after_core()
        r = m.rmse(*test)  # synchronises: the step's result reaches the host
        if record is not None:
            e3.record(stream)
            record.append((e0, e1, e2, e3))
        return r

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = m.launches
    rec = []
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        t0 = ev()
        t1 = ev()
        t0.record(stream)
        for _ in range(args.steps):
            last = step(rec)
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = t0.elapsed_time(t1)
    launches = m.launches - launches0
    f_ms = [a.elapsed_time(b) for a, b, _, _ in rec]
    c_ms = [b.elapsed_time(c) for _, b, c, _ in rec]
    r_ms = [c.elapsed_time(d) for _, _, c, d in rec]

    # end to end through the C ABI with host buffers: every step copies its
    # inputs (the training and the test COO) from pinned host memory and
    # reads the RMSE back.  Two device copies of the inputs alternate: while
    # step k trains on one, a second stream copies step k+1's inputs into the
    # other and, once step k's passes are enqueued, points the context at it
    # (ft_rebind rebuilds the hot-row coordinates on that stream).
    host_in = [t.cpu().pin_memory() for t in list(tri) + [trx] + list(tei) + [tex]]
    h2d = sum(t.numel() * t.element_size() for t in host_in)
    e2e_steps = max(1, args.steps)           # the same K steps as the device-resident leg
    dev_in = [list(tri) + [trx] + list(tei) + [tex], [torch.empty_like(t, device=dev) for t in host_in]]
    bufs = [(d[:N], d[N], d[N + 1:2 * N + 1], d[2 * N + 1]) for d in dev_in]
    copy_stream = torch.cuda.Stream(dev)
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    free = [torch.cuda.Event(), torch.cuda.Event()]

    def copy_in(k):
        b = k % 2
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(free[b])        # the step that last read buffer b is done
            for dst, src in zip(dev_in[b], host_in):
                dst.copy_(src, non_blocking=True)

    def rebind_in(k):
        b = k % 2
        m.rebind(bufs[b][0], bufs[b][1], stream=copy_stream)   # after the copy, same stream
        ready[b].record(copy_stream)

    def e2e_run(steps):
        copy_stream.wait_stream(stream)
        copy_in(0)
        rebind_in(0)
        for k in range(steps):
            b = k % 2
            stream.wait_event(ready[b])
            nxt = None
            if k + 1 < steps:
                copy_in(k + 1)
                nxt = (lambda kk=k + 1: rebind_in(kk))
            step(test=(bufs[b][2], bufs[b][3]), after_core=nxt)
            free[b].record(stream)

    e2e_run(args.warmup)          # untimed: first use of the pinned buffers and the second copy
    torch.cuda.synchronize()
    te0, te1 = ev(), ev()
    te0.record(stream)
    e2e_run(e2e_steps)
    te1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = te0.elapsed_time(te1) / e2e_steps
    m.rebind(tri, trx)

    (total_ms, e2e_ms), value = aggregate_replicas([total_ms, e2e_ms], nnz_train, args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    if rank != 0:
        return None

    per_nnz = algorithmic_bytes_factor(N, J)
    coo_bytes = (4 * N + 4) * nnz_train
    fac_ms = statistics.mean(f_ms)
    achieved = per_nnz * nnz_train / (fac_ms / 1e3) / 1e9
    peak, peak_kind = peak_hbm()
    traffic = recorded_traffic(args.precision, args.workload, args.nnz, args.engine, m.cfg.hot_window)
    clocks = clk.summary()
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "tf32", "bf16": "bf16"}[args.precision],
        "data": describe_data(w),
        "config": {
            "workload": args.workload if args.nnz is None else f"{args.workload} at {args.nnz} coordinates", "N": N, "I": list(w.I), "J": J, "R": R,
            "nnz_train": nnz_train, "nnz_test": nnz_test, "precision": args.precision,
            "scatter": "hogwild", "engine": args.engine, "core_scheme": args.core_scheme,
            "l2_persist": bool(args.l2_persist),
            "hot_rows": m.cfg.hot_rows,
            "hot_window": m.cfg.hot_window,
            "lr_a": LR, "lr_b": LR_B, "lambda": LAM,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": f"inputs larger than L2 (training COO stream {coo_bytes / 1e9:.2f} GB per epoch)",
        },
        "phases_ms": {"factor": statistics.median(f_ms), "core": statistics.median(c_ms),
                      "rmse": statistics.median(r_ms)},
        "test_rmse": last[0],
        "roofline": {
            "bound": "hbm", "kernel": "k_factor_tc" if args.engine == "tcgen05" else "k_factor",
            "achieved": achieved, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "bytes_per_nnz": per_nnz, "nnz_per_launch": nnz_train,
            "launch_ms": fac_ms,
        },
        "e2e": {"value": world * nnz_train / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 24},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if not args.no_time_to_rmse:
        out["time_to_rmse"] = time_to_rmse(w, tri, trx, tei, tex, dev, args.ttr_epochs, args.precision)
        out["learned_step"] = learned_step_ab(dev)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_sample)
    return out


def time_phases(m, steps, warmup, stream, lr=LR):
    """Median factor-pass and core-pass times (CUDA events) over `steps`
    factor + core epochs after `warmup` untimed ones."""
    for _ in range(warmup):
        m.epoch_factors(lr, LAM)
        m.epoch_core(LR_B, LAM)
    torch.cuda.synchronize()
    rec = []
    for _ in range(steps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        m.epoch_factors(lr, LAM)
        e[1].record(stream)
        m.epoch_core(LR_B, LAM)
        e[2].record(stream)
        rec.append(e)
    torch.cuda.synchronize()
    f = statistics.median(a.elapsed_time(b) for a, b, _ in rec)
    c = statistics.median(b.elapsed_time(c) for _, b, c in rec)
    return f, c


def engine_for(args, N, J, R):
    """The requested factor-pass engine where it applies (tcgen05: BF16,
    N <= 4, J, R <= 16), else the warp-tile kernels."""
    ok = args.precision == "bf16" and N <= 4 and J <= 16 and R <= 16
    return args.engine if ok else "warp"


def run_sweep(args, local_rank):
    """The paper's studies on this GPU (Sec. 5): per-iteration factor and core
    times (a) over the synthetic orders N = 3..10 (I = 10,000 per mode, 1e8
    uniform coordinates, J = R = 16), (b) over (R, J) in {16, 32}^2 on the
    Netflix-shaped Zipf tensor, (c) for the two core-phase schemes of
    Sec. 5.6 (calculation vs storage) per precision on that tensor, (d) for
    the Algorithm 3 readings on that tensor: per-set core SGD and a reshuffle
    of the nonzeros before every epoch, against Algorithm 5 in stored order
    (core time, permutation time and the test-RMSE curve over 10 epochs)."""
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    ft.load()
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = peak_hbm()
    rows = []
    if args.sweep in ("orders", "all"):
        # the synthetic orders take the largest of five factor steps whose run
        # stays finite (the Netflix-shaped step 0.04 diverged at high order,
        # 0.01 from N = 7 and 0.001 from N = 8, with or without the hot-row
        # cache and at FP32 alike: every row there meets 9e3 nonzeros per
        # epoch, and the step's effect grows with the N - 1 factors of d)
        for N in range(3, 11):
            w = synth.synthetic_order(N, nnz=args.nnz or 100_000_000)
            w_, tri, trx, tei, tex, A0, B0 = make_workload(dev, None, w)
            eng = engine_for(args, N, 16, 16)
            # the largest of LR_ORDERS / 1, 3, 10, 30, 100 whose run stays finite
            for lr in (LR_ORDERS, LR_ORDERS / 3, LR_ORDERS / 10, LR_ORDERS / 30, LR_ORDERS / 100):
                A = [a.clone() for a in A0]
                B = [b.clone() for b in B0]
                m = ft.FastTuckerPlus(tri, trx, A, B, precision=args.precision, hot_rows=args.hot_rows,
                                      hot_window=args.hot_window, engine=eng)
                f, c = time_phases(m, args.steps, args.warmup, stream, lr=lr)
                try:
                    rmse = m.rmse(tei, tex)[0]
                except ft.FtError:
                    rmse = "diverged"
                m.close()
                if rmse != "diverged":
                    break
            nnz = int(trx.numel())
            per = algorithmic_bytes_factor(N, w.J)
            rows.append({"study": "order", "N": N, "I": w.I[0], "J": 16, "R": 16, "engine": eng, "nnz_train": nnz,
                         "lr_a": lr,
                         "factor_ms": f, "core_ms": c, "value": nnz / ((f + c) / 1e3),
                         "factor_frac_hbm": per * nnz / (f / 1e3) / 1e9 / peak, "test_rmse": rmse})
            del tri, trx, tei, tex, A, B, A0, B0
            torch.cuda.empty_cache()
    if args.sweep in ("ranks", "all"):
        w0, tri, trx, tei, tex, _, _ = make_workload(dev, args.nnz, args.workload)
        base = None
        for R, J in ((16, 16), (16, 32), (32, 16), (32, 32)):
            w = synth.Workload(**{**w0.__dict__, "J": (J,) * w0.N, "R": R})
            A, B = synth.initial_factors(w, device=dev)
            eng = engine_for(args, w0.N, J, R)
            m = ft.FastTuckerPlus(tri, trx, A, B, precision=args.precision, hot_rows=args.hot_rows,
                                  hot_window=args.hot_window, engine=eng)
            f, c = time_phases(m, args.steps, args.warmup, stream)
            nnz = int(trx.numel())
            base = base or (f, c)
            rows.append({"study": "rank", "workload": w0.name, "R": R, "J": J, "engine": eng, "nnz_train": nnz,
                         "factor_ms": f, "core_ms": c, "factor_x": f / base[0], "core_x": c / base[1],
                         "value": nnz / ((f + c) / 1e3)})
            m.close()
    if args.sweep in ("schemes", "all"):
        # Sec. 5.6: the core phase forming the rows of C per nonzero
        # (calculation) or gathering them from C = A B precomputed once per
        # core phase (storage), per precision
        w0, tri, trx, tei, tex, A0, B0 = make_workload(dev, args.nnz, args.workload)
        for prec in ("fp32", "tf32", "bf16"):
            for scheme in ("calc", "store"):
                A = [a.clone() for a in A0]
                B = [b.clone() for b in B0]
                m = ft.FastTuckerPlus(tri, trx, A, B, precision=prec, hot_rows=args.hot_rows,
                                      hot_window=args.hot_window, core_scheme=scheme)
                f, c = time_phases(m, args.steps, args.warmup, stream)
                rows.append({"study": "core_scheme", "workload": w0.name, "precision": prec, "scheme": scheme,
                             "nnz_train": int(trx.numel()), "factor_ms": f, "core_ms": c})
                m.close()
    if args.sweep in ("variants", "all"):
        # Algorithm 3 readings (per-set core SGD, reshuffle every iteration)
        # on the Netflix-shaped tensor: 10 epochs from the same start
        w0, tri, trx, tei, tex, A0, B0 = make_workload(dev, args.nnz, args.workload)
        nnz = int(trx.numel())
        epochs = 10
        gen = torch.Generator(device=dev)
        for variant, S, reshuffle in (("algorithm5", nnz, False), ("core_sgd", 10_000_000, False),
                                      ("core_sgd", 1_000_000, False), ("reshuffle", nnz, True)):
            gen.manual_seed(0)
            A = [a.clone() for a in A0]
            B = [b.clone() for b in B0]
            m = ft.FastTuckerPlus(tri, trx, A, B, precision=args.precision, hot_rows=args.hot_rows,
                                  hot_window=args.hot_window)
            lr_b = LR_B * S / nnz   # the same total core movement per epoch
            ms_core, ms_perm, curve = [], [], []
            for _ in range(epochs):
                if reshuffle:
                    perm = torch.randperm(nnz, generator=gen, device=dev).to(torch.int32)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    m.permute(perm)
                    e1.record(stream)
                    e1.synchronize()
                    ms_perm.append(e0.elapsed_time(e1))
                m.epoch_factors(LR, LAM)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if S >= nnz:
                    m.epoch_core(LR_B, LAM)
                else:
                    m.epoch_core_sgd(lr_b, LAM, S)
                e1.record(stream)
                curve.append(round(m.rmse(tei, tex)[0], 5))
                ms_core.append(e0.elapsed_time(e1))
            rows.append({"study": "variant", "workload": w0.name, "variant": variant, "set_size": S,
                         "lr_b": lr_b if S < nnz else LR_B, "core_ms": statistics.median(ms_core),
                         "permute_ms": statistics.median(ms_perm) if ms_perm else None,
                         "test_rmse_curve": curve})
            m.close()
    return {"metric": METRIC, "unit": UNIT, "sweep": args.sweep, "precision": args.precision,
            "steps": args.steps, "warmup": args.warmup, "peak_hbm_gbs": peak, "peak_kind": peak_kind,
            "data": "synthetic", "rows": rows}


def learned_step_ab(dev, epochs=20, lam=0.01, lr_b=0.01,
                    lrs=(0.005, 0.01, 0.02, 0.04, 0.08, 0.16, 0.32)):
    """The planted 3-order tensor (1e5 coordinates, planted J = R = 4, noise
    0.1) with uniform coordinates (the learned-step configuration) and with
    Zipf(1.1) coordinates: lambda = 0.01, core step 0.01, the learned per-row
    step against plain FP32 SGD at fixed factor steps `lrs` (eta* = the
    lowest test RMSE after `epochs` epochs); see learned_step.ab_study."""
    from paper_2404_10087_gb300 import learned_step as ls
    out = {}
    for name in ("planted_uniform_1e5", "planted_zipf_1e5"):
        w = synth.WORKLOADS[name]
        d = synth.draw_workload(w, device=dev)
        allidx = [d.idx[n].contiguous() for n in range(w.N)]
        pm = ft.FastTuckerPlus(allidx, torch.zeros(d.idx.shape[1], device=dev),
                               [a.contiguous() for a in d.planted_A], [b.contiguous() for b in d.planted_B],
                               hot_rows=0)
        x = pm.predict(allidx) + d.noise
        pm.close()
        tri = [d.idx[n, d.train].contiguous() for n in range(w.N)]
        tei = [d.idx[n, d.test].contiguous() for n in range(w.N)]
        xtr, xte = x[d.train].contiguous(), x[d.test].contiguous()

        def make_model(start, w=w, tri=tri, xtr=xtr):
            A, B = synth.initial_factors(w, device=dev, seed_offset=start)
            return ft.FastTuckerPlus(tri, xtr, A, B)

        out[name] = ls.ab_study(make_model, tei, xte, lrs, lam, lr_b, lam, epochs=epochs)
    return out


def time_to_rmse(w, tri, trx, tei, tex, dev, epochs, precision, window=3, starts=(1, 2, 3)):
    """Wall time for the mixed-precision run to reach the test RMSE of plain
    FP32 (the FP32-accurate mode), both from the same start, for several
    starts.  Hogwild test RMSE wobbles from epoch to epoch and the runs leave
    their initial plateau at slightly different epochs, so (a) a run reaches
    a threshold at the first epoch whose mean over the last `window` epochs
    is at or below it, and (b) the comparison is repeated from each start
    and the median speed-up is the headline.  Two thresholds: 'strict' = the
    FP32 run's final window mean after `epochs` epochs, and 'within_1pct' =
    1.01 x that.  An epoch is factor phase + core phase + test RMSE; times
    are CUDA events from the start of the run."""

    def run(A0, B0, prec, n_epochs):
        A = [a.clone() for a in A0]
        B = [b.clone() for b in B0]
        m = ft.FastTuckerPlus(tri, trx, A, B, precision=prec)
        stream = torch.cuda.current_stream(dev)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        curve, times = [], []
        for _ in range(n_epochs):
            m.epoch_factors(LR, LAM)
            m.epoch_core(LR_B, LAM)
            r = m.rmse(tei, tex)[0]
            t1 = torch.cuda.Event(enable_timing=True)
            t1.record(stream)
            t1.synchronize()
            curve.append(r)
            times.append(t0.elapsed_time(t1) / 1e3)
        m.close()
        return curve, times

    def first(curve, times, thr):
        for k in range(window - 1, len(curve)):
            if sum(curve[k - window + 1:k + 1]) / window <= thr:
                return k + 1, times[k]
        return None, None

    per_start = []
    for start in starts:
        A0, B0 = synth.initial_factors(w, device=dev, seed_offset=start)
        base_curve, base_times = run(A0, B0, "fp32", epochs)
        fast_curve, fast_times = run(A0, B0, precision, 3 * epochs)
        final = sum(base_curve[-window:]) / window
        one = {"start": start, "baseline_epoch_seconds": base_times[-1] / len(base_times),
               "candidate_epoch_seconds": fast_times[-1] / len(fast_times)}
        for name, thr in (("strict", final), ("within_1pct", 1.01 * final)):
            eb, tb = first(base_curve, base_times, thr)
            ec, tc = first(fast_curve, fast_times, thr)
            one[name] = {"target_test_rmse": thr, "baseline_epochs": eb, "baseline_seconds": tb,
                         "candidate_epochs": ec, "candidate_seconds": tc,
                         "speedup": (tb / tc) if (tb and tc) else None}
        one["baseline_curve"] = [round(v, 5) for v in base_curve]
        one["candidate_curve"] = [round(v, 5) for v in fast_curve]
        per_start.append(one)
    out = {"baseline": "fp32", "candidate": precision, "window": window, "starts": list(starts)}
    for name in ("strict", "within_1pct"):
        sp = [o[name]["speedup"] for o in per_start]
        ok = sorted(v for v in sp if v is not None)
        out[name] = {"speedups": sp,
                     "median_speedup": statistics.median(ok) if len(ok) == len(sp) else None}
    out["per_start"] = per_start
    return out


def oracle_sample(nnz_sample):
    """A bounded sample of the workload for the CPU oracle: the same recipe
    drawn at nnz_sample coordinates on the host, planted values by the oracle."""
    import oracle
    w = synth.WORKLOADS[WORKLOAD]
    d = synth.draw_workload(w, device="cpu", nnz=nnz_sample)
    pred = oracle.predict([a.double().numpy() for a in d.planted_A],
                          [b.double().numpy() for b in d.planted_B], d.idx.numpy(),
                          nthreads=oracle.default_threads())
    vals = synth.to_ratings(torch.from_numpy(pred))
    tr = d.train
    idx = np.ascontiguousarray(d.idx[:, tr].numpy())
    _, xc = synth.centre(vals[tr])
    x = xc.double().numpy()
    A, B = synth.initial_factors(w)
    return w, idx, x, [a.double().numpy() for a in A], [b.double().numpy() for b in B]


def time_oracle_step(idx, x, A, B, threads):
    """One step of the FP64 oracle on the host: the factor epoch as Hogwild on
    `threads` cores (each thread a contiguous range of the nonzeros, S = 1)
    and the core epoch (Algorithm 5, the sum split over the same threads)."""
    import oracle
    t = time.perf_counter()
    A = oracle.factor_epoch_hogwild(A, B, idx, x, LR, LAM, nthreads=threads)
    B = oracle.core_epoch(A, B, idx, x, LR_B, LAM, nthreads=threads)
    return time.perf_counter() - t, A, B


def time_oracle_sequential(idx, x, A, B):
    """The sequential oracle (factor epoch S = 1, one thread) on the same
    nonzeros: the single-core figure, for context."""
    import oracle
    t = time.perf_counter()
    A = oracle.factor_epoch(A, B, idx, x, 1, LR, LAM)
    B = oracle.core_epoch(A, B, idx, x, LR_B, LAM, nthreads=1)
    return time.perf_counter() - t


def cpu_baseline(nnz_sample, seq_sample=1_000_000):
    """The FP64 oracle on every host core over a bounded draw of the same
    recipe; its rate (nonzeros per second) is taken as the full workload's,
    since both phases are linear in the nonzeros."""
    import oracle
    w, idx, x, A, B = oracle_sample(nnz_sample)
    threads = oracle.default_threads()
    dt, _, _ = time_oracle_step(idx, x, A, B, threads)
    n = int(x.shape[0])
    k = min(n, seq_sample)
    dt1 = time_oracle_sequential(np.ascontiguousarray(idx[:, :k]), x[:k], A, B)
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} training nonzeros of the same recipe drawn at {nnz_sample} coordinates "
                      f"(rate extrapolated linearly to the full workload); one FP64 step: Hogwild factor "
                      f"epoch + core epoch on {threads} host threads, {dt:.2f} s",
            "sequential_1_thread": {"value": k / dt1, "unit": UNIT, "nnz": k,
                                    "what": "sequential factor epoch (S=1) + core epoch, one thread"}}


def run_reference(args, rank, world):
    import oracle
    if rank != 0:
        return None
    w, idx, x, A, B = oracle_sample(args.ref_sample)
    threads = oracle.default_threads()
    n = int(x.shape[0])
    for _ in range(args.warmup):
        _, A, B = time_oracle_step(idx, x, A, B, threads)
    ts = []
    for _ in range(args.steps):
        dt, A, B = time_oracle_step(idx, x, A, B, threads)
        ts.append(dt)
    tot = sum(ts)
    value = n * len(ts) / tot
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(ts),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Zipf coordinates, planted-model ratings, centred; Netflix-shaped)",
        "config": {"workload": WORKLOAD, "N": w.N, "I": list(w.I), "J": list(w.J), "R": w.R,
                   "nnz_train_sample": n, "precision": "fp64", "scatter": "hogwild (host threads)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{n} training nonzeros per step (same recipe at {args.ref_sample} "
                                   f"coordinates); FP64 Hogwild factor epoch + core epoch on {threads} "
                                   f"host threads; rate extrapolated linearly to the full workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "tf32", "bf16"], default=None,
                    help="contraction precision (default: bf16; fp32 for the batched workload, "
                         "whose configuration is FP32)")
    ap.add_argument("--cpu-sample", type=int, default=10_000_000)
    ap.add_argument("--ref-sample", type=int, default=4_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-rmse", action="store_true")
    ap.add_argument("--ttr-epochs", type=int, default=20,
                    help="epochs of the plain FP32 run that sets the time-to-RMSE target")
    ap.add_argument("--hot-rows", type=int, default=None,
                    help="rows per mode in the shared-memory hot-row cache (-1 auto, 0 off)")
    ap.add_argument("--hot-window", type=int, default=None,
                    help="cache write-back every hot_window x 128 nonzeros of a CTA")
    ap.add_argument("--engine", choices=["warp", "tcgen05"], default="warp",
                    help="factor-pass kernels: 16-nonzero warp tiles (mma.sync) or 128-nonzero "
                         "warpgroup tiles (tcgen05.mma, TMEM)")
    ap.add_argument("--l2-persist", type=int, choices=[0, 1], default=0,
                    help="mark the factor matrices persisting in L2 for the library's launches "
                         "(measured slower on this workload, so off by default)")
    ap.add_argument("--core-scheme", choices=["calc", "store"], default="calc",
                    help="core phase: rows of C formed per nonzero, or gathered from C = A B "
                         "precomputed once per core phase (Sec. 5.6)")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS) + [BATCHED],
                    help="the timed tensor (default: the Netflix-shaped 1e8 Zipf tensor)")
    ap.add_argument("--sweep", choices=["orders", "ranks", "schemes", "variants", "all"], default=None,
                    help="instead of the headline line: the order sweep N = 3..10, the (R, J) "
                         "sweep, the core-phase schemes (calculation vs storage) per precision, "
                         "and/or the Algorithm 3 variants (per-set core SGD, reshuffle every "
                         "epoch); per-iteration phase times")
    ap.add_argument("--nnz", type=int, default=None,
                    help="distinct coordinates drawn (default: the workload's 1e8); "
                         "a smaller case of the same recipe, e.g. for profiling")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.precision is None:
        args.precision = "fp32" if args.workload == BATCHED else "bf16"

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group(backend)
    try:
        if args.impl == "reference":
            out = run_reference(args, rank, world)
        elif args.sweep:
            out = run_sweep(args, local_rank) if rank == 0 else None
        else:
            out = run_ours(args, rank, world, local_rank)
        if out is not None:
            print(json.dumps(out), flush=True)
    finally:
        if world > 1:
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
