"""Host logic of bench.py that needs no GPU: the roofline's recorded DRAM
traffic is reported only for the launch it was captured on (the kernel
source, the full-size default workload, the warp-tile engine and the hot-row
write-back window), and the factor pass's algorithmic bytes follow the byte
model (coordinates and value read, N rows read and written)."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def recorded_window():
    text = open(os.path.join(ROOT, "profiles", "ncu_factor_netflix_zipf.md")).read()
    m = re.search(r"hot_window:\s*([0-9]+)", text)
    return int(m.group(1)) if m else None


def test_traffic_only_for_the_captured_launch():
    w = recorded_window()
    t = bench.recorded_traffic("bf16", hot_window=w)
    # captured on the current kernel source: a number, a few tens of bytes per
    # nonzero of the 9e7-nonzero launch
    assert t is not None and 9e7 * 10 < t < 9e7 * 100
    assert bench.recorded_traffic("bf16", hot_window=w + 1) is None
    assert bench.recorded_traffic("bf16", nnz=10_000_000, hot_window=w) is None
    assert bench.recorded_traffic("bf16", engine="tcgen05", hot_window=w) is None
    assert bench.recorded_traffic("bf16", workload="order4_zipf_2e8", hot_window=w) is None
    assert bench.recorded_traffic("fp32", hot_window=w) is None


def test_factor_byte_model():
    # N = 3, J = 16: 3 coordinates + 1 value (16 B) + 3 rows of 64 B read and written
    assert bench.algorithmic_bytes_factor(3, [16, 16, 16]) == 400
    # order 4, J = 32
    assert bench.algorithmic_bytes_factor(4, [32] * 4) == 1044
    # the small configuration, J = 4
    assert bench.algorithmic_bytes_factor(3, [4, 4, 4]) == 112


def test_workload_recipes_match_the_configurations():
    """The benchmark's recipes carry the configurations' sizes: the planted
    small tensor, the Netflix-shaped Zipf(1.1) ratings tensor, the order-4
    Zipf(1.05) tensor and the 64 batched tensors' ranges."""
    from paper_2404_10087_gb300 import synth
    w = synth.WORKLOADS["planted_uniform_1e5"]
    assert (w.I, w.nnz, w.J, w.R, w.dist, w.noise_std) == (
        (1000,) * 3, 100_000, (4,) * 3, 4, "uniform", 0.1)
    w = synth.WORKLOADS["netflix_shaped_zipf_1e8"]
    assert (w.I, w.nnz, w.J, w.R, w.dist, w.zipf_s, w.ratings, w.test_frac) == (
        (480_000, 18_000, 2_200), 100_000_000, (16,) * 3, 16, "zipf", 1.1, True, 0.1)
    w = synth.WORKLOADS["order4_zipf_2e8"]
    assert (w.I, w.nnz, w.J, w.R, w.dist, w.zipf_s, w.noise_std) == (
        (1_000_000, 1_000_000, 100_000, 1_000), 200_000_000, (32,) * 4, 32, "zipf", 1.05, 0.05)
    rec = synth.batched_recipe(64, seed=0)
    assert len(rec) == 64
    for w in rec:
        assert w.N in (3, 4, 5) and 10_000 <= w.nnz <= 1_000_000
        assert all(1_000 <= In <= 100_000 for In in w.I)
        assert len(set(w.J)) == 1 and w.J[0] in (4, 8, 16) and w.R in (8, 16, 32)
        assert w.dist == "uniform" and w.noise_std == 0.1
    # the draw is seeded: the same recipe again
    again = synth.batched_recipe(64, seed=0)
    assert [(w.I, w.nnz, w.J, w.R) for w in again] == [(w.I, w.nnz, w.J, w.R) for w in rec]
