"""The benchmark's CPU baselines of the batch and gradient workloads, run on tiny samples (no GPU): the oracle
calls they make, the extrapolation to the whole workload, and the keys of a cpu_baseline object."""
import numpy as np

import bench
from paper_1406_5802_gb300 import workloads as W

CPU_KEYS = {"value", "unit", "cores", "kind", "sample"}


def test_batch_baseline_extrapolates_by_flops(orc):
    sizes = np.array([8, 20, 33, 40])
    systems = [(A, b) for A, b, _ in W.batch_systems(sizes[:2], seed=3)]
    out = bench.oracle_batch_baseline(systems, sizes, seed=3, threads=1)
    assert CPU_KEYS <= set(out) and out["kind"] == "oracle" and out["cores"] == 1
    assert out["max_berr_sample"] <= 1e-13
    assert out["value"] > 0 and abs(out["value"] * out["ms_per_batch"] / 1e3 - len(sizes)) < 1e-9
    # the sample's time scales by the flop ratio of the whole batch to the sample
    ratio = sum(bench.batch_flops(int(n)) for n in sizes) / sum(bench.batch_flops(int(n)) for n in sizes[:2])
    assert ratio > 10


def test_grad_baseline_runs_forward_and_adjoint(orc):
    systems = [W.grad_system(48, 4, seed=5), W.grad_system(40, 4, seed=6)]
    out = bench.oracle_grad_baseline(systems, count=64, seed=5, threads=1)
    assert CPU_KEYS <= set(out) and out["unit"] == "systems/s"
    assert out["value"] > 0 and abs(out["value"] * out["ms_per_batch"] / 1e3 - 64) < 1e-9
