"""The benchmark's contract on the CPU: the intersection count behind the roofline,
and the reference arm's JSON line (the FP64 oracle timed on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import oracle as O  # noqa: E402


@pytest.mark.parametrize("N,V,U", [(64, 90, 95), (96, 120, 137)])
def test_intersection_count_matches_the_explicit_matrix(N, V, U):
    """The roofline's algorithmic work per projection, n sum_v (|cos| + |sin|) d/ds,
    is the expected number of ray-pixel intersections.  The explicit matrix has a
    few more: rays of the two axis-aligned views that run along pixel edges meet
    both neighbours.  So the formula stays within 2 % and never above the count."""
    og = O.Geometry(N, V=V, U=U)
    nnz = int((O.CSR(og).va != 0).sum())
    est = bench.nnz_per_projection(N, V, U)
    assert est <= nnz
    assert est >= 0.98 * nnz


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` runs the oracle on the benchmark's workload and
    prints one JSON line with the contract's keys, its own value as the CPU
    baseline and an end-to-end figure with no device copies."""
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["metric"] == "SupPCG iterations/s" and d["unit"] == "iterations/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"] == bench.workload_config(1)   # the GPU arm's config, key for key
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_both_arms_take_the_same_data():
    """b is generated once from the analytic sinogram (no projector of either arm
    involved), rounded to FP32; the oracle arm widens the same array."""
    b1 = bench.workload_data()
    b2 = bench.workload_data()
    assert b1.dtype.name == "float32" and b1.shape == (bench.WL["V"], bench.WL["U"])
    assert (b1 == b2).all()
