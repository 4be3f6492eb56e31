"""The reference arm of bench.py (no GPU): its oracle leg runs as a CPU-only
subprocess on every host core (spawned worker processes, one BLAS thread each)
and on one core, and the JSON line carries the keys the benchmark contract names."""

import json
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.run_oracle_subprocess("ellipsoid_small", 0.5)
    cores = bench.host_cores()
    assert r["value"] > 0 and r["value_1core"] > 0 and r["cores"] == cores
    assert "ellipsoid_small" in r["sample"] and f"on {cores} process(es)" in r["sample"]
    assert "on 1 process(es)" in r["sample_1core"]
    args = SimpleNamespace(steps=2, warmup=1, workload="ellipsoid_small")
    line = bench.reference_line(args, [r["value"] * 2, r["value"], r["value"]], r["sample"],
                                cores)
    text = json.dumps(line, allow_nan=False)               # strict JSON
    back = json.loads(text)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better",
              "impl", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in back, k
    assert back["impl"] == "reference" and back["value"] == r["value"]    # warm-up excluded
    assert back["metric"] == bench.METRIC and back["unit"] == bench.UNIT
    assert back["cpu_baseline"]["cores"] == cores and back["cpu_baseline"]["kind"] == "oracle"
    assert back["e2e"]["h2d_bytes_per_step"] == 0 and back["e2e"]["value"] == back["value"]


def test_oracle_runner_counts_rows_on_each_process():
    """Every worker evaluates disjoint chunks for the given wall time; the rate with more
    processes is not below the one-process rate by more than scheduling noise."""
    sys.path.insert(0, ROOT)
    import bench
    runner = bench.OracleRunner("ellipsoid_small", 2)
    try:
        v2, d2 = runner.rate(0.5)
        v1, d1 = runner.rate(0.5, processes=1)
    finally:
        runner.close()
    assert v1 > 0 and v2 > 0.5 * v1
    assert "on 2 process(es)" in d2 and "on 1 process(es)" in d1
