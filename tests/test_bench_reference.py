"""The reference arm of bench.py (no GPU): its oracle leg runs as a CPU-only
subprocess and the JSON line carries the keys the benchmark contract names."""

import json
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.run_oracle_subprocess("ellipsoid_small", 0.5)
    assert r["value"] > 0 and "ellipsoid_small" in r["sample"] and "1 thread" in r["sample"]
    args = SimpleNamespace(steps=2, warmup=1, workload="ellipsoid_small")
    line = bench.reference_line(args, [r["value"] * 2, r["value"], r["value"]], r["sample"])
    text = json.dumps(line, allow_nan=False)               # strict JSON
    back = json.loads(text)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better",
              "impl", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in back, k
    assert back["impl"] == "reference" and back["value"] == r["value"]    # warm-up excluded
    assert back["metric"] == bench.METRIC and back["unit"] == bench.UNIT
    assert back["cpu_baseline"]["cores"] == 1 and back["cpu_baseline"]["kind"] == "oracle"
    assert back["e2e"]["h2d_bytes_per_step"] == 0 and back["e2e"]["value"] == back["value"]
