"""Autotuner cache: tuned launch shapes per (GPU, surface-size bucket, nrhs, precision).

A JSON object on disk maps keys from ``tune_key`` to the autotuner's result
(the knobs of ``pm_knobs`` and the timings).  Only host-side bookkeeping lives
here: the timing itself is ``pm_surface_autotune`` in the CUDA library.
"""

from __future__ import annotations

import json
import math
import os
import tempfile

KNOB_FIELDS = ("direct_tpt", "direct_blocks_per_sm", "batch_rhs_per_block",
               "batch_blocks_per_sm", "fmm_depth", "fmm_streams")


def size_bucket(n: int) -> int:
    """Nearest power of two to n in log scale (sizes within a factor sqrt(2) share a bucket)."""
    if n < 1:
        raise ValueError("size must be positive")
    return 1 << int(round(math.log2(n)))


def tune_key(gpu: str, n: int, nrhs: int, prec: str) -> str:
    return f"{gpu}|N~{size_bucket(n)}|nrhs={int(nrhs)}|{prec}"


def load(path: str) -> dict:
    """The cache at path ({} when missing or unreadable)."""
    try:
        with open(path) as fh:
            data = json.load(fh)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def valid_entry(entry) -> bool:
    return (isinstance(entry, dict) and isinstance(entry.get("knobs"), dict)
            and all(isinstance(entry["knobs"].get(f), int) for f in KNOB_FIELDS))


def store(path: str, key: str, entry: dict) -> None:
    """Add or replace one entry (read, update, write to a temporary file, rename)."""
    if not valid_entry(entry):
        raise ValueError("cache entry needs integer knobs " + ", ".join(KNOB_FIELDS))
    data = load(path)
    data[key] = entry
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".tunecache", dir=d)
    try:
        with os.fdopen(fd, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise
