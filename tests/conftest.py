"""Test configuration: the ``gpu`` marker and shared oracle fixtures."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU and the compiled sm_103a library")


def golden(name):
    """A stored fixture of tests/golden/ (closed forms with their sources, or values
    written by tests/golden/make_golden.py from the oracle alone)."""
    import json
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as fh:
        return json.load(fh)


def oracle_processes():
    """Worker processes for the oracle's near-field build (spawned, CPU only)."""
    n = os.cpu_count() or 1
    return max(1, min(16, n))
