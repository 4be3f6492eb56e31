"""Stored values of tests/golden/: the closed forms are consistent with their
expressions, and the oracle reproduces the values make_golden.py wrote from it
(a regression pin: a change to the oracle's arithmetic shows here)."""

import math

import numpy as np
import pytest

from conftest import golden, oracle_processes
from workloads import make_workload, wavy_torus


def test_closed_forms_match_their_expressions():
    g = golden("closed_forms.json")
    assert g["sphere_remainder_constant"]["value"] == pytest.approx(-1 / (4 * math.pi), rel=1e-15)
    ev = g["sphere_parametrix_eigenvalues"]
    assert ev["value"] == pytest.approx([-1 / (l * (l + 1)) for l in ev["l"]], rel=1e-15)
    assert g["sphere_parametrix_constant"]["value"] == pytest.approx(2 * math.log(2) - 1, rel=1e-15)
    lb = g["sphere_laplace_beltrami_eigenvalues"]
    assert lb["value"] == [-float(l * (l + 1)) for l in lb["l"]]
    for k, v in g.items():
        assert v["source"], k


def test_wavy_torus_volume_from_the_fixture():
    s = wavy_torus(51, 18, 8)
    vol = golden("closed_forms.json")["wavy_torus_volume"]["value"]
    assert abs(np.dot(s.weights, np.sum(s.nodes * s.normals, 1)) / 3 - vol) < 1e-12 * vol


@pytest.mark.parametrize("name", ["ellipsoid_small", "wavy_torus_small"])
def test_oracle_reproduces_stored_applies(name):
    from oracle.operator import Discretization, NearField, apply_K, apply_R
    case = golden("oracle_applies.json")["cases"][name]
    wl = make_workload(name)
    assert wl.N == case["N"]
    rows = case["rows"]
    d = Discretization.from_workload(wl)
    nf = NearField(d, rows=rows, processes=oracle_processes())
    sigma = np.random.default_rng(2024).standard_normal(wl.N) + 1.0
    R, K = np.array(case["R"]), np.array(case["K"])
    assert np.abs(apply_R(d, nf, sigma, rows) - R).max() <= 1e-11 * np.abs(R).max()
    assert np.abs(apply_K(d, nf, sigma, rows) - K).max() <= 1e-11 * np.abs(K).max()
