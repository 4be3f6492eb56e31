"""Writes the stored expected values under tests/golden/ from the oracle alone.

The CUDA library is not imported here: every stored value is either a closed
form that follows from the paper's formulas (closed_forms.json, each with its
source) or the float64 oracle's result on a seeded input (oracle_applies.json).

    python tests/golden/make_golden.py
"""

import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

CASES = ("ellipsoid_small", "wavy_torus_small")   # variable a; the paper's wavy torus
SIGMA_SEED = 2024                                 # sigma = N(0,1) + 1, numpy default_rng(seed)


def closed_forms():
    ls = [1, 2, 3, 4, 5, 6]
    return {
        "sphere_remainder_constant": {
            "value": -1.0 / (4.0 * math.pi), "expr": "-1/(4 pi)",
            "source": "eq. explicit_remainderLB with n = x, H = 1 on the unit sphere; "
                      "eq. limiting_behaviour"},
        "sphere_parametrix_eigenvalues": {
            "l": ls, "value": [-1.0 / (l * (l + 1)) for l in ls], "expr": "-1/(l(l+1))",
            "source": "eq. parametrixLB on the unit sphere (Funk-Hecke: the integral of "
                      "log(1 - t) P_l(t) over [-1, 1] is -2/(l(l+1)))"},
        "sphere_parametrix_constant": {
            "value": 2.0 * math.log(2.0) - 1.0, "expr": "2 ln 2 - 1",
            "source": "eq. parametrixLB applied to 1 on the unit sphere"},
        "sphere_laplace_beltrami_eigenvalues": {
            "l": ls, "value": [-float(l * (l + 1)) for l in ls], "expr": "-l(l+1)",
            "source": "Sec. 7.1 (Y_l^m are eigenfunctions of the Laplace-Beltrami operator)"},
        "wavy_torus_volume": {
            "value": 6.0 * math.pi ** 2, "expr": "6 pi^2",
            "source": "Sec. 7 parametrisation: each half-plane at angle u cuts a unit disk "
                      "centred at radius 3 + 0.6 cos 5u"},
    }


def sample_rows(N, pp, stride=13):
    """Every stride-th row plus the first and last node of the first and last patch."""
    return sorted(set(list(range(0, N, stride)) + [0, pp - 1, N - pp, N - 1]))


def oracle_applies(processes):
    import numpy as np
    from oracle.operator import Discretization, NearField, apply_K, apply_R
    from workloads import make_workload
    out = {}
    for name in CASES:
        wl = make_workload(name)
        d = Discretization.from_workload(wl)
        rows = sample_rows(wl.N, wl.surface.p ** 2)
        nf = NearField(d, rows=rows, processes=processes)
        sigma = np.random.default_rng(SIGMA_SEED).standard_normal(wl.N) + 1.0
        out[name] = {"N": wl.N, "sigma": "numpy default_rng(%d).standard_normal(N) + 1" % SIGMA_SEED,
                     "rows": rows,
                     "R": [float(v) for v in apply_R(d, nf, sigma, rows)],
                     "K": [float(v) for v in apply_K(d, nf, sigma, rows)]}
    return out


if __name__ == "__main__":
    sys.path.insert(0, ROOT)
    procs = max(1, min(8, os.cpu_count() or 1))
    with open(os.path.join(HERE, "closed_forms.json"), "w") as fh:
        json.dump(closed_forms(), fh, indent=1)
    with open(os.path.join(HERE, "oracle_applies.json"), "w") as fh:
        json.dump({"note": "float64 oracle applies of R~ and K~ (eq. explicit_remainder, "
                           "eq. diff_param, Sec. 6.1 quadrature) on seeded inputs, at "
                           "sampled rows",
                   "cases": oracle_applies(procs)}, fh)
    print("written")
