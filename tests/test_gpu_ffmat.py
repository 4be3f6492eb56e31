"""Stored float-float smooth-sum matrices (pm_surface_store_ff) against the oracle.

* The stored remainder and parametrix applies match the float64 oracle like the
  unstored float-float sums do (1e-11 relative L2; 864 and 384 nodes, ld = 896 and
  384: a ragged and an exact 64-column tail; the parametrix matrix in the symmetric
  tile layout and in the row layout), the unstored float-float sums to 5e-12 of the
  largest entry (the stored format keeps each entry to 2^-40 of its magnitude, against
  ~2^-46 for the float-float evaluation; the errors have random signs, so a row's
  error stays near 2^-40 |y|) and themselves bit for bit.
* Full size (ellipsoid 9,600 and the 98,304-node torus the bench times, the GEMVs in
  the launch shapes of the solve): sampled rows against the oracle at 1e-10 of the row
  maximum.
* Storing one kernel leaves the other on the pair-by-pair path; release restores it;
  set_coeff re-evaluates the stored remainder (compared with a fresh surface of the
  new coefficient); clones do not inherit; a c != 0 coefficient releases them.
* A solve whose residuals and representation read the stored matrices returns the
  unstored solve's solution to 10 x the tolerance, and its true residual (recomputed from sigma
  with unstored float-float applies) meets the tolerance.
* Too little free memory (PM_FAKE_HBM_BYTES in a child process) refuses the store
  with PM_ERR_OOM and leaves the surface working.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import oracle_processes
from workloads import make_workload

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INVALID, OOM, NO_COEFF = 1, 2, 9          # pm_status values of include/parametrix.h
_ORACLE = {}


def oracle(name, rows=None):
    from oracle.operator import Discretization, NearField
    key = (name, None if rows is None else tuple(rows))
    if key not in _ORACLE:
        wl = make_workload(name)
        d = Discretization.from_workload(wl)
        nf = NearField(d, rows=rows, processes=oracle_processes())
        _ORACLE[key] = (wl, d, nf)
    return _ORACLE[key]


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_12501_gb300 as pm
    c = pm.Context(0)
    yield c
    c.close()


def surface(ctx, name, a_scale=1.0):
    import paper_2401_12501_gb300 as pm
    wl = make_workload(name)
    s = pm.Surface.from_fixture(ctx, wl.surface)
    s.set_coeff(a_scale * wl.coeff.a, a_scale * wl.coeff.grad_a)
    return wl, s


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name,sym", [("ellipsoid_small", 1), ("sphere_384", 1),
                                      ("ellipsoid_small", 0)])
def test_stored_apply_matches_oracle(ctx, name, sym):
    """sym = 1: the parametrix matrix in the symmetric tile layout (7 and 3 tiles of
    128, ragged and exact); sym = 0: both matrices in the row layout."""
    import paper_2401_12501_gb300 as pm
    from oracle.operator import apply_K, apply_R
    wl, d, nf = oracle(name)
    o = pm.default_opts()
    o.direct_symmetric = sym
    s = pm.Surface.from_fixture(ctx, wl.surface, o)
    s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
    sigma = np.random.default_rng(31).standard_normal(d.N) + 1.0
    yR0, yK0 = s.apply_R(sigma, "ff"), s.apply_K(sigma, "ff")     # pair by pair
    s.store_ff("RK")
    assert s.stored_ff() == "RK"
    yR, yK = s.apply_R(sigma, "ff"), s.apply_K(sigma, "ff")
    assert rel(yR, apply_R(d, nf, sigma)) < 1e-11
    assert rel(yK, apply_K(d, nf, sigma)) < 1e-11
    assert np.abs(yR - yR0).max() <= 5e-12 * np.abs(yR0).max()
    assert np.abs(yK - yK0).max() <= 5e-12 * np.abs(yK0).max()
    assert np.array_equal(yR, s.apply_R(sigma, "ff"))          # fixed-order reductions
    assert np.array_equal(yK, s.apply_K(sigma, "ff"))
    s.close()


def test_stored_full_size_rows(ctx):
    from oracle.operator import apply_K, apply_R
    name = "ellipsoid_9600"
    wl = make_workload(name)
    rng = np.random.default_rng(32)
    rows = sorted(set([0, 1, wl.N - 1] + [int(i) for i in rng.integers(0, wl.N, 10)]))
    _, d, nf = oracle(name, rows)
    _, s = surface(ctx, name)
    s.store_ff("RK")
    sigma = rng.standard_normal(wl.N) + 1.0
    oR = apply_R(d, nf, sigma, rows)
    oK = apply_K(d, nf, sigma, rows)
    assert np.abs(s.apply_R(sigma, "ff")[rows] - oR).max() < 1e-10 * np.abs(oR).max()
    assert np.abs(s.apply_K(sigma, "ff")[rows] - oK).max() < 1e-10 * np.abs(oK).max()
    s.close()


def test_stored_full_size_torus_rows(ctx):
    """The 98,304-node torus in the layout the bench times (87 GB of stored matrices):
    sampled rows of both stored applies against the oracle."""
    from oracle.operator import apply_K, apply_R
    name = "torus_98304"
    wl = make_workload(name)
    rng = np.random.default_rng(35)
    rows = sorted(set([0, wl.N - 1] + [int(i) for i in rng.integers(0, wl.N, 8)]))
    _, d, nf = oracle(name, rows)
    _, s = surface(ctx, name)
    s.store_ff("RK")
    assert s.stored_ff() == "RK"
    sigma = np.cos(3 * wl.surface.nodes[:, 0]) + 0.5 * rng.standard_normal(wl.N)
    oR = apply_R(d, nf, sigma, rows)
    oK = apply_K(d, nf, sigma, rows)
    yR = s.apply_R(sigma, "ff")
    yK = s.apply_K(sigma, "ff")
    s.close()
    assert np.abs(yR[rows] - oR).max() < 1e-10 * np.abs(oR).max()
    assert np.abs(yK[rows] - oK).max() < 1e-10 * np.abs(oK).max()


def test_partial_store_release_coefficient_and_clone(ctx):
    name = "ellipsoid_2400"
    wl, s = surface(ctx, name)
    sig = np.random.default_rng(33).standard_normal(wl.N)
    ref = {op: getattr(s, "apply_" + op)(sig, "ff") for op in "RK"}

    def close_to_ref(t, r):
        return np.abs(t - r).max() <= 5e-12 * np.abs(r).max()

    s.store_ff("R")
    assert s.stored_ff() == "R"
    assert close_to_ref(s.apply_R(sig, "ff"), ref["R"])
    assert np.array_equal(s.apply_K(sig, "ff"), ref["K"])          # unstored path, unchanged
    s.store_ff("K")                                                   # replaces the R matrix
    assert s.stored_ff() == "K"
    assert close_to_ref(s.apply_K(sig, "ff"), ref["K"])
    assert np.array_equal(s.apply_R(sig, "ff"), ref["R"])
    s.store_ff("")
    assert s.stored_ff() == ""
    assert np.array_equal(s.apply_R(sig, "ff"), ref["R"])
    # a new coefficient re-evaluates the stored remainder matrix
    s.store_ff("RK")
    c = s.clone()
    assert c.stored_ff() == ""
    s.set_coeff(2.0 + wl.coeff.a, wl.coeff.grad_a)
    c.set_coeff(2.0 + wl.coeff.a, wl.coeff.grad_a)
    assert s.stored_ff() == "RK"
    for op in "RK":
        t = getattr(s, "apply_" + op)(sig, "ff")
        r = getattr(c, "apply_" + op)(sig, "ff")
        assert close_to_ref(t, r), op
    # c != 0 releases the matrices
    s.set_coeff_c(wl.coeff.a, wl.coeff.grad_a, -3.0)
    assert s.stored_ff() == ""
    c.close()
    s.close()


@pytest.mark.parametrize("name", ["ellipsoid_9600", "torus_6144"])
def test_solve_with_stored_matrices(ctx, name):
    wl = make_workload(name)
    _, s0 = surface(ctx, name)
    _, s1 = surface(ctx, name)
    s1.store_ff("RK")
    u0, i0, sig0 = s0.solve(wl.f, tol=1e-10, prec="fp32", return_sigma=True)
    u1, i1, sig1 = s1.solve(wl.f, tol=1e-10, prec="fp32", return_sigma=True)
    w = wl.surface.weights
    nrm = np.sqrt(np.dot(w, u0 * u0))
    assert np.sqrt(np.dot(w, (u1 - u0) ** 2)) < 1e-9 * nrm
    # the true residual of the stored solve's sigma, with unstored float-float applies
    r = wl.f - (sig1 + s0.apply_R(sig1, "ff") + np.dot(w, sig1))
    assert np.linalg.norm(r) / np.linalg.norm(wl.f) <= 1e-10
    assert i1[0].residual <= 1e-10
    s0.close()
    s1.close()


def test_invalid_arguments(ctx):
    import paper_2401_12501_gb300 as pm
    from paper_2401_12501_gb300 import _lib
    lib = _lib.lib()
    assert lib.pm_surface_store_ff(None, 3) == INVALID
    assert lib.pm_surface_stored_ff(None) == 0
    wl, s = surface(ctx, "sphere_384")
    assert lib.pm_surface_store_ff(s.handle, 4) == INVALID
    assert lib.pm_surface_store_ff(s.handle, -1) == INVALID
    t = pm.Surface.from_fixture(ctx, wl.surface)
    assert lib.pm_surface_store_ff(t.handle, 3) == NO_COEFF
    t.close()
    s.close()


_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
import paper_2401_12501_gb300 as pm
from paper_2401_12501_gb300 import _lib
from workloads import make_workload
wl = make_workload("sphere_384")
ctx = pm.Context(0)
s = pm.Surface.from_fixture(ctx, wl.surface)
s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
sig = np.random.default_rng(34).standard_normal(wl.N)
y0 = s.apply_R(sig, "ff")
st = _lib.lib().pm_surface_store_ff(s.handle, 3)
y1 = s.apply_R(sig, "ff")
print(json.dumps({{"status": st, "stored": s.stored_ff(), "same": bool(np.array_equal(y0, y1))}}))
"""


def test_store_refused_without_free_memory(ctx):
    env = dict(os.environ, PM_FAKE_HBM_BYTES="1000000")
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], capture_output=True,
                       text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out == {"status": OOM, "stored": "", "same": True}
