"""GPU boundary-value systems (pm_bvp_*, Sec. 5.2 Neumann, Sec. 5.3 Dirichlet) against the oracle.

* The device operator (surface rows and edge rows, rank-one term included) equals
  the oracle's element by element on random (sigma, mu) for a torus band of 288
  nodes and 2 x 16 edge nodes, F = 16 (1e-10 of the largest value; the two sides
  use different quadrature rules for K'_Gamma on the edge patch, each converged to
  ~1e-12).
* The device solve of the manufactured Newtonian problem equals the oracle's dense
  solve (u to 1e-9, up to the additive constant of the Neumann problem) and both
  reach the exact solution to the same discretisation error; on finer bands the
  error keeps falling (3.5e-7 and below).
* Dirichlet (a = 1): the operator equals the oracle's element by element (1e-10),
  the solve the oracle's dense solve (1e-9) and the exact solution (2.2e-8 at 512
  nodes, F = 32), converging on finer bands.
* Invalid arguments (no coefficient, a node off its patch's edge, an unknown patch,
  a variable coefficient for Dirichlet) are refused before anything runs.
"""

import numpy as np
import pytest

from conftest import oracle_processes
from workloads.bvp import (band_coefficient, constant_band_coefficient, edge_a, edge_patches,
                           newtonian_dirichlet, newtonian_neumann, torus_band)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_12501_gb300 as pm
    c = pm.Context(0)
    yield c
    c.close()


def device_bvp(ctx, os_, kind="neumann"):
    import paper_2401_12501_gb300 as pm
    co = band_coefficient(os_) if kind == "neumann" else constant_band_coefficient(os_)
    s = pm.Surface.from_fixture(ctx, os_.surface)
    s.set_coeff(co.a, co.grad_a)
    patch, uv = edge_patches(os_)
    if kind == "neumann":
        ae, ao = edge_a(os_), edge_a(os_, True)
    else:
        ae, ao = np.ones(os_.M), np.ones(sum(c.F * c.M for c in os_.curves))
    b = pm.BoundaryValueProblem(s, os_.curves, ae, ao, patch, uv, kind=kind)
    return s, b, co


def rel_err_mod_const(u, v, w):
    e = (u - v) - np.dot(w, u - v) / w.sum()
    vv = v - np.dot(w, v) / w.sum()
    return float(np.sqrt(np.dot(w, e * e) / np.dot(w, vv * vv)))


@pytest.fixture(scope="module")
def coarse(ctx):
    from oracle.bvp import NeumannBVP as OracleBVP
    os_ = torus_band(2, 4, 6, 16, 16)
    s, b, co = device_bvp(ctx, os_)
    ora = OracleBVP(os_, co, edge_a(os_), edge_a(os_, True), processes=oracle_processes())
    yield os_, s, b, co, ora
    b.close()
    s.close()


def test_operator_matches_oracle(coarse):
    os_, s, b, co, ora = coarse
    rng = np.random.default_rng(41)
    sigma = rng.standard_normal(s.N) + 1.0
    mu = rng.standard_normal(b.Me)
    ys, ye = b.apply(sigma, mu)
    os_ref, oe_ref = ora.apply(sigma, mu)
    assert np.all(np.isfinite(ys)) and np.all(np.isfinite(ye))
    assert np.abs(ys - os_ref).max() <= 1e-10 * np.abs(os_ref).max()
    assert np.abs(ye - oe_ref).max() <= 1e-10 * np.abs(oe_ref).max()
    # the parts separately: mu only (edge-sourced operators) and sigma only
    ys2, ye2 = b.apply(np.zeros(s.N), mu)
    r2s, r2e = ora.apply(np.zeros(s.N), mu)
    assert np.abs(ys2 - r2s).max() <= 1e-10 * np.abs(r2s).max()
    assert np.abs(ye2 - r2e).max() <= 1e-10 * np.abs(r2e).max()


def test_solve_matches_oracle_and_exact_solution(coarse):
    os_, s, b, co, ora = coarse
    f, fg, v = newtonian_neumann(os_, co)
    u, info, sig, mu = b.solve(f, fg, tol=1e-13)
    assert info.residual <= 1e-13
    _, _, u_ref = ora.solve(f, fg)
    w = os_.surface.weights
    assert rel_err_mod_const(u, u_ref, w) < 1e-9
    e_dev, e_ora = rel_err_mod_const(u, v, w), rel_err_mod_const(u_ref, v, w)
    assert e_dev < 5e-6 and abs(e_dev - e_ora) < 1e-8, (e_dev, e_ora)


@pytest.mark.parametrize("args,bound", [((2, 4, 8, 32, 16), 6e-7), ((4, 8, 8, 64, 16), 1e-7)])
def test_refined_bands_converge(ctx, args, bound):
    os_ = torus_band(*args)
    s, b, co = device_bvp(ctx, os_)
    f, fg, v = newtonian_neumann(os_, co)
    u, info, _, _ = b.solve(f, fg, tol=1e-13)
    err = rel_err_mod_const(u, v, os_.surface.weights)
    assert err < bound, err
    b.close()
    s.close()


def test_invalid_arguments(ctx):
    import paper_2401_12501_gb300 as pm
    os_ = torus_band(2, 4, 6, 16, 4)
    co = band_coefficient(os_)
    s = pm.Surface.from_fixture(ctx, os_.surface)
    patch, uv = edge_patches(os_)
    with pytest.raises(pm.PmError):                         # no coefficient yet
        pm.NeumannBVP(s, os_.curves, edge_a(os_), edge_a(os_, True), patch, uv)
    s.set_coeff(co.a, co.grad_a)
    bad = uv.copy()
    bad[0, 0] = 0.5                                         # not on a patch edge
    with pytest.raises(pm.PmError):
        pm.NeumannBVP(s, os_.curves, edge_a(os_), edge_a(os_, True), patch, bad)
    badp = patch.copy()
    badp[1] = s.N                                           # no such patch
    with pytest.raises(pm.PmError):
        pm.NeumannBVP(s, os_.curves, edge_a(os_), edge_a(os_, True), badp, uv)
    s.close()
    # a coefficient change on the surface invalidates an existing handle
    s3 = pm.Surface.from_fixture(ctx, os_.surface)
    s3.set_coeff(co.a, co.grad_a)
    b3 = pm.NeumannBVP(s3, os_.curves, edge_a(os_), edge_a(os_, True), patch, uv)
    b3.apply(np.ones(s3.N), np.ones(b3.Me))
    s3.set_coeff(2.0 * co.a, 2.0 * co.grad_a)
    with pytest.raises(pm.PmError):
        b3.apply(np.ones(s3.N), np.ones(b3.Me))
    b3.close()
    s3.close()
    # a variable coefficient is refused for Dirichlet
    import paper_2401_12501_gb300 as pm2
    s2 = pm2.Surface.from_fixture(ctx, os_.surface)
    s2.set_coeff(co.a, co.grad_a)
    with pytest.raises(pm2.PmError):
        pm2.BoundaryValueProblem(s2, os_.curves, edge_a(os_), edge_a(os_, True), patch, uv,
                                 kind="dirichlet")
    s2.close()


@pytest.fixture(scope="module")
def dirichlet_fine(ctx):
    from oracle.bvp import DirichletBVP
    os_ = torus_band(2, 4, 8, 32, 32)
    s, b, co = device_bvp(ctx, os_, "dirichlet")
    ora = DirichletBVP(os_, co, np.ones(os_.M), np.ones(sum(c.F * c.M for c in os_.curves)),
                       processes=oracle_processes())
    yield os_, s, b, co, ora
    b.close()
    s.close()


def test_dirichlet_operator_matches_oracle(dirichlet_fine):
    os_, s, b, co, ora = dirichlet_fine
    rng = np.random.default_rng(43)
    sigma = rng.standard_normal(s.N) + 1.0
    mu = rng.standard_normal(b.Me)
    ys, ye = b.apply(sigma, mu)
    rs, re = ora.apply(sigma, mu)
    assert np.abs(ys - rs).max() <= 1e-10 * np.abs(rs).max()
    assert np.abs(ye - re).max() <= 1e-10 * np.abs(re).max()


def test_dirichlet_solve_matches_oracle_and_exact_solution(dirichlet_fine):
    os_, s, b, co, ora = dirichlet_fine
    f, fg, v = newtonian_dirichlet(os_)
    u, info, _, _ = b.solve(f, fg, tol=1e-13)
    _, _, u_ref = ora.solve(f, fg)
    w = os_.surface.weights
    rel = lambda p, q: float(np.sqrt(np.dot(w, (p - q) ** 2) / np.dot(w, q * q)))   # noqa: E731
    assert rel(u, u_ref) < 1e-9
    assert rel(u, v) < 1e-7 and abs(rel(u, v) - rel(u_ref, v)) < 1e-9


def test_dirichlet_refined_band_converges(ctx):
    os_ = torus_band(4, 8, 8, 64, 32)
    s, b, co = device_bvp(ctx, os_, "dirichlet")
    f, fg, v = newtonian_dirichlet(os_)
    u, info, _, _ = b.solve(f, fg, tol=1e-13)
    w = os_.surface.weights
    err = float(np.sqrt(np.dot(w, (u - v) ** 2) / np.dot(w, v * v)))
    assert err < 3e-8, err
    b.close()
    s.close()
