"""GPU parity of the operator applies against the float64 oracle (through the C ABI).

Tolerances: float64 applies agree with the oracle to 1e-10 relative (the two
sides use different quadrature rules, each converged to ~1e-13); float32
applies to 2e-6 relative L2 (per-pair float32 rounding, compensated
accumulation), inside the 1e-5 bound stated for float32 applies.
"""

import numpy as np
import pytest

from conftest import oracle_processes
from workloads import make_workload

pytestmark = pytest.mark.gpu

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


_SURF = {}


def gpu_surface(ctx, name):
    import paper_2401_12501_gb300 as pm
    if name not in _SURF:
        wl = make_workload(name)
        s = pm.Surface.from_fixture(ctx, wl.surface)
        s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
        _SURF[name] = (wl, s)
    return _SURF[name]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name", ["sphere_384", "ellipsoid_small"])
def test_near_structure_and_corrections(ctx, name):
    wl, d, nf = oracle(name)
    _, s = gpu_surface(ctx, name)
    rp, bp, cR, cK = s.get_near()
    pp = d.p * d.p
    assert rp[0] == 0 and rp[-1] == len(bp)
    for i in range(d.N):
        gpu_patches = list(bp[rp[i]:rp[i + 1]])
        ora = nf.corr[i]
        assert gpu_patches[0] == i // pp                      # own patch first
        assert sorted(gpu_patches) == sorted(P for P, _, _ in ora)
        sR = max(np.abs(c[1]).max() for c in ora)
        sK = max(np.abs(c[2]).max() for c in ora)
        for P, CR, CK in ora:
            b = rp[i] + gpu_patches.index(P)
            assert np.abs(cR[b] - CR).max() <= 1e-10 * sR, (i, P)
            assert np.abs(cK[b] - CK).max() <= 1e-10 * sK, (i, P)


@pytest.mark.parametrize("name", ["sphere_384", "ellipsoid_small", "wavy_torus_small",
                                  "ellipsoid_paper_small"])
@pytest.mark.parametrize("prec,tol,tol_max", [("fp64", 1e-11, 1e-10), ("fp32", 2e-6, 1e-5)])
def test_full_apply_parity(ctx, name, prec, tol, tol_max):
    """Every row against the oracle: relative L2, and element by element on the scale
    of the largest entry (an error local to a few nodes near patch edges would hide in
    the norm alone)."""
    from oracle.operator import apply_K, apply_R
    wl, d, nf = oracle(name)
    _, s = gpu_surface(ctx, name)
    rng = np.random.default_rng(1)
    sigma = rng.standard_normal(d.N) + 1.0
    for got, want in ((s.apply_R(sigma, prec), apply_R(d, nf, sigma)),
                      (s.apply_K(sigma, prec), apply_K(d, nf, sigma))):
        assert rel(got, want) < tol
        assert np.abs(got - want).max() <= tol_max * np.abs(want).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_smooth_parts(ctx, prec, tol):
    import paper_2401_12501_gb300 as pm
    wl, d, _ = oracle("ellipsoid_small")
    _, s = gpu_surface(ctx, "ellipsoid_small")
    sigma = np.random.default_rng(2).standard_normal(d.N)
    assert rel(s.apply_part(pm.PM_PART_SMOOTH_R, sigma, prec), d.smooth_apply("R", sigma)) < tol
    assert rel(s.apply_part(pm.PM_PART_SMOOTH_K, sigma, prec), d.smooth_apply("K", sigma)) < tol


@pytest.mark.parametrize("name", ["sphere_1536", "ellipsoid_9600", "torus_98304",
                                  "wavy_torus_58752"])
def test_sampled_rows_full_size(ctx, name):
    """Full-size workloads: sampled rows computed one by one by the oracle."""
    from oracle.operator import apply_K, apply_R
    wl = make_workload(name)
    N, pp = wl.N, wl.surface.p ** 2
    rng = np.random.default_rng(3)
    rows = sorted(set([0, pp - 1, N - 1] + list(rng.integers(0, N, 21))))
    _, d, nf = oracle(name, rows)
    _, s = gpu_surface(ctx, name)
    sigma = rng.standard_normal(N) + 1.0
    oR = apply_R(d, nf, sigma, rows)
    oK = apply_K(d, nf, sigma, rows)
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-5)):
        yR = s.apply_R(sigma, prec)[rows]
        yK = s.apply_K(sigma, prec)[rows]
        assert np.abs(yR - oR).max() <= tol * np.abs(oR).max(), (prec, yR, oR)
        assert np.abs(yK - oK).max() <= tol * np.abs(oK).max(), (prec, yK, oK)


def test_sphere_remainder_closed_form(ctx):
    """Unit sphere, a = 1: R~ sigma = -(1/4 pi) sum_j w_j sigma_j at every node."""
    wl, s = gpu_surface(ctx, "sphere_1536")
    sigma = np.random.default_rng(4).standard_normal(wl.N) + 0.5
    want = -np.dot(wl.surface.weights, sigma) / (4 * np.pi)
    assert np.abs(s.apply_R(sigma, "fp64") - want).max() < 1e-7 * abs(want)
    assert np.abs(s.apply_R(sigma, "fp32") - want).max() < 1e-5 * abs(want)


def test_multi_rhs_and_device_pointers(ctx):
    import torch
    wl, s = gpu_surface(ctx, "ellipsoid_small")
    sig = np.random.default_rng(5).standard_normal((3, wl.N))
    # several right-hand sides go through the batched kernels, which sum in a
    # different order from the one-at-a-time path: equal to working precision
    for prec, tol in (("fp32", 2e-6), ("fp64", 1e-13), ("ff", 5e-13)):
        host = s.apply_R(sig, prec)
        dev = s.apply_R(torch.from_numpy(sig).cuda(), prec).cpu().numpy()
        single = np.stack([s.apply_R(sig[r], prec) for r in range(3)])
        assert np.array_equal(host, dev)          # deterministic kernels
        assert np.abs(host - single).max() <= tol * np.abs(single).max(), prec


def test_invalid_inputs(ctx):
    import paper_2401_12501_gb300 as pm
    wl = make_workload("sphere_small")
    sf = wl.surface
    bad_w = sf.weights.copy()
    bad_w[5] *= 1.01
    with pytest.raises(pm.PmError) as e:
        pm.Surface(ctx, sf.npatch, sf.p, sf.nodes, sf.normals, sf.tangents, sf.curvature, bad_w)
    assert e.value.status == 1
    nodes = sf.nodes.copy()
    nodes[3, 1] = np.nan
    with pytest.raises(pm.PmError) as e:
        pm.Surface(ctx, sf.npatch, sf.p, nodes, sf.normals, sf.tangents, sf.curvature, sf.weights)
    assert e.value.status == 1
    s = pm.Surface.from_fixture(ctx, sf)
    with pytest.raises(pm.PmError) as e:
        s.apply_R(np.ones(sf.N))
    assert e.value.status == 9                    # PM_ERR_NO_COEFF
    with pytest.raises(pm.PmError) as e:
        s.set_coeff(-np.ones(sf.N))
    assert e.value.status == 1
    s.close()


def test_spectral_gradient_matches_closed_form(ctx):
    """grad_a = NULL: the library differentiates the interpolant of a (eq. gradg)."""
    import paper_2401_12501_gb300 as pm
    wl = make_workload("ellipsoid_9600")
    s = pm.Surface.from_fixture(ctx, wl.surface)
    s.set_coeff(wl.coeff.a)          # spectral gradient
    s2 = gpu_surface(ctx, "ellipsoid_9600")[1]
    sigma = np.random.default_rng(6).standard_normal(wl.N)
    a = s.apply_R(sigma, "fp64")
    b = s2.apply_R(sigma, "fp64")
    assert rel(a, b) < 1e-5
    s.close()


@pytest.mark.parametrize("name", ["ellipsoid_small", "sphere_384"])
def test_float_float_apply_parity(ctx, name):
    """Float-float smooth sums + float64 near field match the float64 oracle like the
    float64 path does (the remaining difference is the two sides' quadrature rules),
    and agree with the float64 path itself to 1e-13."""
    from oracle.operator import apply_K, apply_R
    wl, d, nf = oracle(name)
    _, s = gpu_surface(ctx, name)
    sigma = np.random.default_rng(8).standard_normal(d.N) + 1.0
    assert rel(s.apply_R(sigma, "ff"), apply_R(d, nf, sigma)) < 1e-11
    assert rel(s.apply_K(sigma, "ff"), apply_K(d, nf, sigma)) < 1e-11
    assert rel(s.apply_R(sigma, "ff"), s.apply_R(sigma, "fp64")) < 1e-13
    assert rel(s.apply_K(sigma, "ff"), s.apply_K(sigma, "fp64")) < 1e-13


def test_float_float_full_size_rows(ctx):
    from oracle.operator import apply_K, apply_R
    name = "ellipsoid_9600"
    wl = make_workload(name)
    rng = np.random.default_rng(9)
    rows = sorted(set([0, wl.N - 1] + [int(i) for i in rng.integers(0, wl.N, 10)]))
    _, d, nf = oracle(name, rows)
    _, s = gpu_surface(ctx, name)
    sigma = rng.standard_normal(wl.N) + 1.0
    oR = apply_R(d, nf, sigma, rows)
    oK = apply_K(d, nf, sigma, rows)
    assert np.abs(s.apply_R(sigma, "ff")[rows] - oR).max() < 1e-10 * np.abs(oR).max()
    assert np.abs(s.apply_K(sigma, "ff")[rows] - oK).max() < 1e-10 * np.abs(oK).max()


def test_float_float_logarithm(ctx):
    """Tang's table-driven float-float log against the float64 logarithm."""
    _, s = gpu_surface(ctx, "sphere_384")
    rng = np.random.default_rng(10)
    x = np.concatenate([10.0 ** rng.uniform(-12, 6, 20000), 1.0 + rng.uniform(-1e-3, 1e-3, 2000),
                        [1.0, 2.0, 0.5, 1.0 + 2.0 ** -23, 1.9999999]])
    xh = x.astype(np.float32)
    xl = (x - xh.astype(np.float64)).astype(np.float32)
    xx = xh.astype(np.float64) + xl.astype(np.float64)
    got = s.selftest_fflog(xh, xl)
    ref = np.log(xx)
    err = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() < 3e-14, err.max()


@pytest.mark.parametrize("name", ["ellipsoid_small", "ellipsoid_2400", "torus_6144"])
def test_symmetric_tile_pair_sums_match_one_sided(ctx, name):
    """Tile-pair sums (each unordered pair once, row and column sums) against the
    one-sided sums of the same surface: float32 remainder to float32 rounding,
    float-float remainder and parametrix to float-float rounding.  864, 2,400 and
    6,144 nodes are 6.75, 18.75 and 48 tiles of 128 (ragged and exact tails)."""
    import paper_2401_12501_gb300 as pm
    wl = make_workload(name)
    surf = {}
    for sym in (0, 1):
        o = pm.default_opts()
        o.direct_symmetric = sym
        s = pm.Surface.from_fixture(ctx, wl.surface, o)
        s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
        surf[sym] = s
    sig = np.random.default_rng(21).standard_normal(wl.N)
    for op, prec, tol in (("R", "fp32", 2e-6), ("R", "ff", 5e-13), ("K", "ff", 5e-13)):
        f0 = surf[0].apply_R if op == "R" else surf[0].apply_K
        f1 = surf[1].apply_R if op == "R" else surf[1].apply_K
        y0, y1 = f0(sig, prec), f1(sig, prec)
        assert np.all(np.isfinite(y1))
        assert np.abs(y1 - y0).max() <= tol * np.abs(y0).max(), (op, prec)
        assert np.array_equal(y1, f1(sig, prec))            # fixed-order reductions
    for s in surf.values():
        s.close()


@pytest.mark.parametrize("p", [2, 3, 5, 7, 11])
def test_patch_orders_against_oracle_rows(ctx, p):
    """Every supported patch order class: p = 3 (smallest tables), odd p with padded
    float32 rows (p^2 = 25, 49 not a multiple of 4), p = 11 (the largest the library
    accepts).  Ellipsoid (1, 1.5, 2), 24 patches, variable coefficient; the float64,
    float32 and float-float applies against the oracle on sampled rows."""
    import paper_2401_12501_gb300 as pm
    from oracle.operator import Discretization, NearField, apply_K, apply_R
    from workloads.coefficients import ellipsoid_coefficient
    from workloads.surfaces import cubed_sphere
    surf = cubed_sphere(2, p, axes=(1.0, 1.5, 2.0))
    co = ellipsoid_coefficient(surf)
    s = pm.Surface.from_fixture(ctx, surf)
    s.set_coeff(co.a, co.grad_a)
    rng = np.random.default_rng(30 + p)
    rows = sorted(set([0, surf.N - 1, p * p - 1, p * p] + [int(i) for i in rng.integers(0, surf.N, 8)]))
    d = Discretization(surf.nodes, surf.normals, surf.tangents, surf.curvature, surf.weights,
                       co.a, co.grad_a, surf.npatch, surf.p)
    nf = NearField(d, rows=rows, processes=oracle_processes())
    sigma = rng.standard_normal(surf.N) + 1.0
    oR, oK = apply_R(d, nf, sigma, rows), apply_K(d, nf, sigma, rows)
    for prec, tol in (("fp64", 1e-10), ("ff", 1e-10), ("fp32", 1e-5)):
        yR, yK = s.apply_R(sigma, prec)[rows], s.apply_K(sigma, prec)[rows]
        assert np.abs(yR - oR).max() <= tol * np.abs(oR).max(), (p, prec)
        assert np.abs(yK - oK).max() <= tol * np.abs(oK).max(), (p, prec)
    s.close()


@pytest.mark.parametrize("name", ["ellipsoid_small", "wavy_torus_small"])
def test_stored_oracle_values(ctx, name):
    """The CUDA path against the oracle values stored in tests/golden/ (written by
    tests/golden/make_golden.py from the oracle alone), at the stored rows."""
    from conftest import golden
    case = golden("oracle_applies.json")["cases"][name]
    _, s = gpu_surface(ctx, name)
    sigma = np.random.default_rng(2024).standard_normal(case["N"]) + 1.0
    rows = case["rows"]
    R, K = np.array(case["R"]), np.array(case["K"])
    for prec, tol in (("fp64", 1e-10), ("ff", 1e-10), ("fp32", 1e-5)):
        assert np.abs(s.apply_R(sigma, prec)[rows] - R).max() <= tol * np.abs(R).max(), prec
        assert np.abs(s.apply_K(sigma, prec)[rows] - K).max() <= tol * np.abs(K).max(), prec
