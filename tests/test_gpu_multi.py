"""Several operators solved in one lockstep batch (pm_solve_multi): instances of
uneven size (different surfaces and node counts) and clones with different
coefficients, every right-hand side in the same float32 apply launches and each
GMRES cycle one CUDA graph.  Every column must equal the same system solved alone
(pm_solve) within 1e-9, whether solved with float-float refinement or on the float32
operator itself; repeated calls replay the cached graphs and give identical results."""

import numpy as np
import pytest

from workloads import make_workload

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


def rel(a, b, w):
    return float(np.sqrt(np.dot(w, (a - b) ** 2) / np.dot(w, b ** 2)))


def rhs_set(wl, k, seed):
    rng = np.random.default_rng(seed)
    w = wl.surface.weights
    F = np.stack([np.roll(wl.f, int(rng.integers(0, wl.N))) * rng.uniform(0.5, 2.0)
                  for _ in range(k)])
    return F - (F @ w)[:, None] / w.sum()


def _surface(ctx, wl, coeff=None, opts=None):
    import paper_2401_12501_gb300 as pm
    s = pm.Surface.from_fixture(ctx, wl.surface, opts)
    co = wl.coeff if coeff is None else coeff
    s.set_coeff(co.a, co.grad_a)
    return s


def test_uneven_instances_match_solo_solves(ctx):
    import paper_2401_12501_gb300 as pm
    names = [("ellipsoid_9600", 2), ("star_small", 3), ("sphere_1536", 1), ("torus_6144", 2)]
    wls = [make_workload(n) for n, _ in names]
    surfs = [_surface(ctx, wl) for wl in wls]
    F = [rhs_set(wl, k, 3 + i) for i, (wl, (_, k)) in enumerate(zip(wls, names))]
    try:
        U, infos = pm.solve_multi(surfs, F, tol=1e-10)
        U2, _ = pm.solve_multi(surfs, F, tol=1e-10)            # graph replay
        for wl, s, f, u, u2, inf in zip(wls, surfs, F, U, U2, infos):
            assert u.shape == f.shape and np.array_equal(u, u2)
            for r in range(f.shape[0]):
                alone, _ = s.solve(f[r], tol=1e-10, prec="fp32")
                assert inf[r].residual <= 1e-10
                assert rel(u[r], alone, wl.surface.weights) < 1e-9
    finally:
        for s in surfs:
            s.close()


def test_coefficient_clones_and_operator_precision(ctx):
    """Four operators on one geometry (clones, different coefficient fields), four
    right-hand sides each; then the same with residuals on the float32 operator."""
    import paper_2401_12501_gb300 as pm
    from workloads import smooth_random_coefficient
    wl = make_workload("star_small")
    for op_prec in (False, True):
        o = pm.default_opts()
        if op_prec:
            o.residual_prec = pm.PM_PREC_FP32
        base = _surface(ctx, wl, smooth_random_coefficient(wl.surface, 0), o)
        ops = [base] + [base.clone() for _ in range(3)]
        for k in range(1, 4):
            co = smooth_random_coefficient(wl.surface, k)
            ops[k].set_coeff(co.a, co.grad_a)
        F = [rhs_set(wl, 4, 10 + k) for k in range(4)]
        try:
            U, infos = pm.solve_multi(ops, F, tol=1e-9)
            w = wl.surface.weights
            for s, f, u, inf in zip(ops, F, U, infos):
                for r in range(4):
                    alone, _ = s.solve(f[r], tol=1e-9, prec="fp32")
                    assert inf[r].residual <= 1e-9
                    # operator precision: u = K~ sigma comes from two different float32 K
                    # kernels (batched vs single), each within the 2e-6 float32 tolerance
                    assert rel(u[r], alone, w) < (2e-6 if op_prec else 1e-9)
        finally:
            for s in ops:
                s.close()


def test_multi_argument_checks(ctx):
    import paper_2401_12501_gb300 as pm
    wl = make_workload("sphere_384")
    s = _surface(ctx, wl)
    f = rhs_set(wl, 1, 1)
    try:
        with pytest.raises(pm.PmError) as e:
            pm.solve_multi([s, s], [f, f])
        assert e.value.status == 1
        with pytest.raises(pm.PmError) as e:
            pm.solve_multi([s], [f + 1.0])
        assert e.value.status == 6
        u, info = pm.solve_multi([s], [f + 1.0], project_rhs=True, tol=1e-9)
        assert abs(info[0][0].removed_mean - 1.0) < 1e-9 and info[0][0].residual <= 1e-9
    finally:
        s.close()
