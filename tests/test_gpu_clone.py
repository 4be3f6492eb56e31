"""pm_surface_clone: a second operator on the same geometry shares the
near-field quadrature and must act exactly like a surface built from scratch
with the same coefficient, also after the original is destroyed."""

import numpy as np
import pytest

from workloads import make_workload, smooth_random_coefficient

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


def test_clone_matches_a_fresh_surface(ctx):
    import paper_2401_12501_gb300 as pm
    wl = make_workload("ellipsoid_2400")
    s0 = pm.Surface.from_fixture(ctx, wl.surface)
    s0.set_coeff(wl.coeff.a, wl.coeff.grad_a)
    co = smooth_random_coefficient(wl.surface, 3)
    c = s0.clone()
    c.set_coeff(co.a, co.grad_a)
    fresh = pm.Surface.from_fixture(ctx, wl.surface)
    fresh.set_coeff(co.a, co.grad_a)
    assert c.info() == fresh.info()
    sigma = np.random.default_rng(8).standard_normal(wl.N)
    before = s0.apply_R(sigma, "fp64")
    for prec in ("fp64", "ff", "fp32", "fmm"):
        assert np.array_equal(c.apply_R(sigma, prec), fresh.apply_R(sigma, prec)), prec
        assert np.array_equal(c.apply_K(sigma, prec), fresh.apply_K(sigma, prec)), prec
    assert np.array_equal(s0.apply_R(sigma, "fp64"), before)      # the original keeps its coefficient
    assert not np.allclose(before, c.apply_R(sigma, "fp64"))      # and differs from the clone's
    s0.close()                                                    # the clone holds the shared buffers
    f = wl.f - np.dot(wl.surface.weights, wl.f) / wl.surface.weights.sum()
    u1, i1 = c.solve(f, tol=1e-10)
    u2, i2 = fresh.solve(f, tol=1e-10)
    assert i1[0].iterations == i2[0].iterations
    assert np.array_equal(u1, u2)
    F = np.stack([f, np.roll(f, 17) - np.dot(wl.surface.weights, np.roll(f, 17)) /
                  wl.surface.weights.sum()])
    U1, _ = c.solve(F, tol=1e-10)                                 # batched lockstep solve
    U2, _ = fresh.solve(F, tol=1e-10)
    assert np.array_equal(U1, U2)
    c2 = c.clone()                                                # a clone of a clone
    c2.set_coeff(co.a, co.grad_a)
    assert np.array_equal(c2.apply_R(sigma, "ff"), fresh.apply_R(sigma, "ff"))
    c.close()
    assert np.array_equal(c2.apply_R(sigma, "fp64"), fresh.apply_R(sigma, "fp64"))
    c2.close()
    fresh.close()
