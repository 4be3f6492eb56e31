"""Triangle patches on the device (Sec. 6.1, 6.1.2; pm_surface_create_tri) against the
oracle's node-interpolated triangle operators (oracle/triangle_nodes.py) and closed forms.

* Near structure and every correction block against the oracle at 1e-10 of the
  row's largest entry (icosahedral ellipsoid, variable coefficient, p = 6).
* Full applies, element-wise: float64 at 1e-10, float32 at 1e-5 of the largest entry.
* Unit sphere from 80 triangles (p = 8): R~ 1 = -1, K~ Y_3^2 = -Y_3^2/12, and the
  solve of f = Y_3^2 returns -f/12 (float32 applies, float-float refinement).
* A variable-coefficient solve equals the oracle's LU solve to 1e-8.
* Clones, batched right-hand sides and the FMM run on triangle surfaces unchanged.
"""

import numpy as np
import pytest

from conftest import oracle_processes

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


_CASE = {}


def case(ctx):
    """Ellipsoid (1, 1.5, 2) from the 20 icosahedron triangles, p = 6 (420 nodes),
    a = 1 + 0.5 sin(2x) cos(3y): the library surface and the oracle with all rows."""
    if "e" not in _CASE:
        import paper_2401_12501_gb300 as pm
        from oracle.triangle_nodes import TriNodeDiscretization
        from oracle.triangle_operator import tri_near_field
        from workloads import ellipsoid_coefficient
        from workloads.trisurfaces import tri_ellipsoid
        s = tri_ellipsoid(0, 6, axes=(1.0, 1.5, 2.0))
        co = ellipsoid_coefficient(s)
        S = pm.Surface.from_fixture(ctx, s)
        S.set_coeff(co.a, co.grad_a)
        d = TriNodeDiscretization.from_surface(s, a=co.a, grad_a=co.grad_a)
        nf = tri_near_field(d, processes=oracle_processes())
        _CASE["e"] = (s, co, S, d, nf)
    return _CASE["e"]


def test_triangle_near_structure_and_corrections(ctx):
    s, co, S, d, nf = case(ctx)
    rp, bp, cR, cK = S.get_near()
    nt = d.pp
    assert cR.shape[1] == nt and rp[0] == 0 and rp[-1] == len(bp)
    for i in range(d.N):
        gpu_patches = list(bp[rp[i]:rp[i + 1]])
        ora = nf.corr[i]
        assert gpu_patches[0] == i // nt                       # own patch first
        assert sorted(gpu_patches) == sorted(P for P, _, _ in ora)
        sR = max(np.abs(c[1]).max() for c in ora)
        sK = max(np.abs(c[2]).max() for c in ora)
        for P, CR, CK in ora:
            b = rp[i] + gpu_patches.index(P)
            assert np.abs(cR[b] - CR).max() <= 1e-10 * sR, (i, P, np.abs(cR[b] - CR).max() / sR)
            assert np.abs(cK[b] - CK).max() <= 1e-10 * sK, (i, P, np.abs(cK[b] - CK).max() / sK)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5), ("ff", 1e-10)])
def test_triangle_full_applies(ctx, prec, tol):
    from oracle.operator import apply_K, apply_R
    s, co, S, d, nf = case(ctx)
    sigma = np.random.default_rng(2).standard_normal(d.N) + 1.0
    for got, want in ((S.apply_R(sigma, prec), apply_R(d, nf, sigma)),
                      (S.apply_K(sigma, prec), apply_K(d, nf, sigma))):
        assert np.abs(got - want).max() <= tol * np.abs(want).max(), \
            (prec, np.abs(got - want).max() / np.abs(want).max())


def test_triangle_solve_matches_oracle(ctx):
    from oracle.solve import solve
    from workloads import project_mean_zero, real_sph_harm
    s, co, S, d, nf = case(ctx)
    f = project_mean_zero(real_sph_harm(2, 1, s.nodes) + 0.5 * real_sph_harm(3, -2, s.nodes),
                          s.weights)
    u, info = S.solve(f, tol=1e-12, prec="fp32")
    uo = solve(d, nf, f)
    err = np.sqrt(np.dot(s.weights, (u - uo) ** 2) / np.dot(s.weights, uo ** 2))
    assert info[0].residual <= 1e-12
    assert err < 1e-8, err


def test_triangle_sphere_closed_forms(ctx):
    """80 triangles, p = 8 (2,880 nodes): the unit sphere's identities and the Y_3^2 solve."""
    import paper_2401_12501_gb300 as pm
    from workloads import real_sph_harm
    from workloads.trisurfaces import tri_ellipsoid
    s = tri_ellipsoid(1, 8)
    S = pm.Surface.from_fixture(ctx, s)
    S.set_coeff(np.ones(s.N))
    Y = real_sph_harm(3, 2, s.nodes)
    assert np.abs(S.apply_R(np.ones(s.N), "fp64") + 1.0).max() < 1e-6
    assert np.abs(S.apply_R(Y, "fp64")).max() < 1e-6
    assert np.abs(S.apply_K(Y, "fp64") + Y / 12).max() < 1e-6
    u, info = S.solve(Y, tol=1e-10)
    err = np.sqrt(np.dot(s.weights, (u + Y / 12) ** 2) / np.dot(s.weights, (Y / 12) ** 2))
    assert err < 1e-5, err                  # discretisation error: measured 3.2e-6
    # a clone shares the quadrature; batched right-hand sides run the lockstep solver
    C2 = S.clone()
    C2.set_coeff(np.full(s.N, 2.0))
    U, infos = C2.solve(np.stack([Y, real_sph_harm(1, 0, s.nodes)]), tol=1e-10)
    assert np.abs(U[0] - u / 2).max() < 1e-8 * np.abs(u).max()     # a -> 2a scales u by 1/2
    C2.close()
    S.close()


def test_triangle_fmm(ctx):
    """1,280 triangles, p = 6 (26,880 nodes): the FMM apply against the float-float sum."""
    import paper_2401_12501_gb300 as pm
    from workloads import ellipsoid_coefficient
    from workloads.trisurfaces import tri_ellipsoid
    s = tri_ellipsoid(3, 6, axes=(1.0, 1.5, 2.0))
    co = ellipsoid_coefficient(s)
    S = pm.Surface.from_fixture(ctx, s)
    S.set_coeff(co.a, co.grad_a)
    sigma = np.random.default_rng(3).standard_normal(s.N) + 1.0
    for part in (pm.PM_PART_SMOOTH_R, pm.PM_PART_SMOOTH_K):
        assert rel(S.apply_part(part, sigma, "fmm"), S.apply_part(part, sigma, "ff")) < 1e-5
    S.close()
