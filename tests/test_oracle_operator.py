"""Operator- and solve-level pins of the oracle.

* Unit sphere, a = 1 (sphere_384):
  - every near-field correction vanishes up to interpolation error, since
    R_LB = -1/(4 pi) and the Gauss rule integrates l_k J~ exactly;
  - (I + R~) 1 = 0: the constant is the null vector (Sec. 3);
  - K~[Y_l^m] = -Y_l^m / (l (l+1)) and K~[1] = 2 ln 2 - 1 (Funk-Hecke
    applied to eq. parametrixLB);
  - the solve of Y_3^2 returns -Y_3^2/12 (Sec. 7.1: eigenvalues -l(l+1)).
* Any surface, variable a (ellipsoid_small): the range of I + R is mean
  zero (Sec. 3: I + R = div(a grad) K), and a manufactured solution
  (Sec. 7.2 procedure, variable-a right-hand side grad a . grad v + a Lap_G v)
  is recovered.
* Dilation of the near-field weights (Sec. 3 conjecture, item 3).
* Null space (Sec. 3): on the sphere I + R~ has exactly one near-zero singular
  value and the rank-one term removes it; on a torus with a = 1 the null vector
  is alpha - rho (rho: distance to the rotation axis), so (I + R~) 1 and
  (I + R~) rho are parallel, with alpha not the mean of rho.
"""

import numpy as np
import pytest

from conftest import golden, oracle_processes
from oracle.operator import (Discretization, NearField, apply_K, apply_R,
                             second_kind_matrix)
from oracle.solve import gmres, relative_l2, solve
from workloads import make_workload, real_sph_harm


@pytest.fixture(scope="module")
def sphere():
    wl = make_workload("sphere_384")
    d = Discretization.from_workload(wl)
    return wl, d, NearField(d, processes=oracle_processes())


@pytest.fixture(scope="module")
def ellipsoid():
    wl = make_workload("ellipsoid_small")
    d = Discretization.from_workload(wl)
    return wl, d, NearField(d, processes=oracle_processes())


def test_sphere_corrections_vanish(sphere):
    """C_ik = 0 for k != i; C_ii = W_ii = -w_i/(4 pi) (the smooth sum skips j = i)."""
    _, d, nf = sphere
    pp = d.p * d.p
    worst = 0.0
    for i, row in nf.corr.items():
        for P, CR, _ in row:
            c = CR.copy()
            if P == i // pp:
                c[i - P * pp] += d.w[i] / (4 * np.pi)
            worst = max(worst, np.abs(c).max())
    assert worst < 5e-7


def test_sphere_null_vector(sphere):
    _, d, nf = sphere
    one = np.ones(d.N)
    assert np.abs(one + apply_R(d, nf, one)).max() < 2e-6


@pytest.mark.parametrize("l,m", [(1, 0), (2, -1), (3, 2), (4, 3)])
def test_sphere_funk_hecke(sphere, l, m):
    _, d, nf = sphere
    Y = real_sph_harm(l, m, d.x)
    ev = golden("closed_forms.json")["sphere_parametrix_eigenvalues"]
    lam = ev["value"][ev["l"].index(l)]                     # -1/(l(l+1))
    assert relative_l2(apply_K(d, nf, Y), lam * Y, d.w) < 2e-5


def test_sphere_parametrix_of_constant(sphere):
    _, d, nf = sphere
    K1 = apply_K(d, nf, np.ones(d.N))
    c = golden("closed_forms.json")["sphere_parametrix_constant"]["value"]   # 2 ln 2 - 1
    assert np.abs(K1 - c).max() < 1e-6


def test_sphere_solve_eigenfunction(sphere):
    wl, d, nf = sphere
    u = solve(d, nf, wl.f)
    assert relative_l2(u, -wl.f / 12, d.w) < 5e-6
    u2 = solve(d, nf, wl.f, method="gmres", tol=1e-13)
    assert relative_l2(u2, u, d.w) < 1e-11


def test_range_is_mean_zero(ellipsoid):
    wl, d, nf = ellipsoid
    rng = np.random.default_rng(5)
    for _ in range(3):
        s = rng.standard_normal(d.N) + 1.0
        y = s + apply_R(d, nf, s)
        assert abs(np.dot(d.w, y)) < 1e-4 * np.sqrt(np.dot(d.w, s * s))


def test_manufactured_solution_variable_a(ellipsoid):
    wl, d, nf = ellipsoid
    x0 = np.array([-3.0, -3.0, 4.0])
    dx = d.x - x0
    rho = np.linalg.norm(dx, axis=1)
    v = -1.0 / rho
    grad = dx / rho[:, None] ** 3
    n = d.n
    dn = np.sum(grad * n, 1)
    # Hess v = I/rho^3 - 3 dx dx^T / rho^5, so n^T Hess n:
    dnn = 1.0 / rho ** 3 - 3 * np.sum(dx * n, 1) ** 2 / rho ** 5
    lap_G = 0.0 - 2 * d.H * dn - dnn          # eq. LB_rest_p with Lap v = 0
    grad_G = grad - n * dn[:, None]
    f = np.sum(d.g * grad_G, 1) + d.a * lap_G   # div(a grad_G v) = grad a.grad_G v + a Lap_G v
    u = solve(d, nf, f)
    uex = v - np.dot(d.w, v) / d.w.sum()
    assert relative_l2(u, uex, d.w) < 2e-3


def test_near_weights_dilation():
    wl = make_workload("ellipsoid_small")
    d1 = Discretization.from_workload(wl)
    s2 = wl.surface.scaled(3.0)
    d2 = Discretization(s2.nodes, s2.normals, s2.tangents, s2.curvature, s2.weights,
                        wl.coeff.a, wl.coeff.grad_a / 3.0, s2.npatch, s2.p)
    for i in [0, 100, 500]:
        r1, r2 = d1.row_weights(i), d2.row_weights(i)
        assert [P for P, _, _ in r1] == [P for P, _, _ in r2]
        for (P, WR1, WK1), (_, WR2, WK2) in zip(r1, r2):
            assert np.abs(WR1 - WR2).max() < 1e-12 * np.abs(WR1).max()
            # K: W2 = 9 W1 + log(3)/(2 pi) * int l_k J~ (= 9 * omega_k J_k)
            pp = 36
            w = wl.surface.weights[P * pp:(P + 1) * pp]
            assert np.abs(WK2 - 9 * WK1 - np.log(3.0) / (2 * np.pi) * 9 * w).max() < 5e-12 * np.abs(WK2).max()


def test_gmres_matches_dense_solve():
    rng = np.random.default_rng(0)
    A = np.eye(60) + 0.3 * rng.standard_normal((60, 60)) / np.sqrt(60)
    b = rng.standard_normal(60)
    x, it, rr = gmres(lambda v: A @ v, b, tol=1e-13, restart=10)
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-11


def test_sphere_single_null_singular_value(sphere):
    _, d, nf = sphere
    A = second_kind_matrix(d, nf)
    sv0 = np.linalg.svd(A - np.outer(np.ones(d.N), d.w), compute_uv=False)
    assert sv0[-1] < 1e-6 and sv0[-2] > 0.5                  # one null direction, I + R~
    assert np.linalg.svd(A, compute_uv=False)[-1] > 0.5       # removed by the rank-one term


def test_torus_null_vector_alpha_minus_rho():
    from workloads.surfaces import torus
    s = torus(8, 4, 6)
    N = s.N
    d = Discretization(s.nodes, s.normals, s.tangents, s.curvature, s.weights,
                       np.ones(N), np.zeros((N, 3)), s.npatch, s.p, near_tol=1e-10)
    nf = NearField(d, processes=oracle_processes())
    one = np.ones(N)
    rho = np.hypot(s.nodes[:, 0], s.nodes[:, 1])
    y1 = one + apply_R(d, nf, one)
    yr = rho + apply_R(d, nf, rho)
    alpha = np.dot(y1, yr) / np.dot(y1, y1)
    # parallel to discretisation accuracy on 8 x 4 patches of 6 x 6 nodes (0.96 %)
    assert np.linalg.norm(yr - alpha * y1) < 0.03 * np.linalg.norm(yr)
    assert np.linalg.norm(y1) > 0.5 * np.sqrt(N)               # 1 itself is not in the null space
    assert abs(alpha - np.dot(s.weights, rho) / s.weights.sum()) > 0.1
