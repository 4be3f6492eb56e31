"""Pins of the oracle's triangle rule (Sec. 6.1: Koornwinder basis, Vioreanu-Rokhlin nodes).

* The collapsed Gauss rule on T0 integrates u^a v^b to the closed form
  a! b! / (a + b + 2)! (the Beta-function integral over the simplex).
* The Koornwinder basis is orthonormal on T0 (against that pinned rule).
* Order p: p (p + 1) / 2 nodes strictly inside T0, invariant as a set under the
  six permutations of the barycentric coordinates (the triangle's symmetries),
  positive weights, every polynomial of degree <= p - 1 integrated exactly, and
  a well-conditioned Koornwinder Vandermonde matrix (Sec. 6.1.2 relies on it),
  for p = 2..8.
* The interpolant c = U sigma of Sec. 6.1.2 reproduces the node values and
  converges spectrally for a smooth function.
* The operators on curved triangles (unit sphere as projected icosahedron
  triangles): R~ 1 = -1, R~ Y = 0, K~ Y = -Y/(l(l+1)) at sampled rows, and a
  variable-coefficient manufactured solve.
"""

from math import factorial

import numpy as np
import pytest

from oracle.triangle import (collapsed_rule, interpolation_matrix, koornwinder,
                             vioreanu_rokhlin)

ORDERS = [2, 3, 4, 5, 6, 7, 8]


def _monomial(a, b):
    return factorial(a) * factorial(b) / factorial(a + b + 2)


def test_collapsed_rule_integrates_monomials():
    u, v, w = collapsed_rule(9)                 # exact to total degree 16
    for a in range(17):
        for b in range(17 - a):
            assert abs(np.sum(w * u ** a * v ** b) - _monomial(a, b)) < 1e-15


@pytest.mark.parametrize("n", [0, 1, 4, 7, 11])
def test_koornwinder_basis_is_orthonormal(n):
    u, v, w = collapsed_rule(n + 3)
    B = koornwinder(n, u, v)
    assert B.shape[0] == (n + 1) * (n + 2) // 2
    G = (B * w) @ B.T
    assert np.abs(G - np.eye(len(G))).max() < 1e-12


@pytest.mark.parametrize("p", ORDERS)
def test_vioreanu_rokhlin_rule(p):
    u, v, w = vioreanu_rokhlin(p)
    assert len(u) == p * (p + 1) // 2
    bary = np.stack([1.0 - u - v, u, v], 1)
    assert bary.min() > 1e-3                                  # strictly inside
    assert w.min() > 0
    for a in range(p):                                        # degree <= p - 1 exactly
        for b in range(p - a):
            assert abs(np.sum(w * u ** a * v ** b) - _monomial(a, b)) < 1e-14
    # the node set is invariant under every permutation of the barycentric coordinates
    key = np.round(bary, 10)
    ref = {tuple(r) for r in key}
    for perm in ([0, 2, 1], [1, 0, 2], [1, 2, 0], [2, 0, 1], [2, 1, 0]):
        assert {tuple(r) for r in key[:, perm]} == ref
    V = koornwinder(p - 1, u, v)
    assert np.linalg.cond(V) < 10.0


def test_interpolation_converges():
    rng = np.random.default_rng(0)
    s = rng.random((200, 2))
    s = np.where(s.sum(1, keepdims=True) > 1, 1 - s, s)        # random points of T0
    f = lambda u, v: np.exp(u + 2 * v) * np.cos(3 * u - v)
    errs = []
    for p in (4, 6, 8):
        u, v, _ = vioreanu_rokhlin(p)
        c = interpolation_matrix(p) @ f(u, v)
        assert np.abs(c @ koornwinder(p - 1, u, v) - f(u, v)).max() < 1e-13   # interpolates
        approx = c @ koornwinder(p - 1, s[:, 0], s[:, 1])
        errs.append(np.abs(approx - f(s[:, 0], s[:, 1])).max())
    # measured 0.29, 0.017, 3.2e-4
    assert errs[0] > 10 * errs[1] > 100 * errs[2] and errs[2] < 1e-3, errs


def test_triangle_operators_on_the_icosphere():
    """The operators on curved triangles (Sec. 6.1 with the rule above): unit sphere
    as 80 projected icosahedron triangles, order 8 (2,880 nodes), a = 1.  The
    smooth weights sum to 4 pi; at sampled rows R~ 1 = -1 (R_LB = -1/(4 pi),
    Sec. 3), R~ Y_l^m = 0 and K~ Y_l^m = -Y_l^m / (l (l+1)) (Funk-Hecke); measured
    <= 4.3e-7 (1.7e-6 at order 6, 8e-8 on 320 triangles)."""
    from oracle.operator import NearField, apply_K, apply_R
    from oracle.triangle_operator import TriDiscretization
    from workloads import real_sph_harm
    from workloads.trisurfaces import icosphere
    M, ymap = icosphere(1)
    d = TriDiscretization(ymap, M, 8, curvature_fn=lambda x: np.ones(len(x)))
    assert d.N == 80 * 36
    assert abs(d.w.sum() / (4 * np.pi) - 1) < 1e-6               # measured 1.0e-7
    assert np.abs(np.sum(d.n * d.x, 1) - 1).max() < 1e-14        # outward unit normals
    rows = np.arange(0, d.N, 240)
    nf = NearField(d, rows=rows)
    assert np.abs(apply_R(d, nf, np.ones(d.N), rows) + 1).max() < 1e-6
    for l, m in [(1, 0), (2, 1), (3, -2), (4, 3)]:
        Y = real_sph_harm(l, m, d.x)
        assert np.abs(apply_K(d, nf, Y, rows) + Y[rows] / (l * (l + 1))).max() < 1e-6, l
        assert np.abs(apply_R(d, nf, Y, rows)).max() < 1e-6, l


def test_triangle_solve_variable_coefficient():
    """The solve on curved triangles with a variable coefficient (Sec. 7.2 procedure):
    a = 1 + 0.5 sin 2x cos 3y on the unit sphere (80 triangles of order 4, 800 nodes),
    v = -1/|x - x0|, f = grad_G a . grad_G v + a Lap_G v; u recovers v - mean(v)
    (measured 3.8e-5; 1.1e-5 at order 5; without the grad_G a term of R the error
    is 0.12).  Every row's near field is built by spawned workers."""
    from conftest import oracle_processes
    from oracle.solve import relative_l2, solve
    from oracle.triangle_operator import TriDiscretization, tri_near_field
    from workloads.trisurfaces import icosphere

    def a_fn(x):
        return 1.0 + 0.5 * np.sin(2 * x[:, 0]) * np.cos(3 * x[:, 1])

    def grad_a_fn(x, n):
        g = np.stack([np.cos(2 * x[:, 0]) * np.cos(3 * x[:, 1]),
                      -1.5 * np.sin(2 * x[:, 0]) * np.sin(3 * x[:, 1]), 0 * x[:, 0]], 1)
        return g - n * np.sum(g * n, 1, keepdims=True)

    M, ymap = icosphere(1)
    d = TriDiscretization(ymap, M, 4, a_fn=a_fn, grad_a_fn=grad_a_fn,
                          curvature_fn=lambda x: np.ones(len(x)))
    nf = tri_near_field(d, processes=oracle_processes())
    x0 = np.array([-3.0, -3.0, 4.0])
    dx = d.x - x0
    rho = np.linalg.norm(dx, axis=1)
    v = -1.0 / rho
    grad = dx / rho[:, None] ** 3
    dn = np.sum(grad * d.n, 1)
    dnn = 1.0 / rho ** 3 - 3 * np.sum(dx * d.n, 1) ** 2 / rho ** 5
    f = np.sum(d.g * (grad - d.n * dn[:, None]), 1) + d.a * (-2 * d.H * dn - dnn)
    u = solve(d, nf, f)
    assert relative_l2(u, v - np.dot(d.w, v) / d.w.sum(), d.w) < 2e-4
