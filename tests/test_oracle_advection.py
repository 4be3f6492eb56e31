"""Pins of the oracle's advection term (b != 0; Sec. 4.3, eq. adv_remainder, eq. IE_adv).

* Thm. advectionparametrix off the diagonal: div_G(a grad_G K) + b . grad_G K
  + c K = R_b, by finite differences of K in ambient space on a torus with
  variable a, a tangential b, and c = 0 or a variable complex c.
* For tangential b the advection term b . grad_G K = G'(r) b . r^ has the form
  of the grad_G a term of eq. explicit_remainder, so R_b is R with grad_G a(x)
  replaced by grad_G a(x) + b(x) (the identity that lets the library's
  coefficient-gradient input carry b).
* Manufactured solutions (Sec. 7.2 procedure with the advection term):
  v = -1/|x - x0| on a 216-node ellipsoid with variable a,
  f = div_G(a grad_G v) + b . grad_G v, for a divergence-free b = n x grad_G psi
  (mean-zero f, the solvability condition of c = 0 is unchanged) and for a
  gradient field b = grad_G phi (f has a non-zero mean; the range of the
  operator is no longer the mean-zero functions).  With the rank-one term
  (sum w sigma) 1 the projection of f is harmless: 1 is not in the range of
  I + R_b, so A sigma = f - m 1 forces (sum w sigma) = -m and (I + R_b) sigma = f,
  and u is the same with or without projecting f (discretely up to the
  discretisation error: measured 8.6e-6 against a solution error of 6.3e-4).
"""

import numpy as np
import pytest

from conftest import oracle_processes
from oracle.kernels import (advection_term, parametrix, parametrix_c, remainder,
                            remainder_c)
from oracle.operator import Discretization, NearField
from oracle.solve import relative_l2, solve
from test_oracle_kernels import _torus_point
from workloads import cubed_sphere


def _a(x):
    return 1.0 + 0.3 * np.sin(x[0]) * np.cos(2 * x[1]) + 0.1 * x[2]


def _grad_a(x):
    return np.array([0.3 * np.cos(x[0]) * np.cos(2 * x[1]),
                     -0.6 * np.sin(x[0]) * np.sin(2 * x[1]), 0.1])


def _b_ambient(x):
    return np.array([np.cos(x[1]), 0.5 * x[2], np.sin(x[0]) - 0.3])


@pytest.mark.parametrize("with_c", [False, True])
def test_advection_remainder_equals_surface_operator_of_parametrix(with_c):
    rng = np.random.default_rng(21)

    def c_fn(x):
        return 2.0 * x[0] + 1.5j * np.cos(x[1]) - 1.0

    checked = 0
    while checked < 15:
        th, ph, th2, ph2 = rng.uniform(0, 2 * np.pi, 4)
        x, n, H, _, _, _ = _torus_point(2.0, 0.7, th, ph)
        y = _torus_point(2.0, 0.7, th2, ph2)[0]
        if np.linalg.norm(x - y) < 0.3 or (with_c and abs(c_fn(y)) < 0.2):
            continue
        ay = np.array([_a(y)])
        cy = np.array([c_fn(y)]) if with_c else None

        def K(z):
            if with_c:
                return parametrix_c(z, y[None, :], ay, cy)[0]
            return parametrix(z, y[None, :], ay)[0]

        h = 1e-3
        E = np.eye(3)
        grad = np.array([(K(x + h * e) - K(x - h * e)) / (2 * h) for e in E])
        lap = sum((K(x + h * e) - 2 * K(x) + K(x - h * e)) / h ** 2 for e in E)
        dnn = (K(x + h * n) - 2 * K(x) + K(x - h * n)) / h ** 2
        gG = _grad_a(x) - n * (_grad_a(x) @ n)
        b = _b_ambient(x)
        b = b - n * (b @ n)                              # tangential field
        ax = _a(x)
        fd = gG @ grad + ax * (lap - dnn) - 2 * ax * H * (grad @ n) + b @ (grad - n * (grad @ n))
        if with_c:
            fd = fd + c_fn(x) * K(x)
            val = remainder_c(x, n, H, ax, gG, c_fn(x), y[None, :], ay, cy)[0]
        else:
            val = remainder(x, n, H, ax, gG, y[None, :], ay)[0]
        val = val + advection_term(x, n, b, y[None, :], ay, cy)[0]
        assert abs(fd - val) < 1e-5 * max(1.0, abs(val)), (fd, val)
        checked += 1


def test_advection_is_a_shift_of_the_coefficient_gradient():
    rng = np.random.default_rng(5)
    for _ in range(10):
        th, ph = rng.uniform(0, 2 * np.pi, 2)
        x, n, H, _, _, _ = _torus_point(2.0, 0.7, th, ph)
        y = np.array([_torus_point(2.0, 0.7, *rng.uniform(0, 2 * np.pi, 2))[0] for _ in range(5)])
        ay = 1.0 + rng.random(5)
        cy = rng.standard_normal(5) + 1j * rng.standard_normal(5)
        gG = _grad_a(x) - n * (_grad_a(x) @ n)
        b = _b_ambient(x)
        b = b - n * (b @ n)
        ax = _a(x)
        lhs = remainder(x, n, H, ax, gG, y, ay) + advection_term(x, n, b, y, ay)
        rhs = remainder(x, n, H, ax, gG + b, y, ay)
        assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()
        lhs = remainder_c(x, n, H, ax, gG, 0.7, y, ay, cy) + advection_term(x, n, b, y, ay, cy)
        rhs = remainder_c(x, n, H, ax, gG + b, 0.7, y, ay, cy)
        assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()


def _ellipsoid_problem(kind):
    """216-node ellipsoid (1, 1.5, 2), a of the ellipsoid workloads, b of the given kind."""
    from workloads.coefficients import ellipsoid_coefficient
    s = cubed_sphere(1, 6, axes=(1.0, 1.5, 2.0))
    co = ellipsoid_coefficient(s)
    x, n = s.nodes, s.normals
    if kind == "div_free":           # b = n x grad_G psi, psi = x y + z / 2
        gpsi = np.stack([x[:, 1], x[:, 0], np.full(len(x), 0.5)], 1)
        gpsi -= n * np.sum(gpsi * n, 1, keepdims=True)
        b = np.cross(n, gpsi)
    else:                            # b = grad_G phi, phi = x + y z
        gphi = np.stack([np.ones(len(x)), x[:, 2], x[:, 1]], 1)
        b = gphi - n * np.sum(gphi * n, 1, keepdims=True)
    x0 = np.array([-3.0, -3.0, 4.0])
    dx = x - x0
    rho = np.linalg.norm(dx, axis=1)
    v = -1.0 / rho
    grad = dx / rho[:, None] ** 3
    dn = np.sum(grad * n, 1)
    dnn = 1.0 / rho ** 3 - 3 * np.sum(dx * n, 1) ** 2 / rho ** 5
    grad_G = grad - n * dn[:, None]
    lap_G = -2 * s.curvature * dn - dnn
    f = np.sum(co.grad_a * grad_G, 1) + co.a * lap_G + np.sum(b * grad_G, 1)
    d = Discretization(s.nodes, s.normals, s.tangents, s.curvature, s.weights,
                       co.a, co.grad_a, s.npatch, s.p, b=b)
    return d, f, v


@pytest.mark.parametrize("kind", ["div_free", "gradient"])
def test_manufactured_solution_with_advection(kind):
    d, f, v = _ellipsoid_problem(kind)
    w = d.w
    mean_f = abs(np.dot(w, f)) / np.sqrt(np.dot(w, f * f) * w.sum())
    if kind == "div_free":
        assert mean_f < 1e-4                 # int b . grad v = -int v div b = 0
    else:
        assert mean_f > 1e-2                 # range is not the mean-zero functions
    nf = NearField(d, processes=oracle_processes())
    u = solve(d, nf, f, project_rhs=(kind == "div_free"))
    uex = v - np.dot(w, v) / w.sum()
    assert relative_l2(u, uex, w) < 1.5e-3    # measured 5.6e-4 / 6.3e-4; without b 0.29 / 1.03
    if kind == "gradient":
        up = solve(d, nf, f, project_rhs=True)
        assert relative_l2(up, u, w) < 1e-4


def test_discrete_advection_equals_shifted_gradient():
    """The identity holds for the discrete operators too: R~_b built from the literal
    advection term equals R~ built with grad_G a + b (sampled rows, both quadratures),
    and K~ is unchanged."""
    from oracle.operator import apply_K, apply_R
    d, _, _ = _ellipsoid_problem("div_free")
    shifted = Discretization(d.x, d.n, None, d.H, d.w, d.a, d.g + d.b, d.npatch, d.p,
                             jac=np.concatenate([pt.J.ravel() for pt in d.patches]))
    rows = [0, 37, 100, 171, 215]
    nb = NearField(d, rows=rows, processes=1)
    ns = NearField(shifted, rows=rows, processes=1)
    sigma = np.random.default_rng(4).standard_normal(d.N) + 1.0
    ref = apply_R(shifted, ns, sigma, rows)
    assert np.abs(apply_R(d, nb, sigma, rows) - ref).max() < 1e-12 * np.abs(ref).max()
    refK = apply_K(shifted, ns, sigma, rows)
    assert np.abs(apply_K(d, nb, sigma, rows) - refK).max() < 1e-14 * np.abs(refK).max()
