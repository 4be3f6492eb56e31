"""Pins of the oracle's edge operators (Sec. 5) on planar curves (flat Gamma, a = 1).

* Unit circle: the single layer of cos(m t) is -rho^m cos(m theta) / (2m) inside
  (m >= 1) and 0 for m = 0 (plane potential theory with K = log r / (2 pi)).
* Neumann limit (Sec. 5.2): the interior normal derivative of the single layer,
  -cos(m theta)/2 from the closed form above (0 for m = 0), equals
  -mu/2 + K'_gamma[mu] with the oracle's K'_gamma.
* K'_gamma on an ellipse against QUADPACK (its smooth kernel's diagonal value
  kappa/(4 pi)), and spectral convergence of the trapezoid rule.
* Double layer (Sec. 5.3, Gauss's lemma): N_gamma[1] = 1 inside Gamma and 1/2
  on gamma, on a circle and an ellipse, so the interior limit is
  +mu/2 + N_gamma[mu](on gamma).
* eq. NeuBVPsystem with f = 0 on a flat elliptical Gamma (sigma = 0): the edge
  row recovers a harmonic u from its Neumann data, up to a constant, converging
  spectrally in the number of edge points.
* The Dirichlet trace row with f = 0 recovers a harmonic u from its boundary
  values with the jump +mu/(2a) (measured 1e-4, 1.5e-8, 9e-16 at 64, 128, 256
  points); with the printed -mu/(2a) the operator annihilates constants (Gauss's
  lemma: N_gamma[1] = 1/2 on gamma) and the solve is meaningless.
"""

import numpy as np
import pytest
from scipy.integrate import quad

from oracle.edge import (circle, dirichlet_edge_solve, double_layer,
                         double_layer_on_curve, ellipse, k_prime_on_curve,
                         neumann_edge_solve, single_layer, single_layer_grad)


@pytest.mark.parametrize("m", [0, 1, 2, 4])
def test_single_layer_on_the_circle(m):
    c = circle(128)             # trapezoid error ~ rho^n for targets at radius rho
    mu = np.cos(m * c.t)
    th = np.linspace(0.0, 2 * np.pi, 9)
    for rho in (0.3, 0.7):
        T = np.stack([rho * np.cos(th), rho * np.sin(th)], 1)
        ex = -rho ** m * np.cos(m * th) / (2 * m) if m else 0 * th
        assert np.abs(single_layer(c, mu, T) - ex).max() < 1e-14
        # radial derivative against the closed form -rho^(m-1) cos(m theta) / 2
        g = single_layer_grad(c, mu, T)
        dr = np.sum(g * T, 1) / rho
        exd = -rho ** (m - 1) * np.cos(m * th) / 2 if m else 0 * th
        assert np.abs(dr - exd).max() < 1e-13


@pytest.mark.parametrize("m", [0, 1, 3])
def test_neumann_limit_on_the_circle(m):
    """lim_{rho -> 1-} d/drho K_gamma[cos m t] = -mu/2 + K'_gamma[mu] (Sec. 5.2)."""
    c = circle(64)
    mu = np.cos(m * c.t)
    limit = -0.5 * mu if m else 0 * mu                 # from the closed form
    assert np.abs(-0.5 * mu + k_prime_on_curve(c, mu) - limit).max() < 1e-14


def test_k_prime_on_an_ellipse():
    A, B = 2.0, 0.7
    mu_f = lambda t: np.cos(2 * t) + 0.3 * np.sin(5 * t) + 0.2
    errs = []
    for n in (32, 64, 128, 256):
        e = ellipse(n, A, B)
        kp = k_prime_on_curve(e, mu_f(e.t))
        i = n // 8 + 1
        x, nu = e.x[i], e.nu[i]

        def integrand(t):
            y = np.array([A * np.cos(t), B * np.sin(t)])
            d = x - y
            r2 = d @ d
            sp = np.hypot(A * np.sin(t), B * np.cos(t))
            return 0.0 if r2 < 1e-30 else (d @ nu) / r2 / (2 * np.pi) * mu_f(t) * sp

        ref = quad(integrand, 0, 2 * np.pi, points=[e.t[i]], limit=400, epsabs=1e-15)[0]
        errs.append(abs(kp[i] - ref))
    assert errs[-1] < 1e-13 and errs[0] > 100 * errs[2], errs


@pytest.mark.parametrize("curve", [circle(64), ellipse(320, 2.0, 0.7)])
def test_double_layer_gauss_lemma(curve):
    one = np.ones(len(curve.t))
    assert np.abs(double_layer_on_curve(curve, one) - 0.5).max() < 1e-13
    inside = np.array([[0.1, 0.2], [-0.3, 0.1], [0.0, -0.4]])
    assert np.abs(double_layer(curve, one, inside) - 1.0).max() < 1e-13
    outside = np.array([[3.0, 0.5], [-2.5, -1.0]])
    assert np.abs(double_layer(curve, one, outside)).max() < 1e-13


def test_neumann_system_with_harmonic_solution():
    def u_ex(P):
        z = P[:, 0] + 1j * P[:, 1]
        return (z ** 3).real - 0.5 * (z ** 2).real + P[:, 0]

    def grad_u(P):
        z = P[:, 0] + 1j * P[:, 1]
        dz = 3 * z ** 2 - z + 1                   # f'(z) = u_x - i u_y
        return np.stack([dz.real, -dz.imag], 1)

    T = np.array([[0.3, 0.1], [-1.2, 0.2], [0.5, -0.4], [1.5, 0.0]])
    errs = []
    for n in (64, 128, 256):
        e = ellipse(n, 2.0, 0.7)
        fg = np.sum(grad_u(e.x) * e.nu, 1)
        assert abs(np.dot(e.w, fg)) < 1e-13                   # compatibility
        mu = neumann_edge_solve(e, fg)
        assert abs(np.dot(e.w, mu)) < 1e-12
        u = single_layer(e, mu, T)
        ue = u_ex(T)
        errs.append(np.abs((u - u.mean()) - (ue - ue.mean())).max())
    # measured 1.7e-6, 3.1e-10, 1.1e-14
    assert errs[2] < 1e-12 and errs[0] > 1e3 * errs[1], errs


def test_dirichlet_system_with_harmonic_solution():
    def u_ex(P):
        z = P[:, 0] + 1j * P[:, 1]
        return (z ** 3).real - 0.5 * (z ** 2).imag + P[:, 1] + 0.7

    T = np.array([[0.3, 0.1], [-1.2, 0.2], [0.5, -0.4], [1.5, 0.0]])
    errs = []
    for n in (64, 128, 256):
        e = ellipse(n, 2.0, 0.7)
        mu = dirichlet_edge_solve(e, u_ex(e.x))
        errs.append(np.abs(double_layer(e, mu, T) - u_ex(T)).max())
    assert errs[2] < 1e-12 and errs[0] > 1e3 * errs[1], errs
    e = ellipse(256, 2.0, 0.7)
    wrong = dirichlet_edge_solve(e, u_ex(e.x), jump_sign=-1.0)
    assert np.abs(double_layer(e, wrong, T) - u_ex(T)).max() > 0.1
