"""Pins of the oracle's three quadrature rules (Sec. 6.1.1-6.1.3).

* Flat patch: the polar rule of eq. radial_int reduces to one-dimensional
  integrals over theta with closed-form radial parts (for F = log r:
  int_0^L r log r dr = L^2/2 log L - L^2/4; for the grad a term,
  int_0^L (g.e/r) r dr = g.e L), compared with scipy's adaptive QUADPACK.
* The same flat patch with a single basis function, against nested QUADPACK.
* Curved patches: the self rule and the near rule against scipy's adaptive
  quadrature of the same integrand (no shared panels or nodes).
* Self-convergence against finer settings (the paper's own test, Sec. 6.1.1
  and 6.1.2).
"""

import numpy as np
import pytest
from scipy import integrate

from oracle.kernels import INV_2PI, parametrix_scaled, remainder_scaled
from oracle.operator import Discretization
from oracle.patch import PatchInterpolant, lagrange_basis
from oracle.quadrature import near_weights, ray_length, self_weights, corner_sectors
from workloads import make_workload
from numpy.polynomial.legendre import leggauss


def flat_patch(p):
    t, _ = leggauss(p)
    X = np.zeros((p, p, 3))
    X[..., 0] = t[:, None]
    X[..., 1] = t[None, :]
    return PatchInterpolant(X, np.ones((p, p))), t


def theta_quad(fn, u0, v0):
    total = 0.0
    for a, b in corner_sectors(u0, v0):
        val, _ = integrate.quad(fn, a, b, epsabs=1e-15, epsrel=1e-14, limit=500)
        total += val
    return total


@pytest.mark.parametrize("i0,j0", [(0, 0), (2, 3), (5, 1)])
def test_flat_patch_log_kernel_closed_radial(i0, j0):
    pt, t = flat_patch(6)
    u0, v0 = t[i0], t[j0]
    x = np.array([u0, v0, 0.0])
    _, WK = self_weights(pt, u0, v0, x, np.array([0, 0, 1.0]), 0.0, 1.0, np.zeros(3))

    def f(th):
        L = ray_length(u0, v0, th)
        return INV_2PI * (0.5 * L * L * np.log(L) - 0.25 * L * L)

    assert abs(WK.sum() - theta_quad(f, u0, v0)) < 1e-13


@pytest.mark.parametrize("i0,j0", [(0, 0), (3, 3), (5, 2)])
def test_flat_patch_gradient_term_closed_radial(i0, j0):
    pt, t = flat_patch(6)
    u0, v0 = t[i0], t[j0]
    x = np.array([u0, v0, 0.0])
    g = np.array([0.7, -0.3, 0.0])
    WR, _ = self_weights(pt, u0, v0, x, np.array([0, 0, 1.0]), 0.0, 1.0, g)

    def f(th):
        e = np.array([np.cos(th), np.sin(th), 0.0])
        return -INV_2PI * (g @ e) * ray_length(u0, v0, th)

    assert abs(WR.sum() - theta_quad(f, u0, v0)) < 1e-13


def test_flat_patch_single_basis_function_nested_quad():
    pt, t = flat_patch(5)
    i0, j0, k = 1, 3, 7
    u0, v0 = t[i0], t[j0]
    x = np.array([u0, v0, 0.0])
    g = np.array([0.2, 0.5, 0.0])
    WR, WK = self_weights(pt, u0, v0, x, np.array([0, 0, 1.0]), 0.0, 1.0, g)
    a, b = divmod(k, 5)

    def basis(u, v):
        return lagrange_basis(t, np.array([u]))[0, a] * lagrange_basis(t, np.array([v]))[0, b]

    def inner(th, which):
        L = ray_length(u0, v0, th)
        c, s = np.cos(th), np.sin(th)
        if which == "K":
            f = lambda r: INV_2PI * r * np.log(r) * basis(u0 + r * c, v0 + r * s)
        else:
            f = lambda r: -INV_2PI * (g[0] * c + g[1] * s) * basis(u0 + r * c, v0 + r * s)
        return integrate.quad(f, 0.0, L, epsabs=1e-15, epsrel=1e-13, limit=200)[0]

    refK = theta_quad(lambda th: inner(th, "K"), u0, v0)
    refR = theta_quad(lambda th: inner(th, "R"), u0, v0)
    assert abs(WK[k] - refK) < 1e-12
    assert abs(WR[k] - refR) < 1e-12


@pytest.fixture(scope="module")
def ell():
    wl = make_workload("ellipsoid_small")
    return Discretization.from_workload(wl)


def test_curved_self_rule_against_quadpack(ell):
    d = ell
    P, i0, j0, k = 5, 1, 4, 9
    i = P * 36 + i0 * 6 + j0
    pt = d.patches[P]
    u0, v0 = d.t[i0], d.t[j0]
    WR, WK = self_weights(pt, u0, v0, d.x[i], d.n[i], d.H[i], d.a[i], d.g[i])
    nt = pt.normal_at(u0, v0)
    a, b = divmod(k, 6)

    def integrand(r, th, which):
        u, v = u0 + r * np.cos(th), v0 + r * np.sin(th)
        y, J, Lu, Lv = pt.evaluate(np.array([u]), np.array([v]))
        ell_k = Lu[0, a] * Lv[0, b]
        if which == "R":
            F = remainder_scaled(d.x[i], nt, d.H[i], d.a[i], d.g[i], y)[0]
        else:
            F = parametrix_scaled(d.x[i], y)[0]
        return F * ell_k * J[0] * r

    for which, W in (("R", WR), ("K", WK)):
        def inner(th):
            L = ray_length(u0, v0, th)
            return integrate.quad(integrand, 1e-9, L, args=(th, which), epsabs=1e-14,
                                  epsrel=1e-12, limit=200)[0]
        ref = theta_quad(inner, u0, v0)
        assert abs(W[k] - ref) < 1e-10 * np.abs(W).max(), (which, W[k], ref)


def test_near_rule_against_quadpack(ell):
    d = ell
    i = 0
    P = [q for q in d.near_patches(i) if q != 0][0]
    pt = d.patches[P]
    WR, WK, _ = near_weights(pt, d.x[i], d.n[i], d.H[i], d.a[i], d.g[i])
    k = 0
    a, b = divmod(k, 6)

    def f(v, u, which):
        y, J, Lu, Lv = pt.evaluate(np.array([u]), np.array([v]))
        if which == "R":
            F = remainder_scaled(d.x[i], d.n[i], d.H[i], d.a[i], d.g[i], y)[0]
        else:
            F = parametrix_scaled(d.x[i], y)[0]
        return F * Lu[0, a] * Lv[0, b] * J[0]

    for which, W in (("R", WR), ("K", WK)):
        ref, _ = integrate.dblquad(f, -1, 1, -1, 1, args=(which,), epsabs=1e-14, epsrel=1e-12)
        assert abs(W[k] - ref) < 1e-11 * np.abs(W).max(), (which, W[k], ref)


def test_self_rule_self_convergence(ell):
    d = ell
    for i in [0, 7, 21, 35]:
        pt = d.patches[0]
        u0, v0 = d.t[i // 6], d.t[i % 6]
        args = (d.x[i], d.n[i], d.H[i], d.a[i], d.g[i])
        W0 = self_weights(pt, u0, v0, *args)
        W1 = self_weights(pt, u0, v0, *args, levels=20, h_max=0.25, max_width=np.pi / 48)
        for a, b in zip(W0, W1):
            assert np.abs(a - b).max() < 1e-11 * np.abs(b).max()


def test_near_rule_self_convergence(ell):
    d = ell
    for i in [0, 7, 35]:
        for P in d.near_patches(i)[1:]:
            args = (d.x[i], d.n[i], d.H[i], d.a[i], d.g[i])
            a = near_weights(d.patches[P], *args, tol=1e-13)
            b = near_weights(d.patches[P], *args, tol=1e-15)
            assert np.abs(a[0] - b[0]).max() < 1e-13 * np.abs(b[0]).max()
            assert np.abs(a[1] - b[1]).max() < 1e-13 * np.abs(b[1]).max()
