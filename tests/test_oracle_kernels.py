"""Pins of the oracle's kernels against what the paper fixes independently.

* R is the surface operator applied to K (eq. diff_remainder): checked by
  finite differences of K in ambient space, R = grad_G a . grad K
  + a (Lap K - d_nn K) - 2 a H d_n K, on random points of a torus with a
  variable coefficient (no reuse of the closed form).
* Unit sphere, a = 1: R_LB = -1/(4 pi) for every pair (the constant of
  Sec. 3, with the sign of eq. explicit_remainderLB).
* Diagonal limit (Thm. remainderLB, eq. limiting_behaviour):
  R_LB -> -(H^2 sin^2 2t + kappa_G cos^2 2t)/(4 pi) along direction t.
* Dilation (Sec. 3 conjecture, item 3): R_{s Gamma}(s x, s y) s^2 = R_Gamma(x, y).
* Brute force in 40-digit arithmetic on a tiny random point set.
"""

import numpy as np
import pytest

from oracle.kernels import parametrix, remainder
from oracle.operator import Discretization
from workloads import cubed_sphere, torus, make_workload


def _torus_point(R, r, th, ph):
    rho = R + r * np.cos(ph)
    x = np.array([rho * np.cos(th), rho * np.sin(th), r * np.sin(ph)])
    n = np.array([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)])
    H = (R + 2 * r * np.cos(ph)) / (2 * r * rho)
    kg = np.cos(ph) / (r * rho)
    e_th = np.array([-np.sin(th), np.cos(th), 0.0])
    e_ph = np.array([-np.sin(ph) * np.cos(th), -np.sin(ph) * np.sin(th), np.cos(ph)])
    return x, n, H, kg, e_th, e_ph


def test_remainder_equals_surface_operator_of_parametrix():
    rng = np.random.default_rng(1)
    R0, r0 = 2.0, 0.7

    def a_fn(x):
        return 1.0 + 0.3 * np.sin(x[0]) * np.cos(2 * x[1]) + 0.1 * x[2]

    def grad_a(x):
        return np.array([0.3 * np.cos(x[0]) * np.cos(2 * x[1]),
                         -0.6 * np.sin(x[0]) * np.sin(2 * x[1]), 0.1])

    for _ in range(20):
        th, ph, th2, ph2 = rng.uniform(0, 2 * np.pi, 4)
        x, n, H, _, _, _ = _torus_point(R0, r0, th, ph)
        y, _, _, _, _, _ = _torus_point(R0, r0, th2, ph2)
        if np.linalg.norm(x - y) < 0.3:
            continue
        ay = a_fn(y)

        def K(z):
            return parametrix(z, y[None, :], np.array([ay]))[0]

        h = 1e-3
        E = np.eye(3)
        grad = np.array([(K(x + h * e) - K(x - h * e)) / (2 * h) for e in E])
        lap = sum((K(x + h * e) - 2 * K(x) + K(x - h * e)) / h ** 2 for e in E)
        dnn = (K(x + h * n) - 2 * K(x) + K(x - h * n)) / h ** 2
        dn = grad @ n
        g = grad_a(x)
        gG = g - n * (g @ n)
        ax = a_fn(x)
        fd = gG @ grad + ax * (lap - dnn) - 2 * ax * H * dn
        val = remainder(x, n, H, ax, gG, y[None, :], np.array([ay]))[0]
        assert abs(fd - val) < 1e-5 * max(1.0, abs(val)), (fd, val)


def _sphere_constant():
    from conftest import golden
    return golden("closed_forms.json")["sphere_remainder_constant"]["value"]   # -1/(4 pi)


R_SPHERE = _sphere_constant()


def test_sphere_remainder_is_constant():
    s = cubed_sphere(1, 6)
    rng = np.random.default_rng(0)
    i = rng.integers(0, s.N, 10)
    for k in i:
        ys = np.delete(s.nodes, k, axis=0)
        v = remainder(s.nodes[k], s.normals[k], s.curvature[k], 1.0, np.zeros(3), ys,
                      np.ones(len(ys)))
        assert np.abs(v - R_SPHERE).max() < 1e-13


@pytest.mark.parametrize("alpha", [0.0, 0.4, np.pi / 4, 1.1, np.pi / 2])
def test_remainder_diagonal_limit(alpha):
    R0, r0 = 2.0, 0.7
    th, ph = 0.3, 0.8
    x, n, H, kg, e_th, e_ph = _torus_point(R0, r0, th, ph)
    rho = R0 + r0 * np.cos(ph)
    s = 1e-4
    y, _, _, _, _, _ = _torus_point(R0, r0, th + s * np.cos(alpha) / rho, ph + s * np.sin(alpha) / r0)
    v = remainder(x, n, H, 1.0, np.zeros(3), y[None, :], np.ones(1))[0]
    lim = -(H * H * np.sin(2 * alpha) ** 2 + kg * np.cos(2 * alpha) ** 2) / (4 * np.pi)
    assert abs(v - lim) < 1e-3 * abs(lim) + 1e-5


def test_dilation_invariance_of_smooth_remainder():
    wl = make_workload("ellipsoid_small")
    s = wl.surface
    d1 = Discretization.from_workload(wl)
    s2 = s.scaled(2.5)
    d2 = Discretization(s2.nodes, s2.normals, s2.tangents, s2.curvature, s2.weights,
                        wl.coeff.a, wl.coeff.grad_a / 2.5, s2.npatch, s2.p)
    rows = [0, 17, 400, 863]
    M1 = d1.smooth_matrix("R", rows)
    M2 = d2.smooth_matrix("R", rows)
    assert np.abs(M1 - M2).max() < 1e-12 * np.abs(M1).max()
    # K on the dilated surface: w scales by s^2 and log gains log(s)
    K1 = d1.smooth_matrix("K", rows)
    K2 = d2.smooth_matrix("K", rows)
    shift = np.log(2.5) / (2 * np.pi) * (s2.weights / wl.coeff.a)
    shift = np.tile(shift, (len(rows), 1))
    shift[np.arange(len(rows)), rows] = 0.0
    assert np.abs(K2 - (6.25 * K1 + shift)).max() < 1e-12 * np.abs(K2).max()


def test_brute_force_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(3)
    N = 12
    x = rng.standard_normal((N, 3))
    n = rng.standard_normal((N, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    H = rng.uniform(-1, 1, N)
    a = rng.uniform(0.5, 1.5, N)
    g = rng.standard_normal((N, 3))
    w = rng.uniform(0.1, 1, N)
    sig = rng.standard_normal(N)
    d = Discretization(x, n, np.tile([1, 0, 0, 0, 1, 0.0], (N, 1)), H, w, a, g, npatch=N, p=1)
    yR = d.smooth_apply("R", sig)
    yK = d.smooth_apply("K", sig)
    for i in range(N):
        accR = mp.mpf(0)
        accK = mp.mpf(0)
        for j in range(N):
            if j == i:
                continue
            r = [mp.mpf(x[i, c]) - mp.mpf(x[j, c]) for c in range(3)]
            r2 = sum(c * c for c in r)
            q = sum(mp.mpf(n[i, c]) * r[c] for c in range(3)) / r2
            gr = sum(mp.mpf(g[i, c]) * r[c] for c in range(3))
            Rv = (mp.mpf(a[i]) / mp.mpf(a[j])) * (q * q / mp.pi - mp.mpf(H[i]) * q / mp.pi) \
                + gr / (2 * mp.pi * mp.mpf(a[j]) * r2)
            Kv = mp.log(mp.sqrt(r2)) / (2 * mp.pi * mp.mpf(a[j]))
            accR += mp.mpf(w[j]) * Rv * mp.mpf(sig[j])
            accK += mp.mpf(w[j]) * Kv * mp.mpf(sig[j])
        assert abs(float(accR) - yR[i]) < 1e-13 * max(1.0, abs(float(accR)))
        assert abs(float(accK) - yK[i]) < 1e-13 * max(1.0, abs(float(accK)))
