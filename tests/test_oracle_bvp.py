"""Pins of the Neumann boundary-value oracle (Sec. 5.2, eq. NeuBVPsystem; oracle/bvp.py).

* Fourier oversampling: the trigonometric interpolant is exact on band-limited data.
* K'_Gamma on the edge patch: the polar rule about a point on the patch edge matches
  scipy's adaptive quad (QUADPACK), nested, of the same integral.
* The jump relation of Lemma jumpcdt: nu . grad_Gamma K_gamma[mu] at surface points
  approaching gamma tends to -mu / (2a) + K'_gamma[mu] (pins K'_gamma, its diagonal
  limit and the sign of the jump).
* The discrete operator without the rank-one term has exactly one near-zero singular
  value (reading 31); with it, the solution of a manufactured Newtonian problem on a
  torus band converges to the exact u (up to a constant) under refinement.
* Dirichlet (Sec. 5.3, constant a): the log-kernel polar rule on the edge patch
  (K_Gamma on gamma) matches nested QUADPACK; the double layer N_gamma[mu] from inside
  Gamma tends to +mu/(2a) + N_gamma[mu] on gamma (reading 28); the system has no null
  space and its manufactured solution converges under refinement.
* The edge-node correction rows do not depend on how many processes compute them.
"""

import numpy as np
import pytest

from conftest import oracle_processes
from oracle.bvp import (DirichletBVP, NeumannBVP, edge_correction_rows, k_edge_self_weights,
                        kp_self_weights, trig_interp_matrix)
from oracle.kernels import INV_2PI
from workloads.bvp import (band_coefficient, constant_band_coefficient, edge_a, newtonian_dirichlet,
                           newtonian_neumann, torus_band)


def test_trig_interpolation_is_exact_for_band_limited_data():
    M, F = 16, 6
    tk = 2 * np.pi * (np.arange(M) + 0.5) / M
    t = 2 * np.pi * np.arange(F * M) / (F * M)
    f = lambda s: 0.3 + np.cos(3 * s) - 0.5 * np.sin(7 * s) + 0.25 * np.cos(5 * s + 1)   # noqa: E731
    assert np.abs(trig_interp_matrix(M, F) @ f(tk) - f(t)).max() < 1e-13
    # the edge nodes are the oversampled points k F + F/2 (F even)
    F2 = 4
    I = trig_interp_matrix(M, F2)
    assert np.abs(I[F2 // 2::F2] - np.eye(M)).max() < 1e-13


def test_edge_patch_polar_rule_against_quadpack():
    from scipy.integrate import quad
    os_ = torus_band(2, 4, 6, 16, 4)
    co = band_coefficient(os_)
    B = NeumannBVP.__new__(NeumannBVP)          # geometry only: no operators built
    from oracle.operator import Discretization
    s = os_.surface
    B.osurf, B.curves = os_, os_.curves
    B.disc = Discretization(s.nodes, s.normals, s.tangents, s.curvature, s.weights, co.a,
                            co.grad_a, s.npatch, s.p)
    e = 3                                       # an edge node of the first circle
    P, u0, v0 = B.edge_patch(e)
    xe, nue = os_.curves[0].x[e], os_.curves[0].nu[e]
    patch = B.disc.patches[P]
    W = kp_self_weights(patch, u0, v0, xe, nue)
    xt = patch.evaluate(np.array([u0]), np.array([v0]))[0][0]    # the rule's centre
    p = patch.p
    for k in (0, p * p // 2 + 1, p * p - 1):
        ka, kb = divmod(k, p)

        def inner(u):
            def f(v):
                y, J, Lu, Lv = patch.evaluate(np.array([u]), np.array([v]))
                d = xt - y[0]
                return INV_2PI * float(d @ nue) / float(d @ d) * J[0] * Lu[0, ka] * Lv[0, kb]
            return quad(f, -1, 1, points=[v0], limit=200, epsabs=1e-15, epsrel=1e-12)[0]
        val = quad(inner, -1, 1, limit=200, epsabs=1e-15, epsrel=1e-12)[0]
        assert abs(W[k] - val) <= 1e-10 * np.abs(W).max(), (k, W[k], val)


def test_jump_relation_of_the_edge_single_layer():
    """nu . grad K_gamma[mu] from inside Gamma -> -mu/(2a) + K'_gamma[mu] (Lemma jumpcdt)."""
    os_ = torus_band(2, 4, 6, 32, 2)
    c0 = os_.curves[0]
    R, r = os_.R, os_.r
    a_e = edge_a(os_)[:c0.M]
    mu = 1.0 + 0.4 * np.cos(c0.t) + 0.2 * np.sin(2 * c0.t)
    # K'_gamma on curve 0 alone, trapezoid with the diagonal limit
    d = c0.x[:, None, :] - c0.x[None, :, :]
    r2 = np.sum(d * d, axis=2)
    np.fill_diagonal(r2, 1.0)
    Kp = INV_2PI * np.einsum("ijk,ik->ij", d, c0.nu) / r2 / a_e[None, :]
    np.fill_diagonal(Kp, INV_2PI * (-np.sum(c0.nu * c0.d2, 1) / (2 * np.sum(c0.d1 ** 2, 1))) / a_e)
    e = 5
    limit = -mu[e] / (2 * a_e[e]) + (Kp[e] * c0.w) @ mu
    # surface points at (theta0 + h / rho, t_e) with a fine trapezoid of the same
    # trigonometric interpolant of mu (exact quadrature of the smooth line integral)
    from oracle.bvp import trig_interp_matrix as tim
    from workloads.bvp import ambient_a
    Ff = 4096
    I = tim(c0.M, Ff)
    t = 2 * np.pi * np.arange(Ff * c0.M) / (Ff * c0.M)
    xs = np.stack([(R + r * np.cos(t)) * np.cos(c0.theta), (R + r * np.cos(t)) * np.sin(c0.theta),
                   r * np.sin(t)], -1)
    ws = (2 * np.pi / (Ff * c0.M)) * r
    mus = I @ mu
    a_s = ambient_a(xs)[0]
    te = c0.t[e]
    rho = R + r * np.cos(te)
    vals = []
    hs = np.array([4e-3, 2e-3, 1e-3])
    for h in hs:
        th = c0.theta + h / rho
        x = np.array([rho * np.cos(th), rho * np.sin(th), r * np.sin(te)])
        n = np.array([np.cos(te) * np.cos(th), np.cos(te) * np.sin(th), np.sin(te)])
        dd = x[None, :] - xs
        g = INV_2PI * (dd / np.sum(dd * dd, 1)[:, None] / a_s[:, None]).T @ (ws * mus)
        g = g - n * (g @ n)                      # surface gradient
        vals.append(g @ c0.nu[e])
    vals = np.array(vals)
    # O(h) approach: Richardson on h, h/2, h/4
    r1 = 2 * vals[1] - vals[0]
    r2_ = 2 * vals[2] - vals[1]
    extrap = (4 * r2_ - r1) / 3
    assert abs(extrap - limit) < 1e-6 * abs(limit), (vals, extrap, limit)
    # and the jump is the -1/(2a) of the lemma: the one-sided value is not the on-curve integral
    assert abs(extrap - (Kp[e] * c0.w) @ mu) > 0.1 * abs(mu[e] / (2 * a_e[e]))


@pytest.fixture(scope="module")
def small_systems():
    out = {}
    for key, args in (("coarse", (2, 4, 6, 16, 16)), ("fine", (2, 4, 8, 32, 16))):
        os_ = torus_band(*args)
        co = band_coefficient(os_)
        B = NeumannBVP(os_, co, edge_a(os_), edge_a(os_, True), processes=oracle_processes())
        out[key] = (os_, co, B)
    return out


def test_one_dimensional_null_space(small_systems):
    _, _, B = small_systems["coarse"]
    A = B.matrix()
    A[B.N:, B.N:] -= np.outer(np.ones(B.M), B.we)          # without the rank-one term
    sv = np.linalg.svd(A, compute_uv=False)
    assert sv[-1] < 1e-6 * sv[0]
    assert sv[-2] > 1e-2
    assert np.linalg.svd(B.matrix(), compute_uv=False)[-1] > 1e-3


def test_manufactured_neumann_solution_converges(small_systems):
    errs = []
    for key in ("coarse", "fine"):
        os_, co, B = small_systems[key]
        f, fg, v = newtonian_neumann(os_, co)
        sigma, mu, u = B.solve(f, fg)
        w = os_.surface.weights
        e = (u - v) - np.dot(w, u - v) / w.sum()
        vv = v - np.dot(w, v) / w.sum()
        errs.append(np.sqrt(np.dot(w, e * e) / np.dot(w, vv * vv)))
        # the operator form equals the assembled matrix
        top, bot = B.apply(sigma, mu)
        assert np.abs(np.concatenate([top, bot]) - B.matrix() @ np.concatenate([sigma, mu])).max() < 1e-10
    assert errs[0] < 5e-6 and errs[1] < 6e-7 and errs[1] < errs[0] / 4, errs


def test_log_kernel_edge_polar_rule_against_quadpack():
    from scipy.integrate import quad
    from oracle.operator import Discretization
    os_ = torus_band(2, 4, 6, 16, 4)
    co = constant_band_coefficient(os_)
    s = os_.surface
    B = NeumannBVP.__new__(NeumannBVP)
    B.osurf, B.curves = os_, os_.curves
    B.disc = Discretization(s.nodes, s.normals, s.tangents, s.curvature, s.weights, co.a,
                            co.grad_a, s.npatch, s.p)
    e = 19                                      # an edge node of the second circle
    P, u0, v0 = B.edge_patch(e)
    patch = B.disc.patches[P]
    W = k_edge_self_weights(patch, u0, v0)
    xt = patch.evaluate(np.array([u0]), np.array([v0]))[0][0]
    p = patch.p
    for k in (0, p * p // 2 + 1, p * p - 1):
        ka, kb = divmod(k, p)

        def inner(u):
            def f(v):
                y, J, Lu, Lv = patch.evaluate(np.array([u]), np.array([v]))
                d = xt - y[0]
                return INV_2PI * 0.5 * np.log(float(d @ d)) * J[0] * Lu[0, ka] * Lv[0, kb]
            return quad(f, -1, 1, points=[v0], limit=200, epsabs=1e-15, epsrel=1e-12)[0]
        val = quad(inner, -1, 1, limit=200, epsabs=1e-15, epsrel=1e-12)[0]
        assert abs(W[k] - val) <= 1e-10 * np.abs(W).max(), (k, W[k], val)


def test_double_layer_jump_from_inside():
    """N_gamma[mu] at surface points approaching gamma -> +mu/(2a) + N_gamma[mu](on gamma)."""
    os_ = torus_band(2, 4, 6, 32, 2)
    c0 = os_.curves[0]
    R, r = os_.R, os_.r
    a0 = 1.0
    mu = 1.0 + 0.4 * np.cos(c0.t) + 0.2 * np.sin(2 * c0.t)
    d = c0.x[:, None, :] - c0.x[None, :, :]
    r2 = np.sum(d * d, axis=2)
    np.fill_diagonal(r2, 1.0)
    Nd = -INV_2PI * np.einsum("ijk,jk->ij", d, c0.nu) / r2 / a0
    np.fill_diagonal(Nd, INV_2PI * (-np.sum(c0.nu * c0.d2, 1) / (2 * np.sum(c0.d1 ** 2, 1))) / a0)
    e = 9
    limit = mu[e] / (2 * a0) + (Nd[e] * c0.w) @ mu
    Ff = 4096
    I = trig_interp_matrix(c0.M, Ff)
    t = 2 * np.pi * np.arange(Ff * c0.M) / (Ff * c0.M)
    th0 = c0.theta
    xs = np.stack([(R + r * np.cos(t)) * np.cos(th0), (R + r * np.cos(t)) * np.sin(th0), r * np.sin(t)], -1)
    nus = np.stack([np.sin(th0) * np.ones_like(t), -np.cos(th0) * np.ones_like(t), 0 * t], -1)
    ws = (2 * np.pi / (Ff * c0.M)) * r
    mus = I @ mu
    te = c0.t[e]
    rho = R + r * np.cos(te)
    vals = []
    for h in (4e-3, 2e-3, 1e-3):
        th = th0 + h / rho
        x = np.array([rho * np.cos(th), rho * np.sin(th), r * np.sin(te)])
        dd = x[None, :] - xs
        vals.append(-INV_2PI / a0 * np.sum(np.sum(dd * nus, 1) / np.sum(dd * dd, 1) * ws * mus))
    r1 = 2 * vals[1] - vals[0]
    r2_ = 2 * vals[2] - vals[1]
    extrap = (4 * r2_ - r1) / 3
    assert abs(extrap - limit) < 1e-6 * abs(limit), (vals, extrap, limit)
    assert abs(extrap - (Nd[e] * c0.w) @ mu) > 0.1 * abs(mu[e] / (2 * a0))


def test_manufactured_dirichlet_solution_converges():
    errs = []
    for args in ((2, 4, 6, 16, 32), (2, 4, 7, 24, 32)):
        os_ = torus_band(*args)
        co = constant_band_coefficient(os_)
        B = DirichletBVP(os_, co, np.ones(os_.M), np.ones(sum(c.F * c.M for c in os_.curves)),
                         processes=oracle_processes())
        if not errs:
            assert np.linalg.svd(B.matrix(), compute_uv=False)[-1] > 1e-2     # no null space
        f, fg, v = newtonian_dirichlet(os_)
        sigma, mu, u = B.solve(f, fg)
        w = os_.surface.weights
        errs.append(float(np.sqrt(np.dot(w, (u - v) ** 2) / np.dot(w, v * v))))
        top, bot = B.apply(sigma, mu)
        assert np.abs(np.concatenate([top, bot]) - B.matrix() @ np.concatenate([sigma, mu])).max() < 1e-10
    assert errs[0] < 1e-6 and errs[1] < 1e-7 and errs[1] < errs[0] / 5, errs


def test_edge_correction_rows_do_not_depend_on_the_worker_count():
    """The edge-node correction rows (K'_Gamma and K~ kinds) computed over spawned
    processes equal the serial ones to rounding (the workers rebuild the patches from
    the surface arrays; each row's terms and their order are the same)."""
    from oracle.operator import Discretization
    os_ = torus_band(2, 4, 6, 16, 4)
    co = band_coefficient(os_)
    s = os_.surface
    B = NeumannBVP.__new__(NeumannBVP)          # geometry only: no operators built
    B.osurf, B.curves = os_, os_.curves
    disc = Discretization(s.nodes, s.normals, s.tangents, s.curvature, s.weights, co.a,
                          co.grad_a, s.npatch, s.p)
    xe = np.concatenate([c.x for c in os_.curves])
    nue = np.concatenate([c.nu for c in os_.curves])
    tasks = [(kind, xe[e], nue[e], *B.edge_patch(e), {})
             for kind, e in (("kp", 0), ("kp", 7), ("kp", 19), ("k", 3), ("k", 24))]
    serial = np.array(edge_correction_rows(disc, tasks, None))
    pooled = np.array(edge_correction_rows(disc, tasks, 2))
    assert np.all(np.isfinite(serial)) and np.abs(serial).max() > 0
    assert np.abs(pooled - serial).max() <= 1e-14 * np.abs(serial).max()
