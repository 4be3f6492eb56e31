"""Pins of the oracle's c != 0 kernels and operators (Sec. 4.2, Sec. 7.1).

What the paper and the mathematics fix independently of the code:

* The planar Green's function solves (a Delta_2 + c) G = delta: its radial
  derivatives match finite differences, a G' 2 pi r -> 1 (unit source
  strength, which fixes the sign of G), G - log(r)/(2 pi a) tends to a
  constant, and for c/a < 0 G is the modified-Helmholtz kernel
  -K0(kappa r)/(2 pi a) (an independent library routine).
* eq. explicit_remainder with constant a, c equals the Corollary's
  eq. bdd_remainder_helm (derived in the paper through Hankel identities).
* Thm. parametrix off the diagonal: div_G(a grad_G K) + c K = R, checked by
  finite differences of K in ambient space (eq. diff_remainder) on a torus
  with variable a and variable complex c.
* c -> 0 recovers the c = 0 remainder of Thm. parametrixLB.
* Dilation: Gamma -> s Gamma with c is Gamma with s^2 c (K unchanged, R times s^-2).
* Sec. 4.2's theorem on the zero set of c: K and R grow like log c(x') as c(x') -> 0
  (K - log(k)/(2 pi a) and R - c(x) log(k)/(2 pi a) converge).
* Unit sphere, constant a and c (Sec. 7.1: adding c shifts the eigenvalues
  -a l(l+1) of the surface operator): K and R are zonal, so by the
  Funk-Hecke formula Y_l^m is an eigenfunction of both, with eigenvalues
  kappa_l = 2 pi int_0^2 K(r) P_l(1 - r^2/2) r dr and rho_l likewise.
  Thm. parametrix in spectral form is (c - a l(l+1)) kappa_l = 1 + rho_l
  for every l; at a resonance c = a l(l+1), I + R has the null vector Y_l.
* The discrete operators K~ and R~ reproduce kappa_l, rho_l on the sphere,
  and the solve of f = sum f_lm Y_l^m returns sum f_lm Y_l^m / (c - l(l+1))
  (216-node sphere).
"""

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import eval_legendre, k0

from conftest import oracle_processes
from oracle.kernels import (green, parametrix_c, remainder, remainder_c,
                            remainder_constant_c, remainder_scaled_c, wavenumber)
from oracle.operator import Discretization, NearField, apply_K, apply_R
from oracle.solve import relative_l2, solve
from test_oracle_kernels import _torus_point
from workloads import cubed_sphere, real_sph_harm

COEFFS = [(1.0, 4.0), (1.0, -4.0), (2.0, 3.0 + 1.0j), (0.5, -1.0)]


@pytest.mark.parametrize("a,c", COEFFS)
def test_green_derivatives_match_finite_differences(a, c):
    r = np.linspace(0.2, 3.0, 13)
    G, G1, G2 = green(r, a, c)
    h = 1e-4
    Gp, Gm = green(r + h, a, c)[0], green(r - h, a, c)[0]
    assert np.all(np.abs((Gp - Gm) / (2 * h) - G1) < 1e-6 * np.abs(G1) + 1e-9)
    assert np.all(np.abs((Gp - 2 * G + Gm) / h ** 2 - G2) < 1e-5 * np.abs(G2) + 1e-6)
    # away from 0 the radial Helmholtz equation a (G'' + G'/r) + c G = 0
    assert np.abs(a * (G2 + G1 / r) + c * G).max() < 1e-12 * np.abs(a * G2).max()


@pytest.mark.parametrize("a,c", COEFFS)
def test_green_has_unit_source_strength(a, c):
    """Flux of a grad G through a small circle -> 1, and G ~ log(r)/(2 pi a)."""
    r = np.array([1e-3, 1e-5, 1e-7])
    G, G1, _ = green(r, a, c)
    flux = 2 * np.pi * r * a * G1
    assert np.abs(flux - 1.0).max() < 1e-4
    assert abs(flux[-1] - 1.0) < 1e-11
    d = G - np.log(r) / (2 * np.pi * a)
    assert abs(d[1] - d[2]) < 1e-9


def test_modified_helmholtz_green_is_k0():
    r = np.linspace(0.01, 5.0, 50)
    for a, c in [(1.0, -4.0), (2.0, -3.0), (0.3, -0.01)]:
        kappa = np.sqrt(-c / a)
        G = green(r, a, c)[0]
        ref = -k0(kappa * r) / (2 * np.pi * a)
        assert np.abs(G.imag).max() < 1e-15 * np.abs(G).max()
        assert np.abs(G.real - ref).max() < 1e-13 * np.abs(ref).max()


def test_wavenumber_branch():
    """k^2 = c/a on the real axis as physics fixes it, and continuous across both real
    half-axes (the cut is on the negative imaginary axis of c/a, outside the wedge)."""
    assert wavenumber(-4.0, 1.0) == 2j
    assert wavenumber(complex(-4.0, -0.0), 1.0) == 2j
    assert wavenumber(9.0, 1.0) == 3.0
    assert wavenumber(complex(9.0, -0.0), 1.0) == 3.0
    k = wavenumber(3.0 + 1.0j, 2.0)
    assert abs(k * k - (3.0 + 1.0j) / 2.0) < 1e-15
    t = np.linspace(-1.0, 1.0, 2001)
    for q in (4.0 + 0.8j * t, -4.0 + 0.8j * t, 2.0 * t + 0.0j, 2.0 * t - 0.3j * t ** 2):
        k = wavenumber(q, 1.0)
        assert np.allclose(k * k, q, atol=1e-14)
        assert np.abs(np.diff(k)).max() < 0.05        # no jump between neighbours


@pytest.mark.parametrize("a0,c0", COEFFS)
def test_constant_coefficient_remainder_is_the_corollary(a0, c0):
    """eq. explicit_remainder == eq. bdd_remainder_helm on torus points."""
    rng = np.random.default_rng(7)
    for _ in range(10):
        th, ph, th2, ph2 = rng.uniform(0, 2 * np.pi, 4)
        x, n, H, _, _, _ = _torus_point(2.0, 0.7, th, ph)
        y = np.array([_torus_point(2.0, 0.7, th2 + d, ph2 - d)[0] for d in (0.0, 0.3, 1.1)])
        ones = np.ones(len(y))
        R1 = remainder_c(x, n, H, a0, np.zeros(3), c0, y, a0 * ones, c0 * ones)
        R2 = remainder_constant_c(x, n, H, a0, c0, y)
        assert np.abs(R1 - R2).max() < 1e-13 * max(1.0, np.abs(R2).max())


def test_remainder_equals_surface_operator_of_parametrix_c():
    """div_G(a grad_G K) + c(x) K = R away from x = y (Thm. parametrix, eq. diff_form)."""
    rng = np.random.default_rng(3)

    def a_fn(x):
        return 1.0 + 0.3 * np.sin(x[0]) * np.cos(2 * x[1]) + 0.1 * x[2]

    def grad_a(x):
        return np.array([0.3 * np.cos(x[0]) * np.cos(2 * x[1]),
                         -0.6 * np.sin(x[0]) * np.sin(2 * x[1]), 0.1])

    def c_fn(x):                        # complex, sign-changing real part
        return 2.0 * x[0] + 1.5j * np.cos(x[1]) - 1.0

    checked = 0
    while checked < 20:
        th, ph, th2, ph2 = rng.uniform(0, 2 * np.pi, 4)
        x, n, H, _, _, _ = _torus_point(2.0, 0.7, th, ph)
        y = _torus_point(2.0, 0.7, th2, ph2)[0]
        if np.linalg.norm(x - y) < 0.3 or abs(c_fn(y)) < 0.2:
            continue
        ay, cy = np.array([a_fn(y)]), np.array([c_fn(y)])

        def K(z):
            return parametrix_c(z, y[None, :], ay, cy)[0]

        h = 1e-3
        E = np.eye(3)
        grad = np.array([(K(x + h * e) - K(x - h * e)) / (2 * h) for e in E])
        lap = sum((K(x + h * e) - 2 * K(x) + K(x - h * e)) / h ** 2 for e in E)
        dnn = (K(x + h * n) - 2 * K(x) + K(x - h * n)) / h ** 2
        g = grad_a(x)
        gG = g - n * (g @ n)
        ax = a_fn(x)
        fd = gG @ grad + ax * (lap - dnn) - 2 * ax * H * (grad @ n) + c_fn(x) * K(x)
        val = remainder_c(x, n, H, ax, gG, c_fn(x), y[None, :], ay, cy)[0]
        sc = remainder_scaled_c(x, n, H, ax, gG, c_fn(x), y[None, :], wavenumber(cy, ay))[0]
        assert abs(fd - val) < 1e-5 * max(1.0, abs(val)), (fd, val)
        assert abs(sc / ay[0] - val) < 1e-13 * max(1.0, abs(val))
        checked += 1


def test_kernels_grow_like_log_c_as_c_vanishes():
    """Sec. 4.2 theorem on Gamma_c = {c = 0}: K and R are O(log c(x')) as c(x') -> 0.
    With k = sqrt(c/a), K = -(i/4a) H0(k r) = (log k + log r - log 2 + gamma)/(2 pi a)
    - i/(4a) + o(1), so K - log(k)/(2 pi a) tends to that constant; R's c-term
    (c(x) - a(x) c(y)/a(y)) G tends to c(x) G, so R - c(x) log(k)/(2 pi a) converges
    (measured: R itself falls by c(x) ln(10)/(2 pi a) per factor 100 in c)."""
    x = np.array([0.3, -0.2, 0.9])
    n = np.array([0.0, 0.0, 1.0])
    y = np.array([[1.1, 0.4, 0.2]])
    a, cx = 1.7, 0.3
    r = np.linalg.norm(x - y)
    lim = (np.log(r) - np.log(2.0) + np.euler_gamma) / (2 * np.pi * a) - 0.25j / a
    shifted = []
    for c in (1e-4, 1e-6, 1e-8, 1e-10):
        k = np.sqrt(c / a)
        K = parametrix_c(x, y, np.array([a]), np.array([c]))[0]
        assert abs(K - np.log(k) / (2 * np.pi * a) - lim) < 10 * c, c
        R = remainder_c(x, n, 0.5, a, np.zeros(3), cx, y, np.array([a]), np.array([c]))[0]
        shifted.append(R - cx * np.log(k) / (2 * np.pi * a))
    steps = np.abs(np.diff(shifted))
    assert steps[-1] < 1e-6 and steps[0] > steps[-1]
    assert abs(shifted[0] - shifted[-1]) < 1e-3 * abs(shifted[-1])


def test_dilation_scales_c():
    """Dilating Gamma by s turns a Delta + c into a Delta + s^2 c on the original
    surface: K_{s Gamma, c}(s x, s y) = K_{Gamma, s^2 c}(x, y) (no log shift when
    c != 0) and s^2 R_{s Gamma, c}(s x, s y) = R_{Gamma, s^2 c}(x, y), with H and
    grad_G a scaling as 1/s.  A term of eq. explicit_remainder with a wrong power
    of k or r breaks it."""
    rng = np.random.default_rng(13)
    for sc in (0.5, 3.0):
        for _ in range(5):
            th, ph = rng.uniform(0, 2 * np.pi, 2)
            x, n, H, _, _, _ = _torus_point(2.0, 0.7, th, ph)
            y = np.array([_torus_point(2.0, 0.7, *rng.uniform(0, 2 * np.pi, 2))[0]
                          for _ in range(4)])
            ay = 1.0 + rng.random(4)
            cy = rng.standard_normal(4) + 0.5j * rng.standard_normal(4)
            cx = 1.3 - 0.4j
            gG = rng.standard_normal(3)
            gG -= n * (gG @ n)
            K1 = parametrix_c(sc * x, sc * y, ay, cy)
            K2 = parametrix_c(x, y, ay, sc ** 2 * cy)
            assert np.abs(K1 - K2).max() < 1e-13 * np.abs(K2).max()
            R1 = remainder_c(sc * x, n, H / sc, 1.7, gG / sc, cx, sc * y, ay, cy)
            R2 = remainder_c(x, n, H, 1.7, gG, sc ** 2 * cx, y, ay, sc ** 2 * cy)
            assert np.abs(sc ** 2 * R1 - R2).max() < 1e-12 * np.abs(R2).max()


def test_remainder_tends_to_the_c_zero_remainder():
    rng = np.random.default_rng(11)
    for _ in range(10):
        x = rng.standard_normal(3)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        g = rng.standard_normal(3)
        g -= n * (g @ n)
        y = x + 0.7 * rng.standard_normal((4, 3))
        ay = 1.0 + rng.random(4)
        R0 = remainder(x, n, 0.4, 1.3, g, y, ay)
        Rc = remainder_c(x, n, 0.4, 1.3, g, 1e-10 * 1.3, y, ay, 1e-10 * ay)
        assert np.abs(Rc - R0).max() < 1e-8 * np.abs(R0).max()


# ------------------------------------------------------------------ unit sphere
_POLE = np.array([0.0, 0.0, 1.0])


def _sphere_point(r):
    t = 1.0 - 0.5 * r * r
    return np.array([np.sqrt(max(0.0, 1.0 - t * t)), 0.0, t])


def _funk_hecke(F, l):
    """2 pi int_0^2 F(r) P_l(1 - r^2/2) r dr (Funk-Hecke with t = 1 - r^2/2)."""
    o = {"limit": 400, "epsabs": 1e-14, "epsrel": 1e-13}
    re = quad(lambda r: (F(r) * eval_legendre(l, 1 - r * r / 2) * r).real, 0, 2, **o)[0]
    im = quad(lambda r: (F(r) * eval_legendre(l, 1 - r * r / 2) * r).imag, 0, 2, **o)[0]
    return 2 * np.pi * (re + 1j * im)


def sphere_eigenvalues(a, c, l):
    """(kappa_l, rho_l) of K and R on the unit sphere (n = x, H = 1, grad a = 0)."""
    av, cv = np.array([a]), np.array([c])

    def FK(r):
        return parametrix_c(_POLE, _sphere_point(r)[None, :], av, cv)[0]

    def FR(r):
        return remainder_c(_POLE, _POLE, 1.0, a, np.zeros(3), c,
                           _sphere_point(r)[None, :], av, cv)[0]

    return _funk_hecke(FK, l), _funk_hecke(FR, l)


@pytest.mark.parametrize("a,c", COEFFS)
def test_sphere_spectral_identity(a, c):
    """(c - a l(l+1)) kappa_l = 1 + rho_l: Thm. parametrix on each spherical harmonic."""
    for l in range(0, 11):
        kap, rho = sphere_eigenvalues(a, c, l)
        assert abs((c - a * l * (l + 1)) * kap - (1 + rho)) < 1e-11 * max(1.0, abs(1 + rho)), l


def test_sphere_resonance_gives_a_null_vector():
    """At c = a l(l+1) the surface operator kills Y_l, and so does I + R."""
    for a, l in [(1.0, 2), (0.5, 3)]:
        _, rho = sphere_eigenvalues(a, a * l * (l + 1), l)
        assert abs(1 + rho) < 1e-11


def _sphere_disc(m, p, c):
    s = cubed_sphere(m, p)
    N = len(s.weights)
    return Discretization(s.nodes, s.normals, s.tangents, s.curvature, s.weights,
                          np.ones(N), np.zeros((N, 3)), s.npatch, s.p, c=c)


@pytest.mark.parametrize("c", [4.0, -4.0, 2.0 + 1.0j])
def test_sphere_operators_reproduce_the_eigenvalues(c):
    """K~ Y_l = kappa_l Y_l, R~ Y_l = rho_l Y_l on a 1536-node sphere (sampled rows)."""
    d = _sphere_disc(2, 8, c)
    rows = np.arange(0, d.N, 61)
    nf = NearField(d, rows=rows, processes=oracle_processes())
    for l, m in [(0, 0), (1, 0), (2, 1), (3, -3), (5, 4)]:
        Y = real_sph_harm(l, m, d.x)
        kap, rho = sphere_eigenvalues(1.0, c, l)
        eK = np.abs(apply_K(d, nf, Y, rows) - kap * Y[rows]).max()
        eR = np.abs(apply_R(d, nf, Y, rows) - rho * Y[rows]).max()
        assert eK < 1e-8, (l, eK)
        assert eR < 1e-5, (l, eR)


@pytest.fixture(scope="module")
def helmholtz_sphere():
    return _sphere_disc(1, 6, 4.0)              # 216 nodes


def test_sphere_helmholtz_solve(helmholtz_sphere):
    """Sec. 7.1 with c = 4: u = sum f_lm Y_l^m / (c - l(l+1))."""
    d = helmholtz_sphere
    nf = NearField(d, processes=oracle_processes())
    terms = [(1, 0, 1.0), (3, 3, -0.5), (0, 0, 0.25), (2, -1, 0.7)]
    f = sum(cf * real_sph_harm(l, m, d.x) for l, m, cf in terms)
    uex = sum(cf * real_sph_harm(l, m, d.x) / (4.0 - l * (l + 1)) for l, m, cf in terms)
    u, sigma, _ = solve(d, nf, f, return_sigma=True)
    assert relative_l2(u, uex, d.w) < 1e-4      # measured 4.3e-5 (216 nodes)
    # sigma solves eq. IE: on the sphere sigma = sum f_lm Y / (1 + rho_l)
    sex = sum(cf * real_sph_harm(l, m, d.x) / (1 + sphere_eigenvalues(1.0, 4.0, l)[1])
              for l, m, cf in terms)
    assert relative_l2(sigma, sex, d.w) < 1e-3  # measured 2.9e-4
    u2, _, info = solve(d, nf, f, method="gmres", tol=1e-13, return_sigma=True)
    assert relative_l2(u2, u, d.w) < 1e-11
    assert info["iters"] < 40


def _e4_real(x, n):
    """a linear in z, 1 to 3 over the ellipsoid (z in [-2, 2]); c = -4 - exp(x/2)."""
    from workloads.coefficients import _tangential
    ga = np.tile([0.0, 0.0, 0.5], (len(x), 1))
    return 2.0 + 0.5 * x[:, 2], _tangential(ga, n), -4.0 - np.exp(x[:, 0] / 2)


def _e4_complex(x, n):
    from workloads.coefficients import _tangential
    ez = np.exp(x[:, 2])
    ga = np.stack([0 * ez, 0 * ez, ez], 1)
    return 1.0 + ez, _tangential(ga, n), 4.0 * (1 + 0.2 * x[:, 1] + 0.2j * np.sin(x[:, 0]))


@pytest.mark.parametrize("coeffs,tol", [(_e4_real, 1e-3), (_e4_complex, 6e-3)])
def test_manufactured_solution_variable_a_and_c(coeffs, tol):
    """Sec. 7.4 procedure with the paper's two variable-coefficient examples.

    Real: a linear in z varying by a factor of 3, c = -4 - exp(x/2) (measured
    2.0e-4).
    Complex: a = 1 + e^z, c = 4 (1 + 0.2 y + 0.2 i sin x) (measured 2.7e-3; the
    imaginary part changes sign across the surface, so this also pins the branch
    of k = sqrt(c/a): the root with Im k >= 0 jumps there and gave 0.34).
    v = -1/|x - x0| restricted to an ellipsoid (216 nodes), f = div_G(a grad_G v)
    + c v from the closed-form gradient and Hessian of v (eq. diff_remainder
    with Lap v = 0); the solve must return v itself (no mean projection when
    c != 0).
    """
    s = cubed_sphere(1, 6, axes=(1.0, 1.5, 2.0))
    a, ga, c = coeffs(s.nodes, s.normals)
    d = Discretization(s.nodes, s.normals, s.tangents, s.curvature, s.weights,
                       a, ga, s.npatch, s.p, c=c)
    nf = NearField(d, processes=oracle_processes())
    x0 = np.array([-3.0, -3.0, 4.0])
    dx = d.x - x0
    rho = np.linalg.norm(dx, axis=1)
    v = -1.0 / rho
    grad = dx / rho[:, None] ** 3
    dn = np.sum(grad * d.n, 1)
    dnn = 1.0 / rho ** 3 - 3 * np.sum(dx * d.n, 1) ** 2 / rho ** 5
    lap_G = -2 * d.H * dn - dnn
    grad_G = grad - d.n * dn[:, None]
    f = np.sum(d.g * grad_G, 1) + d.a * lap_G + c * v
    u = solve(d, nf, f)
    if np.isrealobj(c):
        assert np.abs(u.imag).max() < 1e-12      # real c: the kernels are real
    assert relative_l2(u, v, d.w) < tol
