"""Inputs of the paper's own test problems (Sec. 7) against closed forms and
independent computations: the wavy torus geometry, the Newtonian manufactured
right-hand side and the four-harmonic sphere problem.  No GPU."""

import numpy as np
import pytest
from numpy.polynomial.legendre import legval

from workloads import cubed_sphere, wavy_torus, newtonian_problem, four_harmonic_problem
from workloads import constant_coefficient, paper_problem
from workloads.rhs import real_sph_harm


def spectral_area(amp, n=256):
    """Area of the wavy torus by the periodic trapezoid rule with FFT derivatives
    of the position map (independent of the analytic tangents)."""
    u = 2 * np.pi * np.arange(4 * n) / (4 * n)
    v = 2 * np.pi * np.arange(n) / n
    U, V = np.meshgrid(u, v, indexing="ij")
    rho = 3 + np.cos(V) + amp * np.cos(5 * U)
    X = np.stack([rho * np.cos(U), rho * np.sin(U), np.sin(V)], -1)
    ku = np.fft.fftfreq(4 * n, 1.0 / (4 * n))[:, None, None]
    kv = np.fft.fftfreq(n, 1.0 / n)[None, :, None]
    Xu = np.real(np.fft.ifft(1j * ku * np.fft.fft(X, axis=0), axis=0))
    Xv = np.real(np.fft.ifft(1j * kv * np.fft.fft(X, axis=1), axis=1))
    J = np.linalg.norm(np.cross(Xu, Xv), axis=-1)
    return J.mean() * 4 * np.pi ** 2


def test_wavy_torus_geometry():
    """At the paper's 58,752 nodes (51 x 18 patches of 8 x 8)."""
    s = wavy_torus(51, 18, 8)
    w, n, x = s.weights, s.normals, s.nodes
    area = spectral_area(0.6)
    assert abs(w.sum() - area) < 1e-12 * area
    assert abs(np.dot(w, s.gauss_curvature)) < 1e-7                  # genus 1
    assert np.abs(w @ n).max() < 1e-10
    assert abs(np.dot(w, np.sum(x * n, 1)) / 3 - 6 * np.pi ** 2) < 1e-12 * 6 * np.pi ** 2
    # Minkowski: int H n = 0, int H x.n = area (H = 1 on the unit sphere)
    assert np.abs(w @ (s.curvature[:, None] * n)).max() < 1e-7
    assert abs(np.dot(w, s.curvature * np.sum(x * n, 1)) - area) < 1e-9 * area
    # outward normals: x.n > 0 on the outer equator (v = 0)
    outer = np.cos(s.params["v"]) > 0.99
    assert np.all(np.sum((x * n)[outer], 1) > 0)


def test_wavy_torus_without_waves_is_the_standard_torus():
    s = wavy_torus(16, 6, 8, amp=0.0)
    v = s.params["v"]
    H = (3 + 2 * np.cos(v)) / (2 * (3 + np.cos(v)))                # R = 3, r = 1
    KG = np.cos(v) / (3 + np.cos(v))
    assert np.abs(s.curvature - H).max() < 1e-13
    assert np.abs(s.gauss_curvature - KG).max() < 1e-13
    assert abs(s.weights.sum() - 12 * np.pi ** 2) < 1e-10


def test_newtonian_rhs_on_the_unit_sphere_matches_the_legendre_series():
    """-1/|x - x0| = -sum_l P_l(cos g) / r0^(l+1) on |x| = 1 < r0, and the surface
    Laplacian multiplies P_l by -l(l+1): Lap_G v = sum_l l(l+1) P_l(cos g) / r0^(l+1)."""
    s = cubed_sphere(3, 8)
    c = constant_coefficient(s)
    x0 = np.array([-3.0, -3.0, 4.0])
    f, u = newtonian_problem(s, c, x0)
    r0 = np.linalg.norm(x0)
    cg = s.nodes @ x0 / r0
    L = np.arange(0, 80)
    lap = legval(cg, L * (L + 1) / r0 ** (L + 1))
    w = s.weights
    lap -= np.dot(w, lap) / w.sum()
    assert np.abs(f - lap).max() < 1e-12
    v = -legval(cg, 1.0 / r0 ** (L + 1))
    assert np.abs(u - (v - np.dot(w, v) / w.sum())).max() < 1e-13


def test_newtonian_rhs_integrates_to_zero_before_projection():
    # div_G(a grad_G v) has zero surface integral (divergence theorem on a closed surface)
    s = wavy_torus(51, 18, 8)
    from workloads import smooth_random_coefficient
    co = smooth_random_coefficient(s, 1)
    x0 = np.array([-3.0, -3.0, 4.0])
    d = s.nodes - x0
    rho = np.linalg.norm(d, axis=1)
    f_raw, _ = newtonian_problem(s, co, x0)
    # the projection removed only quadrature-level noise
    grad = d / rho[:, None] ** 3
    dn = np.sum(grad * s.normals, 1)
    dnn = 1 / rho ** 3 - 3 * np.sum(d * s.normals, 1) ** 2 / rho ** 5
    f_unproj = (np.sum(co.grad_a * (grad - s.normals * dn[:, None]), 1)
                + co.a * (-2 * s.curvature * dn - dnn))
    assert abs(np.dot(s.weights, f_unproj)) < 1e-9 * np.dot(s.weights, np.abs(f_unproj))
    assert np.abs(f_raw - f_unproj).max() < 1e-7


def test_four_harmonic_problem_eigen_relation():
    s = cubed_sphere(2, 8)
    f, u = four_harmonic_problem(s, 0)
    terms = [(1, 0), (3, 3), (10, 6), (10, 7)]
    Y = np.stack([real_sph_harm(l, m, s.nodes) for l, m in terms], 1)
    c, *_ = np.linalg.lstsq(Y, f, rcond=None)
    assert np.abs(Y @ c - f).max() < 1e-12
    lam = np.array([-l * (l + 1) for l, _ in terms], dtype=float)
    assert np.abs(Y @ (c / lam) - u).max() < 1e-12


@pytest.mark.parametrize("name", ["wavy_torus_small", "ellipsoid_paper_small", "sphere_paper_1536"])
def test_paper_problems_are_mean_zero(name):
    wl, u = paper_problem(name)
    w = wl.surface.weights
    assert abs(np.dot(w, wl.f)) < 1e-12 * np.dot(w, np.abs(wl.f))
    assert abs(np.dot(w, u)) < 1e-12 * np.dot(w, np.abs(u))
