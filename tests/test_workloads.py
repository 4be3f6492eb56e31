"""Geometry fixtures against closed forms (surface area, Gauss-Bonnet, volume,
Minkowski identities, torus mean curvature).  These pin the inputs shared by
the oracle and the CUDA path; none of the method's arithmetic is involved."""

import numpy as np
import pytest

from workloads import cubed_sphere, torus, make_workload
from workloads.rhs import real_sph_harm


SURFACES = [
    ("sphere", lambda: cubed_sphere(2, 8)),
    ("ellipsoid", lambda: cubed_sphere(2, 10, axes=(1.0, 1.5, 2.0))),
    ("torus", lambda: torus(16, 6, 8)),
]


def ellipsoid_area(a, b, c):
    """Area of an ellipsoid by Legendre's elliptic-integral formula (c >= b >= a)."""
    from scipy.special import ellipeinc, ellipkinc
    a, b, c = sorted((a, b, c))[::-1]          # a >= b >= c
    phi = np.arccos(c / a)
    m = (a * a * (b * b - c * c)) / (b * b * (a * a - c * c))
    s = np.sin(phi)
    return 2 * np.pi * c * c + 2 * np.pi * a * b / s * (
        ellipeinc(phi, m) * s * s + ellipkinc(phi, m) * np.cos(phi) ** 2)


@pytest.mark.parametrize("name,make", SURFACES)
def test_geometry_invariants(name, make):
    s = make()
    w, n, x = s.weights, s.normals, s.nodes
    area = ellipsoid_area(1.0, 1.5, 2.0) if name == "ellipsoid" else s.area
    assert abs(w.sum() - area) < 1e-9 * area
    # Gauss-Bonnet: int kappa_G = 2 pi chi = 4 pi (1 - genus)
    assert abs(np.dot(w, s.gauss_curvature) - 4 * np.pi * (1 - s.genus)) < 1e-8
    # int n = 0 and int x.n = 3 Vol (divergence theorem)
    assert np.abs(w @ n).max() < 1e-12
    assert abs(np.dot(w, np.sum(x * n, 1)) / 3 - s.volume) < 1e-9 * s.volume
    # Minkowski: int H n = 0, int H (x.n) = area
    assert np.abs((w * s.curvature) @ n).max() < 1e-11
    assert abs(np.dot(w * s.curvature, np.sum(x * n, 1)) - area) < 1e-9 * area
    # normals are unit and agree with y_u x y_v
    c = np.cross(s.tangents[:, :3], s.tangents[:, 3:])
    c /= np.linalg.norm(c, axis=1)[:, None]
    assert np.abs(np.sum(c * n, 1) - 1).max() < 1e-13


def test_torus_mean_curvature_closed_form():
    s = torus(8, 4, 6)
    R, r = 2.0, 0.7
    ph = s.params["phi"]
    # principal curvatures 1/r and cos(phi)/(R + r cos(phi))
    H = 0.5 * (1 / r + np.cos(ph) / (R + r * np.cos(ph)))
    assert np.abs(H - s.curvature).max() < 1e-13


def test_spherical_harmonics_orthonormal():
    s = cubed_sphere(3, 12)
    ys = [real_sph_harm(l, m, s.nodes) for l, m in [(0, 0), (1, -1), (3, 2), (3, -2), (8, 5)]]
    G = np.array([[np.dot(s.weights, a * b) for b in ys] for a in ys])
    assert np.abs(G - np.eye(len(ys))).max() < 1e-9
    # Y_3^2 closed form (1/4) sqrt(105/pi) (x^2 - y^2) z
    x, y, z = s.nodes.T
    assert np.abs(real_sph_harm(3, 2, s.nodes) - 0.25 * np.sqrt(105 / np.pi) * (x * x - y * y) * z).max() < 1e-13


def test_workloads_mean_zero_rhs():
    for name in ["sphere_1536", "ellipsoid_9600", "torus_6144"]:
        wl = make_workload(name)
        assert abs(np.dot(wl.surface.weights, wl.f)) < 1e-12 * np.abs(wl.f).max()
        assert wl.coeff.a.min() > 0
        # surface gradient is tangential
        assert np.abs(np.sum(wl.coeff.grad_a * wl.surface.normals, 1)).max() < 1e-12
