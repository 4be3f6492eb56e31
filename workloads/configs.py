"""Named workloads: the surfaces, coefficients and right-hand sides used by the
tests and the benchmark.

Full-size workloads (the paper-style test problems at production size):

* ``sphere_1536``     unit sphere, cubed sphere 6 x 2 x 2 patches, 8 x 8 GL
                      nodes (1,536 nodes), a = 1, f = Y_3^2.
* ``ellipsoid_9600``  ellipsoid (1, 1.5, 2), 6 x 4 x 4 patches, 10 x 10 nodes
                      (9,600 nodes), a = 1 + 0.5 sin(2x) cos(3y), f = seeded
                      sum of 10 Y_l^m (l <= 8), mean zero.
* ``torus_98304``     torus R = 2, r = 0.7, 64 x 24 patches, 8 x 8 nodes
                      (98,304 nodes), a = exp(0.3 cos(theta) sin(2 phi)),
                      f = cos(3 phi) sin(theta), mean zero.

Reduced versions of the same families (``*_small``) keep the oracle fast.

The paper's own test problems (Sec. 7), a = 1:

* ``wavy_torus_<N>``      r = ((3 + cos v + 0.6 cos 5u) cos u, (...) sin u, sin v),
                          f from the Newtonian potential centred at (-3, -3, 4)
                          (manufactured solution; ``paper_problem`` returns u too).
* ``ellipsoid_paper_<N>`` semi-axes (4.5, 2.25, 3), same manufactured solution.
* ``sphere_paper_<N>``    unit sphere, f = random combination of Y_1^0, Y_3^3,
                          Y_10^6, Y_10^7 (exact u from the eigenvalues).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .coefficients import (Coefficient, constant_coefficient, ellipsoid_coefficient,
                           smooth_random_coefficient, torus_coefficient)
from .rhs import (four_harmonic_problem, newtonian_problem, random_harmonic_rhs,
                  sphere_harmonic_rhs, torus_rhs)
from .surfaces import Surface, cubed_sphere, star_surface, torus, wavy_torus


@dataclass
class Workload:
    name: str
    surface: Surface
    coeff: Coefficient
    f: np.ndarray
    description: str

    @property
    def N(self) -> int:
        return self.surface.N


def _sphere(m, p):
    s = cubed_sphere(m, p)
    return s, constant_coefficient(s), sphere_harmonic_rhs(s, 3, 2)


def _ellipsoid(m, p, seed=0):
    s = cubed_sphere(m, p, axes=(1.0, 1.5, 2.0))
    return s, ellipsoid_coefficient(s), random_harmonic_rhs(s, seed)


def star_batch(m: int = 8, p: int = 8, n_rhs: int = 64, n_coeff: int = 8):
    """Batched workload: the star-shaped surface with n_coeff smooth random
    coefficient fields a = 1 + 0.4 tanh(g) (seeds 0..n_coeff-1) and n_rhs
    right-hand sides, each a mean-zero N(0,1) combination of all real Y_l^m with
    1 <= l <= 12 (seeds 0..n_rhs-1)."""
    s = star_surface(m, p)
    coeffs = [smooth_random_coefficient(s, seed) for seed in range(n_coeff)]
    fs = np.stack([random_harmonic_rhs(s, seed, n_terms=168, lmax=12) for seed in range(n_rhs)])
    return s, coeffs, fs


def _torus(nt, nph, p):
    s = torus(nt, nph, p)
    return s, torus_coefficient(s), torus_rhs(s)


WORKLOADS = {
    "sphere_1536": (lambda: _sphere(2, 8),
                    "unit sphere, 6x2x2 patches, 8x8 GL nodes (1,536), a=1, f=Y_3^2"),
    "ellipsoid_9600": (lambda: _ellipsoid(4, 10),
                       "ellipsoid (1,1.5,2), 6x4x4 patches, 10x10 GL nodes (9,600), "
                       "a=1+0.5 sin(2x)cos(3y), f=sum of 10 Y_l^m (l<=8), mean zero"),
    "torus_98304": (lambda: _torus(64, 24, 8),
                    "torus R=2 r=0.7, 64x24 patches, 8x8 GL nodes (98,304), "
                    "a=exp(0.3 cos(theta) sin(2 phi)), f=cos(3 phi) sin(theta)"),
    # reduced sizes of the same families
    "sphere_small": (lambda: _sphere(1, 6), "unit sphere, 6x1x1 patches, 6x6 nodes (216)"),
    "sphere_384": (lambda: _sphere(1, 8), "unit sphere, 6x1x1 patches, 8x8 nodes (384)"),
    "ellipsoid_small": (lambda: _ellipsoid(2, 6),
                        "ellipsoid (1,1.5,2), 6x2x2 patches, 6x6 nodes (864)"),
    "ellipsoid_2400": (lambda: _ellipsoid(2, 10),
                       "ellipsoid (1,1.5,2), 6x2x2 patches, 10x10 nodes (2,400)"),
    "torus_small": (lambda: _torus(16, 6, 6),
                    "torus R=2 r=0.7, 16x6 patches, 6x6 nodes (3,456)"),
    "torus_6144": (lambda: _torus(16, 6, 8),
                   "torus R=2 r=0.7, 16x6 patches, 8x8 nodes (6,144)"),
    "star_24576": (lambda: (lambda s: (s, smooth_random_coefficient(s, 0),
                                       random_harmonic_rhs(s, 0, n_terms=168, lmax=12)))(
                       star_surface(8, 8)),
                   "star rho=1+0.3 sin(3 theta) cos(2 phi), 6x8x8 patches, 8x8 nodes (24,576), "
                   "a=1+0.4 tanh(g) seed 0, f=mean-zero N(0,1) combination of Y_l^m, l<=12"),
    "wavy_torus_small": (lambda: _paper("wavy", wavy_torus(9, 3, 6)),
                         "wavy torus, 9x3 patches, 6x6 nodes (972), a=1, Newtonian f"),
    "wavy_torus_12288": (lambda: _paper("wavy", wavy_torus(24, 8, 8)),
                         "wavy torus, 24x8 patches, 8x8 nodes (12,288), a=1, Newtonian f"),
    "wavy_torus_58752": (lambda: _paper("wavy", wavy_torus(51, 18, 8)),
                         "wavy torus, 51x18 patches, 8x8 nodes (58,752), a=1, Newtonian f"),
    "ellipsoid_paper_small": (lambda: _paper("ell", cubed_sphere(2, 6, axes=(4.5, 2.25, 3.0))),
                              "ellipsoid (4.5, 2.25, 3), 6x2x2 patches, 6x6 nodes (864), a=1"),
    "ellipsoid_paper_6144": (lambda: _paper("ell", cubed_sphere(4, 8, axes=(4.5, 2.25, 3.0))),
                             "ellipsoid (4.5, 2.25, 3), 6x4x4 patches, 8x8 nodes (6,144), a=1"),
    "ellipsoid_paper_24576": (lambda: _paper("ell", cubed_sphere(8, 8, axes=(4.5, 2.25, 3.0))),
                              "ellipsoid (4.5, 2.25, 3), 6x8x8 patches, 8x8 nodes (24,576), a=1"),
    "sphere_paper_1536": (lambda: _paper("sph", cubed_sphere(2, 8)),
                          "unit sphere, 6x2x2 patches, 8x8 nodes, f = Y_1^0, Y_3^3, Y_10^6, Y_10^7"),
    "sphere_paper_6144": (lambda: _paper("sph", cubed_sphere(4, 8)),
                          "unit sphere, 6x4x4 patches, 8x8 nodes, f = Y_1^0, Y_3^3, Y_10^6, Y_10^7"),
    "star_small": (lambda: (lambda s: (s, smooth_random_coefficient(s, 0),
                                       random_harmonic_rhs(s, 0, n_terms=168, lmax=12)))(
                       star_surface(2, 6)),
                   "star, 6x2x2 patches, 6x6 nodes (864)"),
}


def _paper(kind, s):
    c = constant_coefficient(s)
    f, _ = four_harmonic_problem(s) if kind == "sph" else newtonian_problem(s, c)
    return s, c, f


def paper_problem(name: str):
    """(Workload, exact u) of one of the paper's test problems."""
    wl = make_workload(name)
    if name.startswith("sphere_paper"):
        _, u = four_harmonic_problem(wl.surface)
    else:
        _, u = newtonian_problem(wl.surface, wl.coeff)
    return wl, u


def make_workload(name: str) -> Workload:
    build, desc = WORKLOADS[name]
    s, c, f = build()
    return Workload(name=name, surface=s, coeff=c, f=np.asarray(f, dtype=np.float64),
                    description=desc)
