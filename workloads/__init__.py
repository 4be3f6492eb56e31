"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package only *describes problems*: closed surfaces sampled at tensor
Gauss-Legendre nodes on quadrilateral patches (positions, outward normals,
tangent vectors, mean curvature, smooth-rule weights), coefficient fields
``a`` with their surface gradients, and right-hand sides ``f``.  It contains
none of the parametrix method's arithmetic (kernels, quadrature corrections,
solvers); both the CUDA library and the oracle consume what it produces.
"""

from .surfaces import (  # noqa: F401
    Surface,
    cubed_sphere,
    torus,
    star_surface,
    wavy_torus,
    gauss_legendre,
)
from .coefficients import (  # noqa: F401
    Coefficient,
    constant_coefficient,
    ellipsoid_coefficient,
    torus_coefficient,
    smooth_random_coefficient,
)
from .rhs import (  # noqa: F401
    real_sph_harm,
    project_mean_zero,
    sphere_harmonic_rhs,
    random_harmonic_rhs,
    torus_rhs,
    newtonian_problem,
    four_harmonic_problem,
)
from .configs import (  # noqa: F401
    Workload,
    make_workload,
    paper_problem,
    star_batch,
    WORKLOADS,
)
