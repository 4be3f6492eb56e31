"""Plain, slow float64 CPU oracle of the parametrix method's discrete operators.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library (its own
Gauss-Legendre rules come from numpy, its own Lagrange interpolation,
quadrature, kernels and solver are written here from the paper).

What it computes (Goodwill & O'Neil, "A parametrix method for elliptic
surface PDEs"):

* kernels.py   -- the parametrix K = log r / (2 pi a(x')) (Sec. 4.2, eq.
  diff_param) and its remainder R for c = 0, b = 0 (Thm. parametrix, eq.
  explicit_remainder), which reduces to R_LB (Thm. parametrixLB, eq.
  explicit_remainderLB) for constant a; and for c != 0 the Hankel Green's
  function G = -(i / 4a) H0(sqrt(c/a) r), the remainder with its c terms
  and the constant-coefficient form of the Corollary (eq. bdd_remainder_helm).
* patch.py     -- tensor Lagrange interpolation of node data on a quad patch
  (the quad analogue of the interpolation in Sec. 6.1.1 remark / 6.1.2).
* quadrature.py-- the three quadrature classes of Sec. 6.1: smooth (6.1.3),
  singular self-patch polar rule (6.1.1, eq. radial_int) and nearly singular
  adaptive subdivision (6.1.2), plus the "near" test of Sec. 6.1.2.
* operator.py  -- the Nystrom operators R~ and K~ (Sec. 6.1, eq. IEsum):
  dense smooth sums plus near-field corrections; the second-kind operator
  I + R~ + (rank one) of Sec. 3 (null-space removal by adding int sigma),
  or I + R~ when c != 0 (complex weights).
* triangle.py  -- triangle patches (Sec. 6.1): the Koornwinder basis on the
  simplex and order-p Vioreanu-Rokhlin nodes and weights, generated from the
  published method (the paper's precomputed table is not available).
* triangle_operator.py -- the Nystrom operators on curved triangle patches
  given by their parameterisations (Sec. 6.1): polar self rule over the
  simplex, adaptive subdivision near rule, same correction form as operator.py.
* edge.py      -- the edge potentials of the boundary-value systems (Sec. 5) on
  planar curves with the trapezoid rule: single layer, its normal derivative
  K'_gamma on the curve, double layer N_gamma; their limits from inside Gamma.
* solve.py     -- restarted GMRES and dense LU, the solve of eq. IE and the
  representation u = K[sigma] (eq. representation) with the mean projection.

Readings of points the paper leaves open are listed in the design notes; the
ones that change arithmetic are restated in the docstrings where they apply.
Parity status: kernels, smooth sums, self rule, near rule, operators and the
solve are each pinned by tests against closed forms or independent library
quadrature (tests/test_oracle_*.py); the c != 0 kernels, operators and solve
by tests/test_oracle_helmholtz.py (Funk-Hecke eigenvalues on the sphere, the
Corollary's closed form, K0, finite differences, manufactured solutions); the
advection term by tests/test_oracle_advection.py; the triangle rule and
operators by tests/test_oracle_triangle.py; the edge operators by
tests/test_oracle_edge.py (plane potential theory, Gauss's lemma).
"""
