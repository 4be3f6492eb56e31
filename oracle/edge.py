"""Edge operators of the boundary-value systems (Sec. 5), on closed planar curves.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For an open surface Gamma with boundary gamma and binormal nu (tangent to Gamma,
normal to gamma, pointing away from Gamma), Sec. 5 represents the solution with
edge potentials of the parametrix K = log r / (2 pi a) (c = 0):

  K_gamma[mu](x)  = int_gamma K(x, x') mu(x') ds(x')                 (Neumann, eq. BC_rep)
  N_gamma[mu](x)  = int_gamma nu(x') . grad' K(x, x') mu(x') ds(x')  (Dirichlet, eq. DirichletRep)
  K'_gamma[mu](x) = int_gamma nu(x) . grad K(x, x') mu(x') ds(x'),  x on gamma

and imposes the boundary conditions through their limits from inside Gamma.
This module builds them for a flat Gamma in the plane z = 0 (a = 1 unless
given), where the paper's surface operators reduce to plane potential theory,
as the first piece of that row.

Edge quadrature (Sec. 6.1.4): the trapezoid rule in the curve's periodic
parameter, spectrally accurate for smooth periodic integrands.  On the curve the
kernels of K'_gamma and N_gamma are smooth (Thm. kern_smth): for y -> x,
nu(x).(x - y)/|x - y|^2 -> kappa(x)/2 with kappa the curvature (positive for a
convex Gamma), so the diagonal entry takes that limit.

Readings (limits from inside Gamma, K = +log r/(2 pi a)):
* Neumann (Sec. 5.2): nu . grad K_gamma[mu] -> -mu/(2a) + K'_gamma[mu], as printed.
* Dirichlet (Sec. 5.3): N_gamma[mu] -> +mu/(2a) + N_gamma[mu](on gamma).  The paper
  prints -mu/(2a) for this limit; with its own sign of K the double layer of a
  constant density is 1/a inside Gamma and 1/(2a) on gamma (Gauss), which fixes
  the sign as +.  (Its system eq. DirBVPsystem also writes N_Gamma[sigma] in the
  second row where the trace theorem has K_Gamma[sigma]; read as K_Gamma.)
"""

from __future__ import annotations

import numpy as np

INV_2PI = 0.5 / np.pi


class PlanarCurve:
    """Closed curve gamma(t), t in [0, 2 pi), given by callables for the point, first and
    second derivatives, traversed counter-clockwise around Gamma (nu = outward)."""

    def __init__(self, point, d1, d2, n: int):
        t = 2 * np.pi * np.arange(n) / n
        self.t = t
        self.x = point(t)
        xp, xpp = d1(t), d2(t)
        self.speed = np.hypot(xp[:, 0], xp[:, 1])
        tau = xp / self.speed[:, None]
        self.nu = np.stack([tau[:, 1], -tau[:, 0]], 1)         # outward for counter-clockwise
        self.kappa = (xp[:, 0] * xpp[:, 1] - xp[:, 1] * xpp[:, 0]) / self.speed ** 3
        self.w = (2 * np.pi / n) * self.speed                     # trapezoid ds weights


def single_layer(curve: PlanarCurve, mu, targets, a=1.0):
    """K_gamma[mu] at points off the curve [M, 2]."""
    d = targets[:, None, :] - curve.x[None, :, :]
    r2 = np.sum(d * d, axis=2)
    return (INV_2PI / a) * 0.5 * np.log(r2) @ (curve.w * mu)


def single_layer_grad(curve: PlanarCurve, mu, targets, a=1.0):
    """grad K_gamma[mu] at points off the curve: [M, 2]."""
    d = targets[:, None, :] - curve.x[None, :, :]
    r2 = np.sum(d * d, axis=2)
    return (INV_2PI / a) * np.einsum("mjc,mj,j->mc", d, 1.0 / r2, curve.w * mu)


def double_layer(curve: PlanarCurve, mu, targets, a=1.0):
    """N_gamma[mu] at points off the curve: nu(x') . grad' log|x - x'| / (2 pi a)."""
    d = curve.x[None, :, :] - targets[:, None, :]             # x' - x
    r2 = np.sum(d * d, axis=2)
    k = np.einsum("mjc,jc->mj", d, curve.nu) / r2
    return (INV_2PI / a) * k @ (curve.w * mu)


def _on_curve(curve: PlanarCurve, kernel_offdiag, diag, mu):
    n = len(curve.t)
    out = np.empty(n)
    for i in range(n):
        k = kernel_offdiag(i)
        k[i] = diag[i]
        out[i] = k @ (curve.w * mu)
    return out


def k_prime_on_curve(curve: PlanarCurve, mu, a=1.0):
    """K'_gamma[mu](x_i) = int nu(x_i) . (x_i - y) / (2 pi a |x_i - y|^2) mu ds (smooth kernel)."""
    def off(i):
        d = curve.x[i] - curve.x
        r2 = np.sum(d * d, axis=1)
        r2[i] = 1.0
        return (INV_2PI / a) * (d @ curve.nu[i]) / r2
    return _on_curve(curve, off, (INV_2PI / a) * 0.5 * curve.kappa, mu)


def double_layer_on_curve(curve: PlanarCurve, mu, a=1.0):
    """N_gamma[mu](x_i) for x_i on gamma: int nu(y) . (y - x_i) / (2 pi a |y - x_i|^2) mu ds."""
    def off(i):
        d = curve.x - curve.x[i]
        r2 = np.sum(d * d, axis=1)
        r2[i] = 1.0
        return (INV_2PI / a) * np.sum(d * curve.nu, axis=1) / r2
    return _on_curve(curve, off, (INV_2PI / a) * 0.5 * curve.kappa, mu)


def circle(n: int, R: float = 1.0) -> PlanarCurve:
    return PlanarCurve(lambda t: R * np.stack([np.cos(t), np.sin(t)], 1),
                       lambda t: R * np.stack([-np.sin(t), np.cos(t)], 1),
                       lambda t: R * np.stack([-np.cos(t), -np.sin(t)], 1), n)


def ellipse(n: int, A: float, B: float) -> PlanarCurve:
    return PlanarCurve(lambda t: np.stack([A * np.cos(t), B * np.sin(t)], 1),
                       lambda t: np.stack([-A * np.sin(t), B * np.cos(t)], 1),
                       lambda t: np.stack([-A * np.cos(t), -B * np.sin(t)], 1), n)


def neumann_edge_solve(curve: PlanarCurve, f_gamma, a=1.0):
    """mu of eq. NeuBVPsystem's second row on a flat Gamma with f = 0 (so sigma = 0):
    -mu/(2a) + K'_gamma[mu] = f_gamma.  That operator has a one-dimensional null
    space and its range is orthogonal to the constants, so the data must satisfy
    int f_gamma ds = 0 (the Neumann compatibility condition) and the rank-one term
    (int mu ds) 1 added here selects the solution with int mu ds = 0; u = K_gamma[mu]
    is then determined up to the constant the Neumann problem leaves free.
    Dense Nystrom matrix, LU."""
    n = len(curve.t)
    A = np.empty((n, n))
    eye = np.eye(n)
    for j in range(n):
        A[:, j] = k_prime_on_curve(curve, eye[j], a)
    A -= eye / (2 * a)
    A += np.outer(np.ones(n), curve.w)
    return np.linalg.solve(A, f_gamma)


def dirichlet_edge_solve(curve: PlanarCurve, f_gamma, a=1.0, jump_sign=1.0):
    """mu of the Dirichlet trace row on a flat Gamma with f = 0 (so sigma = 0):
    jump_sign * mu/(2a) + N_gamma[mu](on gamma) = f_gamma, u = N_gamma[mu] inside.
    jump_sign = +1 is reading of the module docstring; -1 is the sign printed in
    Sec. 5.3 (kept as a parameter so that the pin can show it fails)."""
    n = len(curve.t)
    A = np.empty((n, n))
    eye = np.eye(n)
    for j in range(n):
        A[:, j] = double_layer_on_curve(curve, eye[j], a)
    A += jump_sign * eye / (2 * a)
    return np.linalg.solve(A, f_gamma)
