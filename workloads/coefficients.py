"""Coefficient fields a(x) > 0 of div_Gamma(a grad_Gamma u) = f, with grad_Gamma a.

Each field returns the nodal values ``a`` [N] and the surface gradient
``grad_a`` [N, 3] (tangential), computed from closed forms: for an ambient
function, grad_Gamma a = (I - n n^T) grad a; for a function of the surface
parameters, grad_Gamma a = [y_s y_t] g^{-1} [a_s; a_t] (Sec. 2.2, eq. gradg).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .surfaces import Surface


@dataclass
class Coefficient:
    kind: str
    a: np.ndarray        # [N]
    grad_a: np.ndarray   # [N, 3] surface gradient


def _tangential(grad, normals):
    return grad - normals * np.sum(grad * normals, axis=-1, keepdims=True)


def constant_coefficient(surf: Surface, value: float = 1.0) -> Coefficient:
    return Coefficient("constant", np.full(surf.N, float(value)), np.zeros((surf.N, 3)))


def ellipsoid_coefficient(surf: Surface) -> Coefficient:
    """a(x) = 1 + 0.5 sin(2 x_1) cos(3 x_2) (first two Cartesian coordinates)."""
    x, y = surf.nodes[:, 0], surf.nodes[:, 1]
    a = 1.0 + 0.5 * np.sin(2 * x) * np.cos(3 * y)
    grad = np.stack([np.cos(2 * x) * np.cos(3 * y),
                     -1.5 * np.sin(2 * x) * np.sin(3 * y),
                     np.zeros_like(x)], -1)
    return Coefficient("sin2x_cos3y", a, _tangential(grad, surf.normals))


def torus_coefficient(surf: Surface) -> Coefficient:
    """a = exp(0.3 cos(theta) sin(2 phi)) on the torus (theta toroidal, phi poloidal)."""
    th, ph = surf.params["theta"], surf.params["phi"]
    R, r = surf.params["R"], surf.params["r"]
    a = np.exp(0.3 * np.cos(th) * np.sin(2 * ph))
    a_th = a * (-0.3 * np.sin(th) * np.sin(2 * ph))
    a_ph = a * (0.6 * np.cos(th) * np.cos(2 * ph))
    rho = R + r * np.cos(ph)
    e_th = np.stack([-np.sin(th), np.cos(th), np.zeros_like(th)], -1)
    e_ph = np.stack([-np.sin(ph) * np.cos(th), -np.sin(ph) * np.sin(th), np.cos(ph)], -1)
    grad = (a_th / rho)[:, None] * e_th + (a_ph / r)[:, None] * e_ph
    return Coefficient("exp_torus", a, grad)


def smooth_random_coefficient(surf: Surface, seed: int, K: int = 32,
                              amp: float = 0.4) -> Coefficient:
    """a = 1 + amp * tanh(g(x)), g(x) = sqrt(2/K) sum_k xi_k cos(omega_k . x + phi_k).

    omega_k ~ N(0, I_3), phi_k ~ U[0, 2 pi), xi_k ~ N(0, 1), drawn from
    numpy's default generator with the given seed.
    """
    rng = np.random.default_rng(seed)
    om = rng.standard_normal((K, 3))
    ph = rng.uniform(0.0, 2 * np.pi, K)
    xi = rng.standard_normal(K)
    arg = surf.nodes @ om.T + ph
    s = np.sqrt(2.0 / K)
    g = s * (np.cos(arg) @ xi)
    dg = -s * (np.sin(arg) * xi) @ om
    th = np.tanh(g)
    a = 1.0 + amp * th
    grad = (amp * (1 - th * th))[:, None] * dg
    return Coefficient(f"tanh_field_{seed}", a, _tangential(grad, surf.normals))
