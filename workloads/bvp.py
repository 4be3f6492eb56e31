"""Open surfaces with boundary for the boundary-value systems (Sec. 5).

A band of the torus ((R + r cos phi) cos theta, (R + r cos phi) sin theta, r sin phi),
theta0 <= theta <= theta0 + n_band dtheta, phi the full circle, on tensor
Gauss-Legendre patches (n_band x n_phi patches of p x p nodes; patch index
a * n_phi + b, theta along u and phi along v, as in surfaces.torus).  Its boundary
is two circles of the tube, gamma_c(t) = point at (theta_c, phi = t), each with M
edge nodes t_k = 2 pi (k + 1/2) / M (never at a patch corner when M is a multiple
of n_phi) and an oversampled grid of F M points t_j = 2 pi j / (F M) (F even: the
edge nodes are the oversampled points j = k F + F / 2).  The binormal nu is tangent
to the surface, normal to gamma and points away from Gamma: -e_theta on the first
circle, +e_theta on the second.

Coefficient: a(x) = exp(0.2 x_1 + 0.3 x_3), an ambient field, with its surface
gradient.  Manufactured data (Sec. 7.5's test): u = v on Gamma for the Newtonian
potential v(x) = -1 / |x - x0|, f = div_Gamma(a grad_Gamma v) from the closed-form
gradient and Hessian of v, and the Neumann data f_gamma = nu . grad v on gamma.
Geometry and data only: no arithmetic of the method.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .coefficients import Coefficient
from .surfaces import Surface, gauss_legendre

A_GRAD = np.array([0.2, 0.0, 0.3])          # a(x) = exp(A_GRAD . x)


@dataclass
class EdgeCurve:
    """One boundary circle: edge nodes (base grid) and the oversampled grid."""
    theta: float
    sign: float            # nu = sign * e_theta
    M: int
    F: int
    t: np.ndarray          # [M] parameters of the edge nodes
    x: np.ndarray          # [M, 3] points
    d1: np.ndarray         # [M, 3] gamma'(t)
    d2: np.ndarray         # [M, 3] gamma''(t)
    nu: np.ndarray         # [M, 3] binormal
    w: np.ndarray          # [M] trapezoid weights (2 pi / M) |gamma'|
    to: np.ndarray         # [F M] oversampled parameters
    xo: np.ndarray         # [F M, 3]
    nuo: np.ndarray        # [F M, 3]
    wo: np.ndarray         # [F M] trapezoid weights (2 pi / (F M)) |gamma'|
    speedo: np.ndarray     # [F M] |gamma'| at the oversampled points


@dataclass
class OpenSurface:
    surface: Surface
    curves: list
    R: float
    r: float

    @property
    def M(self) -> int:
        return sum(c.M for c in self.curves)


def _torus_point(th, ph, R, r):
    rho = R + r * np.cos(ph)
    return np.stack([rho * np.cos(th), rho * np.sin(th), r * np.sin(ph)], -1)


def _curve(theta, sign, M, F, R, r) -> EdgeCurve:
    def geo(t):
        th = np.full_like(t, theta)
        x = _torus_point(th, t, R, r)
        d1 = np.stack([-r * np.sin(t) * np.cos(th), -r * np.sin(t) * np.sin(th), r * np.cos(t)], -1)
        d2 = np.stack([-r * np.cos(t) * np.cos(th), -r * np.cos(t) * np.sin(th), -r * np.sin(t)], -1)
        e_th = np.stack([-np.sin(th), np.cos(th), np.zeros_like(t)], -1)
        return x, d1, d2, sign * e_th
    t = 2 * np.pi * (np.arange(M) + 0.5) / M
    to = 2 * np.pi * np.arange(F * M) / (F * M)
    x, d1, d2, nu = geo(t)
    xo, d1o, _, nuo = geo(to)
    so = np.linalg.norm(d1o, axis=1)
    return EdgeCurve(theta=theta, sign=sign, M=M, F=F, t=t, x=x, d1=d1, d2=d2, nu=nu,
                     w=(2 * np.pi / M) * np.linalg.norm(d1, axis=1), to=to, xo=xo, nuo=nuo,
                     wo=(2 * np.pi / (F * M)) * so, speedo=so)


def torus_band(n_band: int, n_phi: int, p: int, M: int, F: int = 16, theta0: float = 0.0,
               dtheta: float = np.pi / 8, R: float = 2.0, r: float = 0.7) -> OpenSurface:
    if F % 2 or M % n_phi:
        raise ValueError("F must be even and M a multiple of n_phi")
    t, wt = gauss_legendre(p)
    dph = 2 * np.pi / n_phi
    a = np.arange(n_band)[:, None, None, None]
    b = np.arange(n_phi)[None, :, None, None]
    th = theta0 + (a + 0.5) * dtheta + 0.5 * dtheta * t[None, None, :, None] + 0 * b
    ph = (b + 0.5) * dph + 0.5 * dph * t[None, None, None, :] + 0 * a
    th, ph = np.broadcast_arrays(th, ph)
    rho = R + r * np.cos(ph)
    x = _torus_point(th, ph, R, r)
    yu = np.stack([-rho * np.sin(th), rho * np.cos(th), 0 * th], -1) * (0.5 * dtheta)
    yv = np.stack([-r * np.sin(ph) * np.cos(th), -r * np.sin(ph) * np.sin(th),
                   r * np.cos(ph)], -1) * (0.5 * dph)
    nrm = np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)], -1)
    H = (R + 2 * r * np.cos(ph)) / (2 * r * rho)
    kg = np.cos(ph) / (r * rho)
    jac = np.linalg.norm(np.cross(yu, yv), axis=-1)
    w = wt[:, None] * wt[None, :] * jac
    npatch = n_band * n_phi
    N = npatch * p * p
    surf = Surface(
        kind="torus_band", npatch=npatch, p=p,
        nodes=x.reshape(N, 3), normals=nrm.reshape(N, 3),
        tangents=np.concatenate([yu, yv], -1).reshape(N, 6),
        curvature=H.reshape(N), weights=w.reshape(N), gauss_curvature=kg.reshape(N),
        params={"theta": th.reshape(N), "phi": ph.reshape(N), "R": R, "r": r,
                "theta0": theta0, "theta1": theta0 + n_band * dtheta, "n_band": n_band,
                "n_phi": n_phi},
        area=n_band * dtheta * 2 * np.pi * R * r, genus=0)
    curves = [_curve(theta0, -1.0, M, F, R, r), _curve(theta0 + n_band * dtheta, 1.0, M, F, R, r)]
    return OpenSurface(surface=surf, curves=curves, R=R, r=r)


def ambient_a(x):
    """a(x) = exp(A_GRAD . x) and its ambient gradient."""
    a = np.exp(x @ A_GRAD)
    return a, a[:, None] * A_GRAD[None, :]


def band_coefficient(osurf: OpenSurface) -> Coefficient:
    s = osurf.surface
    a, g = ambient_a(s.nodes)
    n = s.normals
    return Coefficient("exp_ambient", a, g - n * np.sum(g * n, 1, keepdims=True))


def edge_a(osurf: OpenSurface, oversampled: bool = False) -> np.ndarray:
    """a at the edge nodes (or the oversampled points) of all curves, curve by curve."""
    return np.concatenate([ambient_a(c.xo if oversampled else c.x)[0] for c in osurf.curves])


def newtonian_neumann(osurf: OpenSurface, coeff: Coefficient, x0=(-3.0, -3.0, 4.0)):
    """(f [N], f_gamma [M total], v at the nodes [N]) for u = v = -1/|x - x0|."""
    s = osurf.surface
    x0 = np.asarray(x0, dtype=np.float64)
    d = s.nodes - x0
    rho = np.linalg.norm(d, axis=1)
    v = -1.0 / rho
    grad = d / rho[:, None] ** 3
    n = s.normals
    dn = np.sum(grad * n, 1)
    dnn = 1.0 / rho ** 3 - 3.0 * np.sum(d * n, 1) ** 2 / rho ** 5
    lap_g = -2.0 * s.curvature * dn - dnn
    grad_g = grad - n * dn[:, None]
    f = np.sum(coeff.grad_a * grad_g, 1) + coeff.a * lap_g
    fg = []
    for c in osurf.curves:
        de = c.x - x0
        re = np.linalg.norm(de, axis=1)
        fg.append(np.sum(c.nu * de, 1) / re ** 3)
    return f, np.concatenate(fg), v


def edge_patches(osurf: OpenSurface):
    """(patch [Me], (u, v) [Me, 2]): the patch whose outer edge holds each edge node and the
    node's reference coordinates there (u = -1 on the first circle, +1 on the second)."""
    s = osurf.surface
    nb, nphi = s.params["n_band"], s.params["n_phi"]
    dph = 2 * np.pi / nphi
    patch, uv = [], []
    for ci, c in enumerate(osurf.curves):
        b = np.floor(c.t / dph).astype(int)
        v0 = (c.t - (b + 0.5) * dph) / (0.5 * dph)
        a = 0 if ci == 0 else nb - 1
        patch.append(a * nphi + b)
        uv.append(np.stack([np.full(c.M, -1.0 if ci == 0 else 1.0), v0], 1))
    return np.concatenate(patch).astype(np.int32), np.concatenate(uv)


def constant_band_coefficient(osurf: OpenSurface, value: float = 1.0) -> Coefficient:
    s = osurf.surface
    return Coefficient("constant", np.full(s.N, float(value)), np.zeros((s.N, 3)))


def newtonian_dirichlet(osurf: OpenSurface, value: float = 1.0, x0=(-3.0, -3.0, 4.0)):
    """(f [N], f_gamma [M total], v at the nodes [N]) for u = v = -1/|x - x0| and the
    constant coefficient a = value: f = a Lap_Gamma v, f_gamma = v on gamma."""
    s = osurf.surface
    x0 = np.asarray(x0, dtype=np.float64)
    d = s.nodes - x0
    rho = np.linalg.norm(d, axis=1)
    v = -1.0 / rho
    grad = d / rho[:, None] ** 3
    n = s.normals
    dn = np.sum(grad * n, 1)
    dnn = 1.0 / rho ** 3 - 3.0 * np.sum(d * n, 1) ** 2 / rho ** 5
    f = value * (-2.0 * s.curvature * dn - dnn)
    fg = np.concatenate([-1.0 / np.linalg.norm(c.x - x0, axis=1) for c in osurf.curves])
    return f, fg, v
