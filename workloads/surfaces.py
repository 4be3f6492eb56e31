"""Closed test surfaces sampled at tensor Gauss-Legendre nodes on quad patches.

Every surface is a union of ``npatch`` quadrilateral patches, each the image
of the reference square [-1,1]^2 under an analytic map y(u, v).  Each patch
carries p x p nodes at the tensor product of the ascending p-point
Gauss-Legendre nodes; node ``i*p + j`` of patch ``P`` (global index
``P*p*p + i*p + j``) sits at (u_i, v_j), i along u and j along v.

Per node the surface provides the quantities a caller hands to
``pm_surface_create``:

* ``nodes``     y(u_i, v_j)                                  [N, 3]
* ``normals``   outward unit normal                          [N, 3]
* ``tangents``  (dy/du, dy/dv) on the reference square        [N, 6]
* ``curvature`` mean curvature H = (1/2) div_Gamma n          [N]
  (outward normal, so H = 1/R on a sphere of radius R)
* ``weights``   w = omega_i omega_j |y_u x y_v|               [N]
  (the smooth tensor Gauss rule for the surface element)

All geometric quantities come from closed forms (analytic derivatives and
level-set curvature formulas), in float64.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from numpy.polynomial.legendre import leggauss


def gauss_legendre(p: int):
    """Ascending p-point Gauss-Legendre nodes and weights on [-1, 1]."""
    t, w = leggauss(p)
    return np.asarray(t, dtype=np.float64), np.asarray(w, dtype=np.float64)


@dataclass
class Surface:
    kind: str
    npatch: int
    p: int
    nodes: np.ndarray
    normals: np.ndarray
    tangents: np.ndarray
    curvature: np.ndarray
    weights: np.ndarray
    gauss_curvature: np.ndarray
    params: dict = field(default_factory=dict)
    area: float | None = None
    volume: float | None = None
    genus: int = 0

    @property
    def N(self) -> int:
        return self.npatch * self.p * self.p

    def scaled(self, s: float) -> "Surface":
        """The dilated surface s*Gamma (same parametrisation, scaled)."""
        return Surface(
            kind=self.kind + f"*{s:g}", npatch=self.npatch, p=self.p,
            nodes=self.nodes * s, normals=self.normals.copy(),
            tangents=self.tangents * s, curvature=self.curvature / s,
            weights=self.weights * s * s,
            gauss_curvature=self.gauss_curvature / (s * s),
            params=dict(self.params),
            area=None if self.area is None else self.area * s * s,
            volume=None if self.volume is None else self.volume * s ** 3,
            genus=self.genus)


# Cube faces as (centre direction c0, e1, e2) with e1 x e2 = c0, so that the
# map (xi, eta) -> c0 + tan(xi) e1 + tan(eta) e2 is orientation preserving and
# y_u x y_v points outward.
_FACES = (
    ((1, 0, 0), (0, 1, 0), (0, 0, 1)),
    ((-1, 0, 0), (0, 0, 1), (0, 1, 0)),
    ((0, 1, 0), (0, 0, 1), (1, 0, 0)),
    ((0, -1, 0), (1, 0, 0), (0, 0, 1)),
    ((0, 0, 1), (1, 0, 0), (0, 1, 0)),
    ((0, 0, -1), (0, 1, 0), (1, 0, 0)),
)


def _level_set_curvatures(x, axes):
    """Mean and Gauss curvature of sum_i x_i^2/a_i^2 = 1 at points x [.., 3]."""
    a2 = np.asarray(axes, dtype=np.float64) ** 2
    g = 2.0 * x / a2                      # gradient of the level-set function
    gn = np.linalg.norm(g, axis=-1)
    hess = 2.0 / a2                       # diagonal Hessian
    div_n = (hess.sum() * gn ** 2 - np.sum(g * g * hess, axis=-1)) / gn ** 3
    H = 0.5 * div_n
    a, b, c = axes
    kg = 1.0 / (a * a * b * b * c * c * np.sum(x * x / a2 ** 2, axis=-1) ** 2)
    return H, kg


def _cubed_sphere_directions(m: int, p: int):
    """Unit-sphere points and their (xi, eta) derivatives for all patches.

    Equiangular gnomonic cubed sphere: each face is split into m x m patches
    in (xi, eta) in [-pi/4, pi/4]^2.  Returns ys [P,p,p,3], dys/du, dys/dv
    (derivatives with respect to the patch coordinates u, v in [-1, 1]) and
    the face/patch parameters.
    """
    t, _ = gauss_legendre(p)
    half = np.pi / 4
    d = 2 * half / m
    ys_l, du_l, dv_l, face_l, xi_l, eta_l = [], [], [], [], [], []
    for f, (c0, e1, e2) in enumerate(_FACES):
        c0, e1, e2 = (np.asarray(v, dtype=np.float64) for v in (c0, e1, e2))
        for a in range(m):
            for b in range(m):
                xi = -half + (a + 0.5) * d + 0.5 * d * t[:, None] + 0 * t[None, :]
                eta = -half + (b + 0.5) * d + 0 * t[:, None] + 0.5 * d * t[None, :]
                tx, te = np.tan(xi), np.tan(eta)
                c = c0 + tx[..., None] * e1 + te[..., None] * e2
                cn = np.linalg.norm(c, axis=-1)[..., None]
                ys = c / cn
                dc_dxi = (1.0 / np.cos(xi) ** 2)[..., None] * e1
                dc_deta = (1.0 / np.cos(eta) ** 2)[..., None] * e2
                dys_dxi = (dc_dxi - ys * np.sum(ys * dc_dxi, -1, keepdims=True)) / cn
                dys_deta = (dc_deta - ys * np.sum(ys * dc_deta, -1, keepdims=True)) / cn
                ys_l.append(ys)
                du_l.append(dys_dxi * (0.5 * d))
                dv_l.append(dys_deta * (0.5 * d))
                face_l.append(np.full((p, p), f))
                xi_l.append(xi)
                eta_l.append(eta)
    return (np.stack(ys_l), np.stack(du_l), np.stack(dv_l),
            np.stack(face_l), np.stack(xi_l), np.stack(eta_l))


def cubed_sphere(m: int, p: int, axes=(1.0, 1.0, 1.0)) -> Surface:
    """Sphere (axes all 1) or ellipsoid x^2/a^2 + y^2/b^2 + z^2/c^2 = 1.

    The ellipsoid is the image of the unit cubed sphere under diag(axes);
    6 m^2 patches with p x p Gauss-Legendre nodes each.
    """
    ys, dys_du, dys_dv, face, xi, eta = _cubed_sphere_directions(m, p)
    D = np.asarray(axes, dtype=np.float64)
    x = ys * D
    yu = dys_du * D
    yv = dys_dv * D
    nrm = ys / D
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    H, kg = _level_set_curvatures(x, D)
    _, wt = gauss_legendre(p)
    jac = np.linalg.norm(np.cross(yu, yv), axis=-1)
    w = wt[None, :, None] * wt[None, None, :] * jac
    npatch = 6 * m * m
    N = npatch * p * p
    sphere = bool(np.all(D == D[0]))
    kind = "sphere" if sphere else "ellipsoid"
    area = 4 * np.pi * D[0] ** 2 if sphere else None
    return Surface(
        kind=kind, npatch=npatch, p=p,
        nodes=x.reshape(N, 3), normals=nrm.reshape(N, 3),
        tangents=np.concatenate([yu, yv], axis=-1).reshape(N, 6),
        curvature=H.reshape(N), weights=w.reshape(N),
        gauss_curvature=kg.reshape(N),
        params={"face": face.reshape(N), "xi": xi.reshape(N), "eta": eta.reshape(N),
                "axes": tuple(float(v) for v in D)},
        area=area, volume=4.0 / 3.0 * np.pi * float(np.prod(D)), genus=0)


def torus(n_theta: int, n_phi: int, p: int, R: float = 2.0, r: float = 0.7) -> Surface:
    """Torus ((R + r cos phi) cos theta, (R + r cos phi) sin theta, r sin phi).

    theta (toroidal, n_theta patches) runs along u and phi (poloidal,
    n_phi patches) along v; patch index = a * n_phi + b.
    """
    t, wt = gauss_legendre(p)
    dth = 2 * np.pi / n_theta
    dph = 2 * np.pi / n_phi
    a = np.arange(n_theta)[:, None, None, None]
    b = np.arange(n_phi)[None, :, None, None]
    th = (a + 0.5) * dth + 0.5 * dth * t[None, None, :, None] + 0 * b
    ph = (b + 0.5) * dph + 0.5 * dph * t[None, None, None, :] + 0 * a
    th, ph = np.broadcast_arrays(th, ph)
    rho = R + r * np.cos(ph)
    x = np.stack([rho * np.cos(th), rho * np.sin(th), r * np.sin(ph)], -1)
    yu = np.stack([-rho * np.sin(th), rho * np.cos(th), 0 * th], -1) * (0.5 * dth)
    yv = np.stack([-r * np.sin(ph) * np.cos(th), -r * np.sin(ph) * np.sin(th),
                   r * np.cos(ph)], -1) * (0.5 * dph)
    nrm = np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)], -1)
    H = (R + 2 * r * np.cos(ph)) / (2 * r * rho)
    kg = np.cos(ph) / (r * rho)
    jac = np.linalg.norm(np.cross(yu, yv), axis=-1)
    w = wt[:, None] * wt[None, :] * jac
    npatch = n_theta * n_phi
    N = npatch * p * p
    return Surface(
        kind="torus", npatch=npatch, p=p,
        nodes=x.reshape(N, 3), normals=nrm.reshape(N, 3),
        tangents=np.concatenate([yu, yv], -1).reshape(N, 6),
        curvature=H.reshape(N), weights=w.reshape(N), gauss_curvature=kg.reshape(N),
        params={"theta": th.reshape(N), "phi": ph.reshape(N), "R": R, "r": r},
        area=4 * np.pi ** 2 * R * r, volume=2 * np.pi ** 2 * R * r * r, genus=1)


def star_surface(m: int, p: int, amp: float = 0.3) -> Surface:
    """Star-shaped surface x = rho(theta, phi) e_r over the cubed-sphere directions.

    rho = 1 + amp sin(3 theta) cos(2 phi), theta the polar angle and phi the
    azimuth of the direction.  Taken literally, rho is Lipschitz but not
    differentiable at the two poles (sin 3 theta ~ 3 theta there); the poles sit
    at patch corners of the cubed sphere, so no node lies on them.  Positions,
    tangents (chain rule through the cubed-sphere map), the normal and the mean
    curvature come from closed-form first and second derivatives in (theta, phi).
    """
    ys, dys_du, dys_dv, face, xi, eta = _cubed_sphere_directions(m, p)
    P = ys.shape[0]
    d = ys.reshape(-1, 3)
    du = dys_du.reshape(-1, 3)
    dv = dys_dv.reshape(-1, 3)
    th = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    ph = np.arctan2(d[:, 1], d[:, 0])
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    rho = 1 + amp * np.sin(3 * th) * np.cos(2 * ph)
    r_t = 3 * amp * np.cos(3 * th) * np.cos(2 * ph)
    r_p = -2 * amp * np.sin(3 * th) * np.sin(2 * ph)
    r_tt = -9 * amp * np.sin(3 * th) * np.cos(2 * ph)
    r_tp = -6 * amp * np.cos(3 * th) * np.sin(2 * ph)
    r_pp = -4 * amp * np.sin(3 * th) * np.cos(2 * ph)
    er = np.stack([st * cp, st * sp, ct], -1)
    et = np.stack([ct * cp, ct * sp, -st], -1)
    ep = np.stack([-sp, cp, np.zeros_like(ph)], -1)
    # parametrisation in (theta, phi)
    X = rho[:, None] * er
    X_t = r_t[:, None] * er + rho[:, None] * et
    X_p = r_p[:, None] * er + (rho * st)[:, None] * ep
    # second derivatives (d er/dt = et, d er/dp = st ep, d et/dt = -er, d et/dp = ct ep,
    # d ep/dp = -(st er + ct et))
    X_tt = r_tt[:, None] * er + 2 * r_t[:, None] * et - rho[:, None] * er
    X_tp = (r_tp[:, None] * er + r_t[:, None] * st[:, None] * ep + r_p[:, None] * et
            + (rho * ct)[:, None] * ep)
    X_pp = (r_pp[:, None] * er + 2 * (r_p * st)[:, None] * ep
            - (rho * st)[:, None] * (st[:, None] * er + ct[:, None] * et))
    nrm = np.cross(X_t, X_p)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    out = np.sum(nrm * er, 1) < 0
    nrm[out] *= -1.0
    E, F, G = np.sum(X_t * X_t, 1), np.sum(X_t * X_p, 1), np.sum(X_p * X_p, 1)
    e, f, g = np.sum(X_tt * nrm, 1), np.sum(X_tp * nrm, 1), np.sum(X_pp * nrm, 1)
    H = -(e * G - 2 * f * F + g * E) / (2 * (E * G - F * F))
    KG = (e * g - f * f) / (E * G - F * F)
    # tangents with respect to the patch coordinates: chain rule through theta(d), phi(d)
    th_u = -du[:, 2] / st
    th_v = -dv[:, 2] / st
    rxy2 = d[:, 0] ** 2 + d[:, 1] ** 2
    ph_u = (d[:, 0] * du[:, 1] - d[:, 1] * du[:, 0]) / rxy2
    ph_v = (d[:, 0] * dv[:, 1] - d[:, 1] * dv[:, 0]) / rxy2
    yu = X_t * th_u[:, None] + X_p * ph_u[:, None]
    yv = X_t * th_v[:, None] + X_p * ph_v[:, None]
    # orient normals like y_u x y_v (outward on the cubed sphere)
    _, wt = gauss_legendre(p)
    jac = np.linalg.norm(np.cross(yu, yv), axis=1)
    w = (wt[:, None] * wt[None, :]).ravel()
    w = np.tile(w, P) * jac
    N = P * p * p
    return Surface(kind="star", npatch=P, p=p, nodes=X, normals=nrm,
                   tangents=np.concatenate([yu, yv], -1), curvature=H, weights=w,
                   gauss_curvature=KG, params={"theta": th, "phi": ph, "amp": amp},
                   area=None, volume=None, genus=0)


def wavy_torus(n_u: int, n_v: int, p: int, amp: float = 0.6) -> Surface:
    """The paper's wavy torus (Sec. 7): r(u, v) = (rho cos u, rho sin u, sin v),
    rho = 3 + cos v + amp cos 5u (amp = 0.6), (u, v) in [0, 2 pi)^2.

    u (n_u patches) and v (n_v patches) run along the patch coordinates as in
    ``torus``; tangents, the outward normal r_u x r_v / |r_u x r_v| and the mean
    and Gauss curvatures come from the closed-form first and second derivatives.
    Each half-plane at angle u cuts a unit disk centred at radius 3 + 0.6 cos 5u,
    so the enclosed volume is the integral of pi (3 + amp cos 5u) du = 6 pi^2.
    """
    t, wt = gauss_legendre(p)
    du_p = 2 * np.pi / n_u
    dv_p = 2 * np.pi / n_v
    a = np.arange(n_u)[:, None, None, None]
    b = np.arange(n_v)[None, :, None, None]
    u = (a + 0.5) * du_p + 0.5 * du_p * t[None, None, :, None] + 0 * b
    v = (b + 0.5) * dv_p + 0.5 * dv_p * t[None, None, None, :] + 0 * a
    u, v = np.broadcast_arrays(u, v)
    cu, su, cv, sv = np.cos(u), np.sin(u), np.cos(v), np.sin(v)
    rho = 3 + cv + amp * np.cos(5 * u)
    rho_u = -5.0 * amp * np.sin(5 * u)
    rho_uu = -25.0 * amp * np.cos(5 * u)
    rho_v, rho_vv = -sv, -cv
    z0 = 0 * u
    X = np.stack([rho * cu, rho * su, sv], -1)
    X_u = np.stack([rho_u * cu - rho * su, rho_u * su + rho * cu, z0], -1)
    X_v = np.stack([rho_v * cu, rho_v * su, cv], -1)
    X_uu = np.stack([rho_uu * cu - 2 * rho_u * su - rho * cu,
                     rho_uu * su + 2 * rho_u * cu - rho * su, z0], -1)
    X_uv = np.stack([-rho_v * su, rho_v * cu, z0], -1)
    X_vv = np.stack([rho_vv * cu, rho_vv * su, -sv], -1)
    nrm = np.cross(X_u, X_v)
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    E, F, G = (np.sum(X_u * X_u, -1), np.sum(X_u * X_v, -1), np.sum(X_v * X_v, -1))
    e, f, g = (np.sum(X_uu * nrm, -1), np.sum(X_uv * nrm, -1), np.sum(X_vv * nrm, -1))
    H = -(e * G - 2 * f * F + g * E) / (2 * (E * G - F * F))
    KG = (e * g - f * f) / (E * G - F * F)
    yu = X_u * (0.5 * du_p)
    yv = X_v * (0.5 * dv_p)
    jac = np.linalg.norm(np.cross(yu, yv), axis=-1)
    w = wt[:, None] * wt[None, :] * jac
    npatch = n_u * n_v
    N = npatch * p * p
    return Surface(
        kind="wavy_torus", npatch=npatch, p=p,
        nodes=X.reshape(N, 3), normals=nrm.reshape(N, 3),
        tangents=np.concatenate([yu, yv], -1).reshape(N, 6),
        curvature=H.reshape(N), weights=w.reshape(N), gauss_curvature=KG.reshape(N),
        params={"u": u.reshape(N), "v": v.reshape(N)},
        area=None, volume=6 * np.pi ** 2, genus=1)
