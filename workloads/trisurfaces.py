"""Closed test surfaces as curved triangle patches over the simplex T0.

``tri_ellipsoid(level, p, axes)``: those patches mapped to an ellipsoid and
sampled at the order-p Vioreanu-Rokhlin nodes (``TriSurface``, the input of the
library's triangle surfaces and of the oracle's node-interpolated operators).

``icosphere(level)``: the unit sphere as the radial projection of the
icosahedron's faces, each split ``4**level`` ways by edge midpoints.  Patch P
is the map y_P(u, v) = q / |q|, q = A + u (B - A) + v (C - A) of T0 onto the
sphere (A, B, C the flat triangle's vertices, ordered so that the normal
y_u x y_v points outward), with the closed-form derivatives
y_u = (e1 - y (y . e1)) / |q|, e1 = B - A, and likewise y_v with e2 = C - A.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    V = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    return [V[list(f)] for f in F]


def _split(tri):
    a, b, c = tri
    ab, bc, ca = 0.5 * (a + b), 0.5 * (b + c), 0.5 * (c + a)
    return [np.array(t) for t in ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca))]


class SphereTriangles:
    """Patch maps of the projected triangles (picklable, for worker processes)."""

    def __init__(self, flat):
        self.flat = flat

    def __call__(self, P, u, v):
        a, e1, e2 = self.flat[P]
        u = np.atleast_1d(np.asarray(u, dtype=np.float64))
        v = np.atleast_1d(np.asarray(v, dtype=np.float64))
        q = a + u[:, None] * e1 + v[:, None] * e2
        rq = np.linalg.norm(q, axis=1, keepdims=True)
        y = q / rq
        yu = (e1 - y * (y @ e1)[:, None]) / rq
        yv = (e2 - y * (y @ e2)[:, None]) / rq
        return y, yu, yv


def icosphere(level: int = 0):
    """(npatch, ymap) with ymap(P, u, v) -> (y, y_u, y_v), each [len(u), 3]."""
    tris = _icosahedron()
    for _ in range(level):
        tris = [t for tri in tris for t in _split(tri)]
    flat = []
    for a, b, c in tris:
        if np.dot(np.cross(b - a, c - a), a + b + c) < 0:
            b, c = c, b
        flat.append((a, b - a, c - a))
    return len(flat), SphereTriangles(flat)


@dataclass
class TriSurface:
    """A closed surface sampled on curved triangle patches at the nodes of an
    order-p rule on T0: node positions, outward unit normals, tangents
    (y_u, y_v) [N, 6], mean curvature, smooth-rule weights w = w_ref J and the
    reference nodes (ref_u, ref_v) of the rule (the same for every patch)."""
    kind: str
    npatch: int
    p: int
    ref_u: np.ndarray
    ref_v: np.ndarray
    ref_w: np.ndarray
    nodes: np.ndarray
    normals: np.ndarray
    tangents: np.ndarray
    curvature: np.ndarray
    weights: np.ndarray
    area: float | None = None

    @property
    def nt(self) -> int:
        return len(self.ref_u)

    @property
    def N(self) -> int:
        return self.npatch * self.nt


def tri_ellipsoid(level: int, p: int, axes=(1.0, 1.0, 1.0)) -> TriSurface:
    """The icosphere's triangles mapped to the ellipsoid with semi-axes ``axes``:
    y_P(u, v) = D q / |q| (D = diag(axes)), sampled at the Vioreanu-Rokhlin nodes of
    order p (workloads.trirule).  axes = (1, 1, 1) is the unit sphere (H = 1)."""
    from .surfaces import _level_set_curvatures
    from .trirule import vioreanu_rokhlin_rule
    npatch, ymap = icosphere(level)
    u, v, w = vioreanu_rokhlin_rule(p)
    D = np.asarray(axes, dtype=np.float64)
    X, T, Nn, W = [], [], [], []
    for P in range(npatch):
        y, yu, yv = ymap(P, u, v)              # on the unit sphere
        y, yu, yv = y * D, yu * D, yv * D
        c = np.cross(yu, yv)
        J = np.linalg.norm(c, axis=1)
        X.append(y)
        T.append(np.hstack([yu, yv]))
        Nn.append(c / J[:, None])
        W.append(w * J)
    x = np.concatenate(X)
    if np.allclose(D, 1.0):
        H = np.ones(len(x))
        area = 4 * np.pi
    else:
        H = _level_set_curvatures(x, tuple(D))[0]
        area = None
    kind = "tri_sphere" if area is not None else "tri_ellipsoid"
    return TriSurface(kind=kind, npatch=npatch, p=p, ref_u=u, ref_v=v, ref_w=w, nodes=x,
                      normals=np.concatenate(Nn), tangents=np.concatenate(T), curvature=H,
                      weights=np.concatenate(W), area=area)
