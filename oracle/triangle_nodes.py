"""Triangle-patch operators on node-interpolated geometry (Sec. 6.1, 6.1.2), c = 0.

TEST INFRASTRUCTURE ONLY (see the package docstring).

triangle_operator.TriDiscretization integrates over each patch's exact map
y_P(u, v).  A surface handed over as node data (positions, tangents, weights at
the order-p nodes of T0) has no map; its patch is the interpolant of the nodes,
the triangle analogue of patch.PatchInterpolant for quads:

    y~(u, v) = sum_k X_k l_k(u, v),    J~(u, v) = sum_k J_k l_k(u, v),

with l_k = sum_n U_nk K_n the Lagrange basis of the nodes (Koornwinder basis K_n,
U the inverse of the Vandermonde matrix V_jn = K_n(u_j, v_j), Sec. 6.1.2 with
reading 27) and J_k = |y_u x y_v| from the given tangents.  The rules are those
of TriDiscretization (polar self rule about the target's node, adaptive
subdivision of T0 for near patches, strict 1.5-radius near test); as for quads
(reading 11), the self rule's curvature terms use the interpolated patch's own
unit normal at the target, (y~_u x y~_v)/|.|, and x - y~ is formed from the
node offsets X_k - x so that it keeps its precision as y~ -> x.  Near patches
use the given normal.
"""

from __future__ import annotations

import numpy as np

from .kernels import parametrix_scaled, remainder_scaled
from .triangle import koornwinder, koornwinder_grad
from .triangle_operator import TriDiscretization, polar_rule


class TriNodeDiscretization(TriDiscretization):
    """Triangle patches given by node data: ref_u, ref_v [nt] (the rule's nodes on T0,
    the same for every patch), nodes/normals [N, 3], tangents [N, 6] (y_u, y_v),
    curvature [N], weights [N]; node k of patch P is row P * nt + k."""

    def __init__(self, ref_u, ref_v, nodes, normals, tangents, curvature, weights, npatch, p,
                 a=None, grad_a=None, near_tol=1e-13):
        self.npatch, self.p = int(npatch), int(p)
        self.dtype = np.float64
        self.c = None
        self.b = None
        self.tu = np.asarray(ref_u, dtype=np.float64)
        self.tv = np.asarray(ref_v, dtype=np.float64)
        self.pp = len(self.tu)
        self.N = self.npatch * self.pp
        self.U = np.linalg.inv(koornwinder(self.p - 1, self.tu, self.tv).T)
        self.x = np.asarray(nodes, dtype=np.float64).reshape(self.N, 3)
        self.n = np.asarray(normals, dtype=np.float64).reshape(self.N, 3)
        tg = np.asarray(tangents, dtype=np.float64).reshape(self.N, 6)
        self.J = np.linalg.norm(np.cross(tg[:, :3], tg[:, 3:]), axis=1)
        self.H = np.asarray(curvature, dtype=np.float64)
        self.w = np.asarray(weights, dtype=np.float64)
        self.a = np.ones(self.N) if a is None else np.asarray(a, dtype=np.float64)
        self.g = np.zeros((self.N, 3)) if grad_a is None else np.asarray(grad_a, dtype=np.float64)
        self.X = self.x.reshape(self.npatch, self.pp, 3)
        self.Jn = self.J.reshape(self.npatch, self.pp)
        L0 = self.lagrange(np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]))
        corners = np.einsum("kq,Pkc->Pqc", L0, self.X)          # [npatch, 3 vertices, 3]
        self.centroid = corners.mean(axis=1)
        self.radius = np.max(np.linalg.norm(corners - self.centroid[:, None, :], axis=2), axis=1)
        self.near_tol = near_tol

    @classmethod
    def from_surface(cls, surf, a=None, grad_a=None, **kw):
        return cls(surf.ref_u, surf.ref_v, surf.nodes, surf.normals, surf.tangents,
                   surf.curvature, surf.weights, surf.npatch, surf.p, a=a, grad_a=grad_a, **kw)

    def normal_at(self, P, u0, v0):
        """Unit normal (y~_u x y~_v)/|.| of patch P's interpolant at (u0, v0)."""
        du, dv = koornwinder_grad(self.p - 1, np.array([u0]), np.array([v0]))
        yu = (self.U.T @ du)[:, 0] @ self.X[P]
        yv = (self.U.T @ dv)[:, 0] @ self.X[P]
        c = np.cross(yu, yv)
        return c / np.linalg.norm(c)

    def _integrand(self, i, P, u, v, w, normal=None):
        """(sum_q w_q J~ a(y)R l_k, same for K) over points (u, v) of patch P; x_i - y~
        from the node offsets; `normal` replaces the target's given normal."""
        L = self.lagrange(u, v)                                  # [nt, Q]
        r = -(L.T @ (self.X[P] - self.x[i]))                     # x_i - y~ [Q, 3]
        J = L.T @ self.Jn[P]
        n = self.n[i] if normal is None else normal
        zero = np.zeros(3)
        fr = w * J * remainder_scaled(zero, n, self.H[i], self.a[i], self.g[i], -r)
        fk = w * J * parametrix_scaled(zero, -r)
        return np.stack([L @ fr, L @ fk])

    def self_weights(self, i):
        loc, P = i % self.pp, i // self.pp
        u0, v0 = float(self.tu[loc]), float(self.tv[loc])
        u, v, w = polar_rule(u0, v0)
        return self._integrand(i, P, u, v, w, normal=self.normal_at(P, u0, v0))
