"""Tensor Lagrange interpolation on one quadrilateral patch.

A patch carries data at the p x p tensor Gauss-Legendre nodes (u_a, v_b) of
[-1, 1]^2.  Sec. 6.1.1 (remark) and 6.1.2 interpolate the density from the
discretisation nodes to the quadrature points; on quads the interpolant is the
tensor product of 1-D Lagrange polynomials on the Gauss nodes,
f~(u, v) = sum_ab f_ab l_a(u) l_b(v).  The same interpolant gives the patch
geometry from the node positions (y~) and the surface element from the nodal
values J = |y_u x y_v| (J~): the reference patch map itself is not an input.
"""

from __future__ import annotations

import numpy as np
from numpy.polynomial.legendre import leggauss


def lagrange_basis(nodes: np.ndarray, s: np.ndarray) -> np.ndarray:
    """l_a(s) for all a: product formula prod_{b != a} (s - t_b)/(t_a - t_b).

    Returns an array of shape s.shape + (p,).
    """
    s = np.asarray(s, dtype=np.float64)
    p = len(nodes)
    diff = s[..., None] - nodes                      # s - t_b
    out = np.empty(s.shape + (p,))
    for a in range(p):
        others = np.arange(p) != a
        out[..., a] = np.prod(diff[..., others] / (nodes[a] - nodes[others]), axis=-1)
    return out


def lagrange_basis_derivative(nodes: np.ndarray, s: np.ndarray) -> np.ndarray:
    """l_a'(s) by the product rule: sum_{m != a} 1/(t_a - t_m) prod_{b != a, m} (s - t_b)/(t_a - t_b)."""
    s = np.asarray(s, dtype=np.float64)
    p = len(nodes)
    out = np.zeros(s.shape + (p,))
    for a in range(p):
        for m in range(p):
            if m == a:
                continue
            term = np.full(s.shape, 1.0 / (nodes[a] - nodes[m]))
            for b in range(p):
                if b != a and b != m:
                    term = term * (s - nodes[b]) / (nodes[a] - nodes[b])
            out[..., a] += term
    return out


class PatchInterpolant:
    """Interpolated geometry of one patch: positions y~(u, v) and element J~(u, v)."""

    def __init__(self, X: np.ndarray, J: np.ndarray):
        # X: [p, p, 3] node positions (i along u, j along v); J: [p, p]
        self.p = X.shape[0]
        self.t, self.wt = leggauss(self.p)
        self.X = np.asarray(X, dtype=np.float64)
        self.J = np.asarray(J, dtype=np.float64)

    def basis(self, u, v):
        return lagrange_basis(self.t, u), lagrange_basis(self.t, v)

    def evaluate(self, u, v):
        """y~ [Q, 3], J~ [Q], and the basis values l_a(u) [Q, p], l_b(v) [Q, p]
        at the points (u[q], v[q]) (1-D arrays of equal length)."""
        Lu, Lv = self.basis(np.ravel(u), np.ravel(v))
        p = self.p
        y = np.sum((Lu @ self.X.reshape(p, 3 * p)).reshape(-1, p, 3) * Lv[:, :, None], axis=1)
        J = np.sum((Lu @ self.J) * Lv, axis=1)
        return y, J, Lu, Lv

    def offsets(self, u, v, x):
        """y~(u, v) - x as the interpolant of the node offsets X_ab - x.

        Equal to evaluate(u, v)[0] - x in exact arithmetic (the tensor basis
        sums to one); formed this way it keeps full relative precision as
        (u, v) approaches a node at x, where the plain difference of two
        O(1) positions would lose n.(y - x) = O(|y - x|^2) to rounding.
        """
        Lu, Lv = self.basis(np.ravel(u), np.ravel(v))
        p = self.p
        D = (self.X - x).reshape(p, 3 * p)
        return np.sum((Lu @ D).reshape(-1, p, 3) * Lv[:, :, None], axis=1)

    def normal_at(self, u0, v0):
        """Unit normal of the interpolated patch, (y~_u x y~_v)/|y~_u x y~_v|, at (u0, v0)."""
        Lu, Lv = lagrange_basis(self.t, u0), lagrange_basis(self.t, v0)
        dLu = lagrange_basis_derivative(self.t, u0)
        dLv = lagrange_basis_derivative(self.t, v0)
        yu = np.einsum("a,abc,b->c", dLu, self.X, Lv)
        yv = np.einsum("a,abc,b->c", Lu, self.X, dLv)
        c = np.cross(yu, yv)
        return c / np.linalg.norm(c)

    def corners(self):
        """Images of the four corners (+-1, +-1) of the reference square."""
        cu = np.array([1.0, -1.0, -1.0, 1.0])
        cv = np.array([1.0, 1.0, -1.0, -1.0])
        y, _, _, _ = self.evaluate(cu, cv)
        return y

    def centroid_radius(self):
        """Sec. 6.1.2 'near' data: centroid = mean of the vertex images, radius =
        largest vertex distance from it (read for quads: the 4 corner images)."""
        c = self.corners()
        ctr = c.mean(axis=0)
        return ctr, float(np.max(np.linalg.norm(c - ctr, axis=1)))
