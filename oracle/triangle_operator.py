"""Nystrom discretisation on curved triangle patches (Sec. 6.1), c = 0, b = 0.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Each patch is a map y_P(u, v) of the simplex T0 (Sec. 6.1, eq. IEsum), given
here by its parameterisation (with derivatives), and carries the order-p
Vioreanu-Rokhlin nodes of triangle.py.  The discrete operators have the same
"all pairs plus sparse correction" form as the quad version (operator.py):

  (R~ sigma)_i = sum_{j != i} w_j R(x_i, x_j) sigma_j + sum_{near k} C_ik sigma_k,
  w_j = w^VR_j J(u_j, v_j),   C_ik = W_ik / a_k - w_k R(x_i, x_k),  C_ii = W_ii / a_i,

with W_ik = int_P a(y) R(x_i, y_P(u, v)) l_k(u, v) J(u, v) du dv, l_k the
Lagrange basis of the nodes (l_k = sum_n U_nk K_n, Sec. 6.1.2), and likewise
for K.

* Self patch (Sec. 6.1.1, eq. radial_int): polar coordinates about the
  target's (u0, v0); theta split at the directions of the three vertices of T0,
  adaptive Gauss panels on int L(theta)^2 capped at pi/24; radial panels graded
  dyadically toward 0 (16 levels), each at most 0.25 long, 16 points each.
* Near patches (Sec. 6.1.2): adaptive midpoint subdivision of T0 into four
  triangles, a 16 x 16 collapsed Gauss rule on each, splitting while the
  children's sum differs from the parent's by more than tol of the patch's
  weights.
* Near test: as for quads, centroid and radius from the three corner images,
  strict < 1.5 radii.

The normal and curvature at a target come from the parameterisation, so the
self rule needs none of the interpolated-normal care of the quad version.
"""

from __future__ import annotations

from functools import lru_cache

import numpy as np
from numpy.polynomial.legendre import leggauss

from .kernels import parametrix_scaled, remainder_scaled, INV_2PI, INV_PI
from .triangle import collapsed_rule, interpolation_matrix, koornwinder, vioreanu_rokhlin

_T16, _W16 = leggauss(16)
NEAR_FACTOR = 1.5


def _panel(a, b):
    h = 0.5 * (b - a)
    return a + h * (_T16 + 1.0), h * _W16


def ray_length(u0, v0, theta):
    """Distance from (u0, v0) to the boundary of T0 along direction theta."""
    c, s = np.cos(theta), np.sin(theta)
    big = np.inf
    with np.errstate(divide="ignore", invalid="ignore"):
        lu = np.where(c < 0, -u0 / c, big)
        lv = np.where(s < 0, -v0 / s, big)
        lw = np.where(c + s > 0, (1.0 - u0 - v0) / (c + s), big)
    return np.minimum(np.minimum(lu, lv), lw)


def _theta_panels(u0, v0, tol=1e-14, max_width=np.pi / 24):
    ang = np.sort(np.mod(np.arctan2(np.array([0.0, 0.0, 1.0]) - v0,
                                    np.array([0.0, 1.0, 0.0]) - u0), 2 * np.pi))
    sectors = [(ang[k], ang[k + 1] if k < 2 else ang[0] + 2 * np.pi) for k in range(3)]

    def l2(a, b):
        th, w = _panel(a, b)
        return np.dot(w, ray_length(u0, v0, th) ** 2)

    panels = []

    def split(a, b, whole, depth):
        m = 0.5 * (a + b)
        left, right = l2(a, m), l2(m, b)
        if depth >= 50 or abs(whole - left - right) <= tol:
            panels.append((a, b))
            return
        split(a, m, left, depth + 1)
        split(m, b, right, depth + 1)

    for a, b in sectors:
        split(a, b, l2(a, b), 0)
    out = []
    for a, b in sorted(panels):
        k = max(1, int(np.ceil((b - a) / max_width)))
        e = np.linspace(a, b, k + 1)
        out.extend(zip(e[:-1], e[1:]))
    return out


@lru_cache(maxsize=1024)
def polar_rule(u0, v0, levels=16, h_max=0.25):
    """Points (u, v) and weights (w_theta w_r r) of the self rule about (u0, v0)."""
    us, vs, ws = [], [], []
    for a, b in _theta_panels(u0, v0):
        th, wth = _panel(a, b)
        for t_k, w_k in zip(th, wth):
            L = float(ray_length(u0, v0, t_k))
            br = [0.0] + [L * 2.0 ** (-k) for k in range(levels, -1, -1)]
            edges = [0.0]
            for lo, hi in zip(br[:-1], br[1:]):
                k = max(1, int(np.ceil((hi - lo) / h_max)))
                edges.extend(list(np.linspace(lo, hi, k + 1)[1:]))
            edges = np.array(edges)
            ra, rb = edges[:-1, None], edges[1:, None]
            r = (ra + 0.5 * (rb - ra) * (_T16 + 1.0)).ravel()
            wr = (0.5 * (rb - ra) * _W16).ravel()
            us.append(u0 + r * np.cos(t_k))
            vs.append(v0 + r * np.sin(t_k))
            ws.append(w_k * wr * r)
    return np.concatenate(us), np.concatenate(vs), np.concatenate(ws)


class TriDiscretization:
    """Curved triangles given by maps ymap(P, u, v) -> (y, y_u, y_v), order-p VR nodes."""

    def __init__(self, ymap, npatch, p, a_fn=None, grad_a_fn=None, curvature_fn=None,
                 near_tol=1e-13):
        self.ymap, self.npatch, self.p = ymap, int(npatch), int(p)
        self.dtype = np.float64
        self.c = None                       # c = 0, b = 0 on triangles (solve.py reads these)
        self.b = None
        self.tu, self.tv, self.tw = vioreanu_rokhlin(self.p)
        self.pp = len(self.tu)
        self.N = self.npatch * self.pp
        self.U = interpolation_matrix(self.p)
        xs, ns, Js = [], [], []
        for P in range(self.npatch):
            y, yu, yv = ymap(P, self.tu, self.tv)
            c = np.cross(yu, yv)
            J = np.linalg.norm(c, axis=1)
            xs.append(y)
            ns.append(c / J[:, None])
            Js.append(J)
        self.x = np.concatenate(xs)
        self.n = np.concatenate(ns)
        self.J = np.concatenate(Js)
        self.w = np.tile(self.tw, self.npatch) * self.J
        self.H = curvature_fn(self.x) if curvature_fn else np.zeros(self.N)
        self.a = a_fn(self.x) if a_fn else np.ones(self.N)
        self.g = grad_a_fn(self.x, self.n) if grad_a_fn else np.zeros((self.N, 3))
        corners = [ymap(P, np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]))[0]
                   for P in range(self.npatch)]
        self.centroid = np.array([c.mean(axis=0) for c in corners])
        self.radius = np.array([np.max(np.linalg.norm(c - c.mean(axis=0), axis=1))
                                for c in corners])
        self.near_tol = near_tol

    # -------------------------------------------------------------- patch data
    def lagrange(self, u, v):
        """l_k(u, v) for the patch nodes: [pp, len(u)]."""
        return self.U.T @ koornwinder(self.p - 1, u, v)

    def near_patches(self, i):
        d = np.linalg.norm(self.centroid - self.x[i], axis=1)
        own = i // self.pp
        return [own] + sorted(int(P) for P in np.nonzero(d < NEAR_FACTOR * self.radius)[0]
                              if P != own)

    def _integrand(self, i, P, u, v, w):
        """(sum_q w_q J_q a(y)R l_k, same for K) over the points (u, v) of patch P."""
        y, yu, yv = self.ymap(P, u, v)
        J = np.linalg.norm(np.cross(yu, yv), axis=1)
        L = self.lagrange(u, v)
        fr = w * J * remainder_scaled(self.x[i], self.n[i], self.H[i], self.a[i], self.g[i], y)
        fk = w * J * parametrix_scaled(self.x[i], y)
        return np.stack([L @ fr, L @ fk])

    def self_weights(self, i):
        loc = i % self.pp
        u, v, w = polar_rule(float(self.tu[loc]), float(self.tv[loc]))
        return self._integrand(i, i // self.pp, u, v, w)

    def near_weights(self, i, P):
        cu, cv, cw = collapsed_rule(16)

        def rule(tri):
            (u0, v0), (u1, v1), (u2, v2) = tri
            det = abs((u1 - u0) * (v2 - v0) - (u2 - u0) * (v1 - v0))
            u = u0 + cu * (u1 - u0) + cv * (u2 - u0)
            v = v0 + cu * (v1 - v0) + cv * (v2 - v0)
            return self._integrand(i, P, u, v, cw * det)

        def kids(tri):
            a, b, c = (np.array(t) for t in tri)
            ab, bc, ca = 0.5 * (a + b), 0.5 * (b + c), 0.5 * (c + a)
            return [(a, ab, ca), (ab, b, bc), (ca, bc, c), (bc, ca, ab)]

        root_tri = ((0.0, 0.0), (1.0, 0.0), (0.0, 1.0))
        root = rule(root_tri)
        scale = np.maximum(np.max(np.abs(root), axis=1), 1e-300)[:, None]

        def recurse(tri, est, depth):
            ch = kids(tri)
            ests = [rule(t) for t in ch]
            total = sum(ests)
            if depth >= 14 or np.max(np.abs(total - est) / scale) <= self.near_tol:
                return total
            return sum(recurse(t, e, depth + 1) for t, e in zip(ch, ests))

        return recurse(root_tri, root, 1)

    # -------------------------------------------------------------- kernels and sums
    def kernel_R(self, i, k):
        k = np.atleast_1d(k)
        r = self.x[i] - self.x[k]
        r2 = np.sum(r * r, axis=1)
        same = r2 == 0.0
        r2 = np.where(same, 1.0, r2)
        q = (r @ self.n[i]) / r2
        val = (self.a[i] * (INV_PI * q * q - self.H[i] * INV_PI * q)
               + INV_2PI * (r @ self.g[i]) / r2) / self.a[k]
        return np.where(same, 0.0, val)

    def kernel_K(self, i, k):
        k = np.atleast_1d(k)
        r = self.x[i] - self.x[k]
        r2 = np.sum(r * r, axis=1)
        same = r2 == 0.0
        val = INV_2PI * 0.5 * np.log(np.where(same, 1.0, r2)) / self.a[k]
        return np.where(same, 0.0, val)

    def row_corrections(self, i):
        out = []
        for P in self.near_patches(i):
            W = self.self_weights(i) if P == i // self.pp else self.near_weights(i, P)
            k = np.arange(P * self.pp, (P + 1) * self.pp)
            CR = W[0] / self.a[k] - self.w[k] * self.kernel_R(i, k)
            CK = W[1] / self.a[k] - self.w[k] * self.kernel_K(i, k)
            if P == i // self.pp:
                CR[i - P * self.pp] = W[0][i - P * self.pp] / self.a[i]
                CK[i - P * self.pp] = W[1][i - P * self.pp] / self.a[i]
            out.append((P, CR, CK))
        return out

    def smooth_matrix(self, which, rows=None):
        """Dense smooth-rule matrix [len(rows), N]: w_j F(x_i, x_j), zero diagonal."""
        rows = np.arange(self.N) if rows is None else np.asarray(rows)
        fn = self.kernel_R if which == "R" else self.kernel_K
        allk = np.arange(self.N)
        return np.stack([self.w * fn(i, allk) for i in rows])

    def smooth_apply(self, which, sigma, rows=None):
        rows = np.arange(self.N) if rows is None else np.asarray(rows)
        fn = self.kernel_R if which == "R" else self.kernel_K
        allk = np.arange(self.N)
        return np.array([np.dot(self.w * fn(i, allk), sigma) for i in rows])


# -------------------------------------------------------------------- process pool
_WORKER_TRI = None


def _init_tri_worker(disc):
    global _WORKER_TRI
    _WORKER_TRI = disc


def _tri_rows(rows):
    return [_WORKER_TRI.row_corrections(i) for i in rows]


def tri_near_field(disc: TriDiscretization, rows=None, processes=None):
    """NearField (operator.py) of a triangle discretisation, rows built by spawned workers."""
    import multiprocessing as mp
    import os
    from .operator import NearField
    rows = np.arange(disc.N) if rows is None else np.asarray(rows)
    nf = NearField.__new__(NearField)
    nf.disc = disc
    nf.rows = [int(i) for i in rows]
    if not processes or processes <= 1:
        nf.corr = {i: disc.row_corrections(i) for i in nf.rows}
        return nf
    order = sorted(nf.rows, key=lambda i: (i % disc.pp, i))   # polar rules reused per worker
    nch = processes * 4
    size = (len(order) + nch - 1) // nch
    chunks = [order[k:k + size] for k in range(0, len(order), size)]
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(processes, initializer=_init_tri_worker,
                                          initargs=(disc,)) as pool:
            res = pool.map(_tri_rows, chunks)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    nf.corr = {}
    for ch, rr in zip(chunks, res):
        for i, r in zip(ch, rr):
            nf.corr[i] = r
    return nf
