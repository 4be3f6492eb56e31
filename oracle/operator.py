"""Nystrom discretisation of R and K (Sec. 6.1, eq. IEsum) on quad patches.

For target node i:

  (R~ sigma)_i = sum over far patches P, k in P of  w_k R(x_i, x_k) sigma_k
               + sum over near patches P, k in P of  W^R_{ik} sigma_k / a_k

where W^R_{ik} = int_P a(y) R(x_i, y~) l_k J~ du dv comes from the singular
rule on the target's own patch and the nearly singular rule on the other
near patches (quadrature.py), and likewise for K.  Written as "all pairs
plus a sparse correction":

  (R~ sigma)_i = sum_{j != i} w_j R(x_i, x_j) sigma_j + sum_{near k} C^R_{ik} sigma_k,
  C^R_{ik} = W^R_{ik} / a_k - w_k R(x_i, x_k)   (k != i),   C^R_{ii} = W^R_{ii} / a_i.

The second-kind operator of Sec. 3 (eq. IELB / eq. IE) with the null space
removed by adding int sigma (Sec. 3, following the one-dimensional update
discussed there) is  A sigma = sigma + R~ sigma + (sum_j w_j sigma_j) 1.
The scale of the rank-one term is not fixed by the paper; any non-zero
multiple gives the same solution for mean-zero f.

c != 0 (Sec. 4.2, Thm. second_kind): the kernels are those of eq. diff_param
and eq. explicit_remainder with the Hankel Green's function (kernels.py), the
weights and corrections are complex, and the second-kind operator is
I + R~ with no rank-one term (eq. IE has no null space away from the
eigenvalues of the surface operator).

b != 0 (Sec. 4.3, eq. adv_remainder, eq. IE_adv): R is replaced by
R_b = R + b . grad_Gamma K in the smooth sums and the quadratures; K and the
second-kind structure are unchanged.
"""

from __future__ import annotations

import numpy as np

from .kernels import INV_2PI, INV_PI, advection_term, parametrix_c, remainder_c
from .patch import PatchInterpolant
from .quadrature import NEAR_FACTOR, near_weights, self_weights


class Discretization:
    """Surface nodes + coefficient, with the near-field structure of Sec. 6.1."""

    def __init__(self, nodes, normals, tangents, curvature, weights, a, grad_a,
                 npatch, p, self_opts=None, near_tol=1e-13, jac=None, c=None, b=None):
        self.x = np.asarray(nodes, dtype=np.float64)
        self.n = np.asarray(normals, dtype=np.float64)
        self.H = np.asarray(curvature, dtype=np.float64)
        self.w = np.asarray(weights, dtype=np.float64)
        self.a = np.asarray(a, dtype=np.float64)
        self.g = np.asarray(grad_a, dtype=np.float64)
        # c at the nodes (complex allowed); None or all zero is the c = 0 path
        self.c = None
        if c is not None and np.any(np.asarray(c) != 0):
            self.c = np.asarray(c, dtype=np.complex128) * np.ones(len(self.a))
        self.dtype = np.float64 if self.c is None else np.complex128
        # tangential advection field b at the nodes [N, 3], or None
        self.b = None if b is None else np.asarray(b, dtype=np.float64)
        self.npatch, self.p = int(npatch), int(p)
        self.N = self.npatch * self.p * self.p
        if jac is None:
            tg = np.asarray(tangents, dtype=np.float64)
            J = np.linalg.norm(np.cross(tg[:, :3], tg[:, 3:]), axis=1)
        else:
            J = np.asarray(jac, dtype=np.float64)
        X = self.x.reshape(self.npatch, self.p, self.p, 3)
        Jp = J.reshape(self.npatch, self.p, self.p)
        self.patches = [PatchInterpolant(X[P], Jp[P]) for P in range(self.npatch)]
        cr = [pt.centroid_radius() for pt in self.patches]
        self.centroid = np.array([c for c, _ in cr])
        self.radius = np.array([r for _, r in cr])
        self.t = self.patches[0].t
        self.self_opts = dict(self_opts or {})
        self.near_tol = near_tol

    @classmethod
    def from_workload(cls, wl, **kw):
        s = wl.surface
        return cls(s.nodes, s.normals, s.tangents, s.curvature, s.weights,
                   wl.coeff.a, wl.coeff.grad_a, s.npatch, s.p, **kw)

    # ---------------------------------------------------------------- near field
    def near_patches(self, i):
        """Patches near target i (strict distance < 1.5 radii), own patch first."""
        d = np.linalg.norm(self.centroid - self.x[i], axis=1)
        own = i // (self.p * self.p)
        near = [P for P in np.nonzero(d < NEAR_FACTOR * self.radius)[0] if P != own]
        return [own] + sorted(int(P) for P in near)

    def row_weights(self, i):
        """[(P, W_R [p*p], W_K [p*p])] for the near patches of target i."""
        pp = self.p * self.p
        own = i // pp
        loc = i - own * pp
        u0, v0 = self.t[loc // self.p], self.t[loc % self.p]
        out = []
        for P in self.near_patches(i):
            args = (self.x[i], self.n[i], self.H[i], self.a[i], self.g[i])
            cq = {}
            if self.c is not None:
                sl = slice(P * pp, (P + 1) * pp)
                cq = {"c_x": self.c[i], "q": (self.c[sl] / self.a[sl]).reshape(self.p, self.p)}
            if self.b is not None:
                cq["b_x"] = self.b[i]
            if P == own:
                WR, WK = self_weights(self.patches[P], u0, v0, *args, **self.self_opts, **cq)
            else:
                WR, WK, _ = near_weights(self.patches[P], *args, tol=self.near_tol, **cq)
            out.append((P, WR, WK))
        return out

    def row_corrections(self, i):
        """[(P, C_R [p*p], C_K [p*p])]: quadrature weights minus the smooth rule."""
        pp = self.p * self.p
        out = []
        for P, WR, WK in self.row_weights(i):
            k = np.arange(P * pp, (P + 1) * pp)
            CR = WR / self.a[k] - self.w[k] * self.kernel_R(i, k)
            CK = WK / self.a[k] - self.w[k] * self.kernel_K(i, k)
            if P == i // pp:
                CR[i - P * pp] = WR[i - P * pp] / self.a[i]
                CK[i - P * pp] = WK[i - P * pp] / self.a[i]
            out.append((P, CR, CK))
        return out

    # ---------------------------------------------------------------- kernels
    def kernel_R(self, i, k):
        """R(x_i, x_k) (eq. explicit_remainder; R_b of eq. adv_remainder when b is set); 0 where k == i."""
        k = np.atleast_1d(k)
        r = self.x[i] - self.x[k]
        r2 = np.sum(r * r, axis=1)
        same = r2 == 0.0
        if self.c is not None or self.b is not None:
            kk = np.where(same, (k + 1) % self.N, k)        # any other node; zeroed below
            if self.c is not None:
                val = remainder_c(self.x[i], self.n[i], self.H[i], self.a[i], self.g[i],
                                  self.c[i], self.x[kk], self.a[kk], self.c[kk])
            else:
                val = self._remainder_c0(i, kk)
            if self.b is not None:
                val = val + advection_term(self.x[i], self.n[i], self.b[i], self.x[kk],
                                           self.a[kk], None if self.c is None else self.c[kk])
            return np.where(same, 0.0, val)
        return self._remainder_c0(i, k)

    def _remainder_c0(self, i, k):
        """R(x_i, x_k) with c = 0 for k != i (the closed form of the module docstring)."""
        r = self.x[i] - self.x[k]
        r2 = np.sum(r * r, axis=1)
        same = r2 == 0.0
        r2 = np.where(same, 1.0, r2)
        q = (r @ self.n[i]) / r2
        val = (self.a[i] * (INV_PI * q * q - self.H[i] * INV_PI * q)
               + INV_2PI * (r @ self.g[i]) / r2) / self.a[k]
        return np.where(same, 0.0, val)

    def kernel_K(self, i, k):
        """K(x_i, x_k) = log|x_i - x_k| / (2 pi a_k) (eq. diff_param); 0 where k == i."""
        k = np.atleast_1d(k)
        r = self.x[i] - self.x[k]
        r2 = np.sum(r * r, axis=1)
        same = r2 == 0.0
        if self.c is not None:
            kk = np.where(same, (k + 1) % self.N, k)
            val = parametrix_c(self.x[i], self.x[kk], self.a[kk], self.c[kk])
            return np.where(same, 0.0, val)
        val = INV_2PI * 0.5 * np.log(np.where(same, 1.0, r2)) / self.a[k]
        return np.where(same, 0.0, val)

    # ---------------------------------------------------------------- smooth sums
    def smooth_matrix(self, which, rows=None):
        """Dense smooth-rule matrix [len(rows), N]: w_j F(x_i, x_j), zero diagonal."""
        rows = np.arange(self.N) if rows is None else np.asarray(rows)
        fn = self.kernel_R if which == "R" else self.kernel_K
        allk = np.arange(self.N)
        return np.stack([self.w * fn(i, allk) for i in rows])

    def smooth_apply(self, which, sigma, rows=None, chunk=256):
        """sum_{j != i} w_j F(x_i, x_j) sigma_j for the given target rows."""
        rows = np.arange(self.N) if rows is None else np.asarray(rows)
        sigma = np.asarray(sigma)
        out = np.empty((len(rows),) + sigma.shape[1:], np.result_type(self.dtype, sigma))
        for s in range(0, len(rows), chunk):
            M = self.smooth_matrix(which, rows[s:s + chunk])
            out[s:s + chunk] = M @ sigma
        return out


class NearField:
    """Near-field corrections of selected target rows: {i: [(P, C_R, C_K)]}."""

    def __init__(self, disc: Discretization, rows=None, processes=None):
        self.disc = disc
        rows = np.arange(disc.N) if rows is None else np.asarray(rows)
        self.rows = [int(i) for i in rows]
        if processes and processes > 1 and len(self.rows) > 1:
            self.corr = dict(zip(self.rows, _pool_map(disc, self.rows, processes)))
        else:
            self.corr = {i: disc.row_corrections(i) for i in self.rows}

    def apply(self, which, sigma, rows=None):
        """sum over near k of C_{ik} sigma_k for the stored rows (or a subset)."""
        rows = self.rows if rows is None else [int(i) for i in rows]
        pp = getattr(self.disc, "pp", self.disc.p ** 2)     # nodes per patch
        sigma = np.asarray(sigma)
        out = np.zeros((len(rows),) + sigma.shape[1:], np.result_type(self.disc.dtype, sigma))
        idx = 1 if which == "R" else 2
        for r, i in enumerate(rows):
            for ent in self.corr[i]:
                P = ent[0]
                out[r] += ent[idx] @ sigma[P * pp:(P + 1) * pp]
        return out

    def dense(self, which):
        """Dense correction matrix [N, N] (requires all rows)."""
        N, pp = self.disc.N, getattr(self.disc, "pp", self.disc.p ** 2)
        C = np.zeros((N, N), self.disc.dtype)
        idx = 1 if which == "R" else 2
        for i in self.rows:
            for ent in self.corr[i]:
                P = ent[0]
                C[i, P * pp:(P + 1) * pp] += ent[idx]
        return C

    def nblocks(self):
        return sum(len(v) for v in self.corr.values())


def apply_R(disc: Discretization, near: NearField, sigma, rows=None):
    """(R~ sigma) at the given rows (all rows if None)."""
    rows = near.rows if rows is None else rows
    return disc.smooth_apply("R", sigma, rows) + near.apply("R", sigma, rows)


def apply_K(disc: Discretization, near: NearField, sigma, rows=None):
    """(K~ sigma) at the given rows (all rows if None)."""
    rows = near.rows if rows is None else rows
    return disc.smooth_apply("K", sigma, rows) + near.apply("K", sigma, rows)


def second_kind_matrix(disc: Discretization, near: NearField):
    """Dense A = I + R~ + 1 w^T (Sec. 3 null-space removal), for small N.

    With c != 0 the matrix is I + R~ (eq. IE).
    """
    A = disc.smooth_matrix("R") + near.dense("R")
    A[np.diag_indices(disc.N)] += 1.0
    if disc.c is None:
        A += np.outer(np.ones(disc.N), disc.w)
    return A


# -------------------------------------------------------------------- process pool
_WORKER_DISC = None


def _init_worker(args, kw):
    global _WORKER_DISC
    _WORKER_DISC = Discretization(*args, **kw)


def _worker_rows(rows):
    return [_WORKER_DISC.row_corrections(i) for i in rows]


def spawn_map(disc, worker, chunks, processes):
    """pool.map(worker, chunks) over `processes` spawned processes, each holding a
    copy of disc (rebuilt from its arrays) as _WORKER_DISC, one BLAS thread each."""
    import multiprocessing as mp
    import os
    J = np.concatenate([pt.J.ravel() for pt in disc.patches])
    args = (disc.x, disc.n, None, disc.H, disc.w, disc.a, disc.g, disc.npatch, disc.p)
    kw = {"self_opts": disc.self_opts, "near_tol": disc.near_tol, "jac": J, "c": disc.c,
          "b": disc.b}
    ctx = mp.get_context("spawn")
    # one BLAS thread per worker process (the children read these at import)
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with ctx.Pool(processes, initializer=_init_worker, initargs=(args, kw)) as pool:
            return pool.map(worker, chunks)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _pool_map(disc, rows, processes):
    # group rows by local node index so each worker reuses its cached polar rules
    pp = disc.p * disc.p
    order = sorted(rows, key=lambda i: (i % pp, i))
    nch = processes * 4
    size = (len(order) + nch - 1) // nch
    chunks = [order[k:k + size] for k in range(0, len(order), size)]
    res = spawn_map(disc, _worker_rows, chunks, processes)
    out = {}
    for ch, rr in zip(chunks, res):
        for i, r in zip(ch, rr):
            out[i] = r
    return [out[i] for i in rows]
