"""Solve of the second-kind equation and the representation (Sec. 3, 4.2, 6).

Thm. LBsolvable: the problem is posed for mean-zero f and mean-zero u.
Thm. second_kind (eq. IE, eq. representation): sigma + R[sigma] = f, then
u = K[sigma].  The discrete system adds the rank-one term (sum_j w_j sigma_j) 1
(Sec. 3 null-space removal) so that A = I + R~ + 1 w^T is invertible; the
solution u is then projected to mean zero, u - (sum w u)/(sum w).

Two solvers: dense LU (numpy.linalg.solve) and restarted GMRES (Saad and
Schultz), the Krylov method the paper couples with its fast apply (Sec. 6).
"""

from __future__ import annotations

import numpy as np

from .operator import Discretization, NearField, apply_K, apply_R, second_kind_matrix


def weighted_mean(v, w):
    return float(np.dot(w, v) / np.sum(w))


def relative_l2(a, b, w):
    """Relative L2 error ||a - b|| / ||b|| in the surface (quadrature-weighted) norm."""
    return float(np.sqrt(np.dot(w, (a - b) ** 2) / np.dot(w, b ** 2)))


def gmres(matvec, b, tol=1e-12, restart=50, maxit=2000, x0=None):
    """Restarted GMRES with modified Gram-Schmidt Arnoldi and Givens rotations.

    Stops when ||b - A x||_2 / ||b||_2 <= tol (the Arnoldi residual estimate,
    confirmed with a true residual at each restart).  Returns (x, iters, relres).
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    iters = 0
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol or iters >= maxit:
            return x, iters, beta / bnorm
        m = restart
        V = np.zeros((m + 1, n))
        Hs = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(m):
            w = matvec(V[k])
            for j in range(k + 1):
                Hs[j, k] = np.dot(V[j], w)
                w = w - Hs[j, k] * V[j]
            Hs[k + 1, k] = np.linalg.norm(w)
            if Hs[k + 1, k] > 0:
                V[k + 1] = w / Hs[k + 1, k]
            for j in range(k):
                t = cs[j] * Hs[j, k] + sn[j] * Hs[j + 1, k]
                Hs[j + 1, k] = -sn[j] * Hs[j, k] + cs[j] * Hs[j + 1, k]
                Hs[j, k] = t
            den = np.hypot(Hs[k, k], Hs[k + 1, k])
            cs[k], sn[k] = Hs[k, k] / den, Hs[k + 1, k] / den
            Hs[k, k] = den
            Hs[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            iters += 1
            k_used = k + 1
            if abs(g[k + 1]) / bnorm <= tol or iters >= maxit:
                break
        y = np.linalg.solve(np.triu(Hs[:k_used, :k_used]), g[:k_used])
        x = x + V[:k_used].T @ y


def solve(disc: Discretization, near: NearField, f, method="lu", tol=1e-12,
          project_rhs=True, return_sigma=False):
    """u with div(a grad u) = f, u mean zero (Thm. second_kind, Sec. 3).

    f is projected to mean zero first when project_rhs (Thm. LBsolvable needs
    a mean-zero right-hand side).
    """
    f = np.asarray(f, dtype=np.float64)
    w = disc.w
    if project_rhs:
        f = f - weighted_mean(f, w)
    if method == "lu":
        A = second_kind_matrix(disc, near)
        sigma = np.linalg.solve(A, f)
        info = {"iters": 0}
    else:
        def matvec(s):
            return s + apply_R(disc, near, s) + np.dot(w, s)
        sigma, it, rr = gmres(matvec, f, tol=tol)
        info = {"iters": it, "relres": rr}
    u = apply_K(disc, near, sigma)
    u = u - weighted_mean(u, w)
    if return_sigma:
        return u, sigma, info
    return u
