"""Solve of the second-kind equation and the representation (Sec. 3, 4.2, 6).

Thm. LBsolvable: the problem is posed for mean-zero f and mean-zero u.
Thm. second_kind (eq. IE, eq. representation): sigma + R[sigma] = f, then
u = K[sigma].  The discrete system adds the rank-one term (sum_j w_j sigma_j) 1
(Sec. 3 null-space removal) so that A = I + R~ + 1 w^T is invertible; the
solution u is then projected to mean zero, u - (sum w u)/(sum w).

c != 0 (Thm. second_kind): sigma + R[sigma] = f has no null space, so f is
not projected, no rank-one term is added and u = K[sigma] is returned as is.

Two solvers: dense LU (numpy.linalg.solve) and restarted GMRES (Saad and
Schultz), the Krylov method the paper couples with its fast apply (Sec. 6);
GMRES runs in complex arithmetic (Hermitian inner products, complex Givens
rotations) when the operator or the right-hand side is complex.
"""

from __future__ import annotations

import numpy as np

from .operator import Discretization, NearField, apply_K, apply_R, second_kind_matrix


def weighted_mean(v, w):
    return float(np.dot(w, v) / np.sum(w))


def relative_l2(a, b, w):
    """Relative L2 error ||a - b|| / ||b|| in the surface (quadrature-weighted) norm."""
    return float(np.sqrt(np.dot(w, np.abs(a - b) ** 2) / np.dot(w, np.abs(b) ** 2)))


def gmres(matvec, b, tol=1e-12, restart=50, maxit=2000, x0=None):
    """Restarted GMRES with modified Gram-Schmidt Arnoldi and Givens rotations.

    Stops when ||b - A x||_2 / ||b||_2 <= tol (the Arnoldi residual estimate,
    confirmed with a true residual at each restart).  Returns (x, iters, relres).
    Real input stays real; complex b or x0 (or a complex matvec) runs in
    complex arithmetic with the rotation [[conj(c), conj(s)], [-s, c]].
    """
    b = np.asarray(b)
    dt = np.result_type(b, np.float64, *(() if x0 is None else (np.asarray(x0),)))
    b = b.astype(dt)
    n = b.shape[0]
    x = np.zeros(n, dt) if x0 is None else np.array(x0, dtype=dt)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    iters = 0
    while True:
        r = b - matvec(x)
        if np.iscomplexobj(r) and dt != r.dtype:
            dt = r.dtype
            x = x.astype(dt)
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol or iters >= maxit:
            return x, iters, beta / bnorm
        m = restart
        V = np.zeros((m + 1, n), dt)
        Hs = np.zeros((m + 1, m), dt)
        cs, sn = np.zeros(m, dt), np.zeros(m, dt)
        g = np.zeros(m + 1, dt)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(m):
            w = matvec(V[k])
            for j in range(k + 1):
                Hs[j, k] = np.vdot(V[j], w)
                w = w - Hs[j, k] * V[j]
            Hs[k + 1, k] = np.linalg.norm(w)
            if Hs[k + 1, k] != 0:
                V[k + 1] = w / Hs[k + 1, k]
            for j in range(k):
                t = np.conj(cs[j]) * Hs[j, k] + np.conj(sn[j]) * Hs[j + 1, k]
                Hs[j + 1, k] = -sn[j] * Hs[j, k] + cs[j] * Hs[j + 1, k]
                Hs[j, k] = t
            den = np.hypot(abs(Hs[k, k]), abs(Hs[k + 1, k]))
            cs[k], sn[k] = Hs[k, k] / den, Hs[k + 1, k] / den
            Hs[k, k] = den
            Hs[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = np.conj(cs[k]) * g[k]
            iters += 1
            k_used = k + 1
            if abs(g[k + 1]) / bnorm <= tol or iters >= maxit:
                break
        y = np.linalg.solve(np.triu(Hs[:k_used, :k_used]), g[:k_used])
        x = x + V[:k_used].T @ y


def solve(disc: Discretization, near: NearField, f, method="lu", tol=1e-12,
          project_rhs=True, return_sigma=False):
    """u with div(a grad u) + c u = f (Thm. second_kind, Sec. 3).

    c = 0: u is mean zero, and f is projected to mean zero first when
    project_rhs (Thm. LBsolvable needs a mean-zero right-hand side).
    c != 0: A = I + R~ and u = K~ sigma, with f taken as given.
    """
    if disc.c is not None:
        return _solve_c(disc, near, f, method, tol, return_sigma)
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


def _solve_c(disc, near, f, method, tol, return_sigma):
    """eq. IE and eq. representation for c != 0 (no null space, no projection)."""
    f = np.asarray(f, dtype=np.complex128)
    if method == "lu":
        sigma = np.linalg.solve(second_kind_matrix(disc, near), f)
        info = {"iters": 0}
    else:
        sigma, it, rr = gmres(lambda s: s + apply_R(disc, near, s), f, tol=tol)
        info = {"iters": it, "relres": rr}
    u = apply_K(disc, near, sigma)
    if return_sigma:
        return u, sigma, info
    return u
