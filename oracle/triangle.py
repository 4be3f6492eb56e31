"""Triangle patches: Koornwinder basis and Vioreanu-Rokhlin nodes (Sec. 6.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 6.1 discretises each curvilinear triangle over the standard simplex
T0 = {(u, v): u, v >= 0, u + v <= 1} at the Vioreanu-Rokhlin nodes (n_p =
p(p+1)/2 nodes of order p) and interpolates the density in the Koornwinder
orthogonal polynomials (Sec. 6.1.2).  The paper reads nodes and weights from a
precomputed table built by the Vioreanu-Rokhlin algorithm; that table is not
available, so this module builds the rule from the published method:

* Koornwinder basis of the polynomials of total degree <= n = p - 1 on T0,
    K_{m,k}(u, v) = P_m((2u + v - 1)/(1 - v)) (1 - v)^m P_k^{(2m+1, 0)}(2v - 1),
  m + k <= n (P_m Legendre, P_k^{(a,b)} Jacobi), normalised to unit L2 norm on T0.
* Nodes (Vioreanu & Rokhlin, "Spectra of multiplication operators as a
  numerical tool", SIAM J. Sci. Comput. 2014): the eigenvalues of the operator
  of multiplication by z = X + iY, compressed to that polynomial space, where
  (X, Y) are the coordinates of the equilateral triangle that T0 maps onto
  affinely.  The compressed operator commutes with the triangle's symmetries,
  so the nodes inherit them.  Mapped back to T0.
* Weights: interpolatory, sum_j w_j K_n(u_j, v_j) = int_T0 K_n for every basis
  function, so the rule integrates every polynomial of degree <= n exactly.
  (Reading: the paper's tables may carry a further optimisation of the nodes for
  a higher degree of exactness; the paper does not state it, and the
  interpolation it uses (Sec. 6.1.2) only needs these nodes.)

Integrals over T0 use a collapsed (Duffy) tensor Gauss rule: u = s (1 - t),
v = t, du dv = (1 - t) ds dt, exact for polynomials of total degree <= 2 q - 2
with q points per direction.
"""

from __future__ import annotations

from functools import lru_cache

import numpy as np
from numpy.polynomial.legendre import leggauss, legval
from scipy.special import eval_jacobi


def collapsed_rule(q: int):
    """(u, v, w) of the collapsed q x q Gauss rule on T0."""
    t, wt = leggauss(q)
    s = 0.5 * (t + 1.0)
    ws = 0.5 * wt
    S, T = np.meshgrid(s, s, indexing="ij")
    W = np.outer(ws, ws) * (1.0 - T)
    return (S * (1.0 - T)).ravel(), T.ravel(), W.ravel()


def _raw_basis(n: int, u, v):
    """Unnormalised K_{m,k}(u, v) for m + k <= n, rows in the order (m + k, k)."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    one_v = 1.0 - v
    with np.errstate(divide="ignore", invalid="ignore"):
        xi = np.where(one_v > 0, (2.0 * u + v - 1.0) / np.where(one_v > 0, one_v, 1.0), 0.0)
    rows = []
    for deg in range(n + 1):
        for k in range(deg + 1):
            m = deg - k
            c = np.zeros(m + 1)
            c[m] = 1.0
            rows.append(legval(xi, c) * one_v ** m * eval_jacobi(k, 2 * m + 1, 0.0, 2.0 * v - 1.0))
    return np.array(rows)


@lru_cache(maxsize=None)
def _norms(n: int):
    u, v, w = collapsed_rule(n + 2)
    B = _raw_basis(n, u, v)
    return np.sqrt(np.sum(B * B * w, axis=1))


def koornwinder(n: int, u, v):
    """Orthonormal Koornwinder basis of degree <= n at (u, v): array [(n+1)(n+2)/2, len(u)]."""
    return _raw_basis(n, u, v) / _norms(n)[:, None]


def koornwinder_grad(n: int, u, v):
    """(d/du, d/dv) of koornwinder(n, u, v) for points with v < 1, same layout.

    With xi = (2u + v - 1)/(1 - v), A = P_m(xi) (1 - v)^m and B = P_k^{(2m+1,0)}(2v - 1):
      dA/du = 2 P_m'(xi) (1 - v)^(m-1),
      dA/dv = [P_m'(xi) (1 + xi) - m P_m(xi)] (1 - v)^(m-1)    (d xi/dv = (1 + xi)/(1 - v)),
      dB/dv = (k + 2m + 2) P_(k-1)^{(2m+2,1)}(2v - 1)           (derivative of a Jacobi polynomial).
    """
    from numpy.polynomial.legendre import legder
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    one_v = 1.0 - v
    xi = (2.0 * u + v - 1.0) / one_v
    du, dv = [], []
    for deg in range(n + 1):
        for k in range(deg + 1):
            m = deg - k
            c = np.zeros(m + 1)
            c[m] = 1.0
            Pm, dPm = legval(xi, c), legval(xi, legder(c)) if m > 0 else 0.0 * xi
            t = 2.0 * v - 1.0
            B = eval_jacobi(k, 2 * m + 1, 0.0, t)
            dB = (k + 2 * m + 2) * eval_jacobi(k - 1, 2 * m + 2, 1.0, t) if k > 0 else 0.0 * t
            pw = one_v ** (m - 1) if m > 0 else 0.0 * one_v
            A = Pm * one_v ** m
            du.append(2.0 * dPm * pw * B)
            dv.append((dPm * (1.0 + xi) - m * Pm) * pw * B + A * dB)
    nrm = _norms(n)[:, None]
    return np.array(du) / nrm, np.array(dv) / nrm


# Affine map T0 -> equilateral triangle with vertices on the unit circle at
# angles 0, 2pi/3, 4pi/3 (u = v = 0 -> vertex 0, (1, 0) -> vertex 1, (0, 1) -> vertex 2).
_E = np.array([[np.cos(a), np.sin(a)] for a in (0.0, 2 * np.pi / 3, 4 * np.pi / 3)])


def to_equilateral(u, v):
    return _E[0] + np.outer(u, _E[1] - _E[0]) + np.outer(v, _E[2] - _E[0])


def from_equilateral(P):
    A = np.stack([_E[1] - _E[0], _E[2] - _E[0]], 1)
    uv = np.linalg.solve(A, (np.atleast_2d(P) - _E[0]).T)
    return uv[0], uv[1]


@lru_cache(maxsize=None)
def vioreanu_rokhlin(p: int):
    """(u, v, w): the order-p rule on T0, n_p = p (p + 1) / 2 nodes (see module docstring)."""
    n = p - 1
    u, v, w = collapsed_rule(p + 2)
    B = koornwinder(n, u, v)
    z = to_equilateral(u, v) @ np.array([1.0, 1.0j])
    M = (B * (w * z)) @ B.T                   # compressed multiplication by z
    lam = np.linalg.eigvals(M)
    nu, nv = from_equilateral(np.stack([lam.real, lam.imag], 1))
    order = np.lexsort((nu, nv))
    nu, nv = nu[order], nv[order]
    V = koornwinder(n, nu, nv)                # V[n, j] = K_n(u_j, v_j)
    mom = (B * w).sum(axis=1)                 # int_T0 K_n
    wq = np.linalg.solve(V, mom)
    return nu, nv, wq


def interpolation_matrix(p: int):
    """U = V^{-1} of Sec. 6.1.2: the Koornwinder coefficients c = U sigma of the interpolant.

    Reading: V maps coefficients to node values, V_{jn} = K_n(u_j, v_j), so that
    sum_n c_n K_n(u_j, v_j) = sigma_j; the paper's V_{nj} = K_n(u_j, v_j) has its
    subscripts in the other order (with it, U sigma does not interpolate).
    """
    nu, nv, _ = vioreanu_rokhlin(p)
    return np.linalg.inv(koornwinder(p - 1, nu, nv).T)
