"""Order-p node sets on the reference triangle T0 = {u, v >= 0, u + v <= 1}.

An input generator, like the Gauss-Legendre nodes of the quadrilateral
surfaces: it produces the nodes and smooth-rule weights that a triangle-patch
surface is sampled at; it holds none of the parametrix method's arithmetic.

The nodes are those of Vioreanu and Rokhlin ("Spectra of multiplication
operators as a numerical tool", SIAM J. Sci. Comput. 36, 2014), which the
paper's Sec. 6.1 uses: the eigenvalues of multiplication by z = X + iY
compressed to the polynomials of total degree <= p - 1 on an equilateral
triangle.  Built here from a tensor-Legendre spanning set made orthonormal on
T0 by a QR factorisation under a collapsed Gauss rule (the eigenvalues do not
depend on which orthonormal basis of the space is used); the weights are the
interpolatory ones (exact for that space).
"""

from __future__ import annotations

from functools import lru_cache

import numpy as np
from numpy.polynomial.legendre import leggauss

# the equilateral triangle's vertices (unit circle, angles 0, 2pi/3, 4pi/3) as
# images of (0, 0), (1, 0), (0, 1)
_V = np.exp(2j * np.pi * np.arange(3) / 3.0)


def collapsed_gauss(q: int):
    """(u, v, w) of the q x q collapsed Gauss rule on T0 (u = s (1 - t), v = t)."""
    x, wx = leggauss(q)
    s, ws = 0.5 * (x + 1.0), 0.5 * wx
    S, T = np.meshgrid(s, s, indexing="ij")
    return (S * (1.0 - T)).ravel(), T.ravel(), (np.outer(ws, ws) * (1.0 - T)).ravel()


def _legendre_table(n: int, x: np.ndarray) -> np.ndarray:
    """P_0..P_n at x by the three-term recurrence: [n + 1, len(x)]."""
    P = np.empty((n + 1,) + x.shape)
    P[0] = 1.0
    if n >= 1:
        P[1] = x
    for k in range(1, n):
        P[k + 1] = ((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1)
    return P


def _spanning_set(n: int, u, v) -> np.ndarray:
    """P_a(2u - 1) P_b(2v - 1), a + b <= n: a basis of the degree-n polynomials."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    Pu, Pv = _legendre_table(n, 2 * u - 1), _legendre_table(n, 2 * v - 1)
    return np.array([Pu[a] * Pv[d - a] for d in range(n + 1) for a in range(d + 1)])


@lru_cache(maxsize=None)
def vioreanu_rokhlin_rule(p: int):
    """(u, v, w): p (p + 1) / 2 nodes in T0 ordered by (v, u), and their weights."""
    n = p - 1
    qu, qv, qw = collapsed_gauss(p + 3)
    Phi = _spanning_set(n, qu, qv)
    _, R = np.linalg.qr((Phi * np.sqrt(qw)).T)
    Psi = np.linalg.solve(R.T, Phi)                  # orthonormal on T0 under the rule
    z = _V[0] + qu * (_V[1] - _V[0]) + qv * (_V[2] - _V[0])
    lam = np.linalg.eigvals((Psi * (qw * z)) @ Psi.T)
    A = np.array([[(_V[1] - _V[0]).real, (_V[2] - _V[0]).real],
                  [(_V[1] - _V[0]).imag, (_V[2] - _V[0]).imag]])
    uv = np.linalg.solve(A, np.stack([lam.real - _V[0].real, lam.imag - _V[0].imag]))
    u, v = uv[0], uv[1]
    order = np.lexsort((np.round(u, 12), np.round(v, 12)))   # by v, then u (ties of rounding)
    u, v = u[order], v[order]
    # interpolatory weights: sum_j w_j psi(u_j, v_j) = int_T0 psi for every basis function
    Vn = np.linalg.solve(R.T, _spanning_set(n, u, v))
    w = np.linalg.solve(Vn, Psi @ qw)
    return u, v, w
