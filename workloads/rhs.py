"""Right-hand sides f for div_Gamma(a grad_Gamma u) = f.

Real, orthonormal spherical harmonics (no Condon-Shortley phase):
Y_l^0 = N_l0 P_l^0(cos t); Y_l^m = sqrt(2) N_lm P_l^m(cos t) cos(m p) for
m > 0 and sqrt(2) N_l|m| P_l^|m|(cos t) sin(|m| p) for m < 0, with
N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).  On a surface other than the unit
sphere they are evaluated at the direction x/|x|.
"""

from __future__ import annotations

from math import factorial

import numpy as np

from .surfaces import Surface


def _assoc_legendre(l: int, m: int, x: np.ndarray) -> np.ndarray:
    """P_l^m(x), m >= 0, without the Condon-Shortley phase (three-term recurrence)."""
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    pmm = np.ones_like(x)
    for k in range(1, m + 1):
        pmm = pmm * (2 * k - 1) * s
    if l == m:
        return pmm
    pm1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pm1
    p_prev, p_cur = pmm, pm1
    for ll in range(m + 2, l + 1):
        p_next = ((2 * ll - 1) * x * p_cur - (ll + m - 1) * p_prev) / (ll - m)
        p_prev, p_cur = p_cur, p_next
    return p_cur


def real_sph_harm(l: int, m: int, dirs: np.ndarray) -> np.ndarray:
    """Real orthonormal Y_l^m at unit directions dirs [N, 3]."""
    d = dirs / np.linalg.norm(dirs, axis=-1, keepdims=True)
    ct = np.clip(d[:, 2], -1.0, 1.0)
    phi = np.arctan2(d[:, 1], d[:, 0])
    am = abs(m)
    norm = np.sqrt((2 * l + 1) / (4 * np.pi) * factorial(l - am) / factorial(l + am))
    P = _assoc_legendre(l, am, ct)
    if m == 0:
        return norm * P
    if m > 0:
        return np.sqrt(2.0) * norm * P * np.cos(am * phi)
    return np.sqrt(2.0) * norm * P * np.sin(am * phi)


def project_mean_zero(f: np.ndarray, w: np.ndarray) -> np.ndarray:
    """f minus its surface mean, with the mean taken with the smooth weights w."""
    if f.ndim == 1:
        return f - np.dot(w, f) / np.sum(w)
    return f - (f @ w)[:, None] / np.sum(w)


def sphere_harmonic_rhs(surf: Surface, l: int, m: int) -> np.ndarray:
    return real_sph_harm(l, m, surf.nodes)


def random_harmonic_rhs(surf: Surface, seed: int, n_terms: int = 10, lmax: int = 8,
                        lmin: int = 1) -> np.ndarray:
    """Sum of n_terms distinct real Y_l^m (lmin <= l <= lmax) with N(0,1)
    coefficients, evaluated at x/|x| and projected to mean zero."""
    rng = np.random.default_rng(seed)
    pool = [(l, m) for l in range(lmin, lmax + 1) for m in range(-l, l + 1)]
    pick = rng.choice(len(pool), size=min(n_terms, len(pool)), replace=False)
    coef = rng.standard_normal(len(pick))
    f = np.zeros(surf.N)
    for c, k in zip(coef, pick):
        l, m = pool[int(k)]
        f += c * real_sph_harm(l, m, surf.nodes)
    return project_mean_zero(f, surf.weights)


def torus_rhs(surf: Surface) -> np.ndarray:
    """f = cos(3 phi) sin(theta) on the torus, projected to mean zero."""
    th, ph = surf.params["theta"], surf.params["phi"]
    return project_mean_zero(np.cos(3 * ph) * np.sin(th), surf.weights)


def newtonian_problem(surf: Surface, coeff, x0=(-3.0, -3.0, 4.0)):
    """Manufactured solution of the paper's Laplace-Beltrami test (Sec. 7.2):
    u = v|_Gamma minus its mean, v(x) = -1 / |x - x0| (harmonic off x0), and

        f = div_Gamma(a grad_Gamma v) = grad_Gamma a . grad_Gamma v + a Lap_Gamma v,
        Lap_Gamma v = Lap v - 2 H dv/dn - d2v/dn2   (Lap v = 0)

    from the closed-form gradient and Hessian of v (a = 1 gives the paper's
    problem).  Returns (f projected to mean zero, u)."""
    x0 = np.asarray(x0, dtype=np.float64)
    d = surf.nodes - x0
    rho = np.linalg.norm(d, axis=1)
    v = -1.0 / rho
    grad = d / rho[:, None] ** 3
    n = surf.normals
    dn = np.sum(grad * n, 1)
    dnn = 1.0 / rho ** 3 - 3.0 * np.sum(d * n, 1) ** 2 / rho ** 5
    lap_g = -2.0 * surf.curvature * dn - dnn
    grad_g = grad - n * dn[:, None]
    f = np.sum(coeff.grad_a * grad_g, 1) + coeff.a * lap_g
    w = surf.weights
    return project_mean_zero(f, w), v - np.dot(w, v) / np.sum(w)


def four_harmonic_problem(surf: Surface, seed: int = 0):
    """The paper's unit-sphere test (Sec. 7.1): f a random (N(0,1), seeded)
    combination of Y_1^0, Y_3^3, Y_10^6, Y_10^7, and u = the same combination
    with each term divided by its eigenvalue -l(l+1) (a = 1).  Returns (f, u)."""
    rng = np.random.default_rng(seed)
    terms = [(1, 0), (3, 3), (10, 6), (10, 7)]
    coef = rng.standard_normal(len(terms))
    f = np.zeros(surf.N)
    u = np.zeros(surf.N)
    for c, (l, m) in zip(coef, terms):
        y = real_sph_harm(l, m, surf.nodes)
        f += c * y
        u -= c * y / (l * (l + 1))
    return f, u
