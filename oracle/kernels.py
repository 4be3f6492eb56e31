"""Parametrix and remainder kernels for div_Gamma(a grad_Gamma u) + c u = f.

The first part is the c = 0 case the solver path uses; the second part
(after the c != 0 banner below) is the Helmholtz / modified-Helmholtz case.

Sec. 4.2: the planar Green's function of a~ Delta_2 is G(r; a~, 0) =
log(r) / (2 pi a~) and the parametrix is K(x, x') = G(|x - x'|; a(x'), 0)
(eq. diff_param).  Thm. parametrix (eq. explicit_remainder) gives the
remainder, with r = x - x', r = |r|, r^ = r / r:

  R = grad_Gamma a(x) . r^ G' - a(x) G'' (n.r)^2 / r^2 + a(x) G' (n.r)^2 / r^3
      - 2 a(x) H(x) (n . r^) G'

(the c terms vanish).  With G' = 1/(2 pi a' r) and G'' = -1/(2 pi a' r^2),
a' = a(x'), the two (n.r)^2 terms add up and

  R(x, x') = (a(x)/a(x')) [ (1/pi) q^2 - (H(x)/pi) q ]
             + grad_Gamma a(x) . r / (2 pi a(x') r^2),      q = n(x).r / r^2.

For constant a this is R_LB of Thm. parametrixLB (eq. explicit_remainderLB).

The "scaled" forms below drop the 1/a(x') factor (they equal a(x') R and
a(x') K); the discrete operators multiply them by sigma(x')/a(x').
"""

from __future__ import annotations

import numpy as np

INV_PI = 1.0 / np.pi
INV_2PI = 0.5 / np.pi


def remainder_scaled(x, n, H, a_x, g_x, y):
    """a(y) * R(x, y) for one target x (arrays [3]) and sources y [..., 3]."""
    r = x - y
    r2 = np.sum(r * r, axis=-1)
    q = (r @ n) / r2
    return a_x * (INV_PI * q * q - H * INV_PI * q) + INV_2PI * (r @ g_x) / r2


def parametrix_scaled(x, y):
    """a(y) * K(x, y) = log|x - y| / (2 pi) for one target x and sources y [..., 3]."""
    r = x - y
    return INV_2PI * 0.5 * np.log(np.sum(r * r, axis=-1))


def remainder(x, n, H, a_x, g_x, y, a_y):
    """R(x, y) of eq. explicit_remainder with c = 0 (see module docstring)."""
    return remainder_scaled(x, n, H, a_x, g_x, y) / a_y


def parametrix(x, y, a_y):
    """K(x, y) = log|x - y| / (2 pi a(y)) (eq. diff_param, c = 0)."""
    return parametrix_scaled(x, y) / a_y


# ---------------------------------------------------------------------------
# c != 0 (Sec. 4.2, Helmholtz- and modified-Helmholtz-Beltrami operators)
#
# The planar Green's function solves (a~ Delta_2 + c~) G = delta.  Write
# k = sqrt(c~/a~) and g(r; k) = a~ G, the Green's function of Delta_2 + k^2:
#
#   g(r; 0) = log(r) / (2 pi),      g(r; k) = -(i/4) H0(k r)    (k != 0).
#
# Reading of the sign: the paper prints G = (i / (4 a~)) H0(.), but with the
# small-argument form H0(z) ~ (2i/pi) log z of eq. asymptotic_H that choice
# behaves like -log(r)/(2 pi a~), i.e. it solves the equation with -delta and
# does not reduce to the c~ = 0 Green's function.  The minus sign used here
# makes (a~ Delta_2 + c~) G = delta hold, matches log(r)/(2 pi a~) up to a
# constant as r -> 0, and is the sign for which eq. explicit_remainder
# reproduces the Corollary's constant-coefficient formula (eq.
# bdd_remainder_helm) exactly.
#
# Branch (Sec. 4.2: the cut of the square root lies outside the wedge that
# holds c): k = |q|^(1/2) exp(i arg(q)/2) with arg(q) in (-pi/2, 3pi/2], q = c~/a~,
# i.e. the cut runs along the negative imaginary axis of q.  On the real axis
# k > 0 for q > 0 (outgoing) and k = i sqrt(-q) for q < 0, where g(r; i kappa)
# = -K0(kappa r) / (2 pi) decays and is real; k is continuous across both real
# half-axes, so a field c whose imaginary part changes sign (the paper's
# 4 (1 + 0.2 y + 0.2 i sin x)) or whose real part passes through zero (2x) has
# a continuous kernel.  (The root with Im k >= 0 would put the cut on q > 0.)
#
# Radial derivatives (H0' = -H1, H0'' = -H0 + H1/z):
#   g'(r)  = (i k / 4) H1(k r)
#   g''(r) = (i k^2 / 4) (H0(k r) - H1(k r) / (k r))
# and g'' - g'/r = -(i k^2 / 4) H2(k r).
# ---------------------------------------------------------------------------

from scipy.special import hankel1 as _hankel1


def wavenumber(c, a):
    """k with k^2 = c/a on the branch arg(k) = arg(c/a)/2, arg(c/a) in (-pi/2, 3pi/2]."""
    q = np.asarray(c, dtype=np.complex128) / np.asarray(a, dtype=np.float64)
    k = np.sqrt(q)                      # principal: arg(q) in (-pi, pi]
    # arg(q) in (-pi, -pi/2] (a -0.0 imaginary part counts as negative) moves to
    # (pi, 3pi/2], which negates the root
    return np.where(np.signbit(q.imag) & (q.real <= 0), -k, k)


def green_scaled(r, k):
    """(g, g', g'') of r for wavenumber k (arrays broadcast); k == 0 is log r / (2 pi)."""
    r = np.asarray(r, dtype=np.float64)
    k = np.asarray(k, dtype=np.complex128)
    r, k = np.broadcast_arrays(r, k)
    g = np.empty(r.shape, np.complex128)
    g1 = np.empty(r.shape, np.complex128)
    g2 = np.empty(r.shape, np.complex128)
    zero = k == 0
    rz = r[zero]
    g[zero] = INV_2PI * np.log(rz)
    g1[zero] = INV_2PI / rz
    g2[zero] = -INV_2PI / (rz * rz)
    nz = ~zero
    kr = k[nz] * r[nz]
    h0 = _hankel1(0, kr)
    h1 = _hankel1(1, kr)
    g[nz] = -0.25j * h0
    g1[nz] = 0.25j * k[nz] * h1
    g2[nz] = 0.25j * k[nz] ** 2 * (h0 - h1 / kr)
    return g, g1, g2


def green(r, a, c):
    """(G, G', G'') of eq. diff_param's planar Green's function G(r; a, c)."""
    g, g1, g2 = green_scaled(r, wavenumber(c, a))
    a = np.asarray(a, dtype=np.float64)
    return g / a, g1 / a, g2 / a


def parametrix_c(x, y, a_y, c_y):
    """K(x, y) = G(|x - y|; a(y), c(y)) (eq. diff_param), sources y [..., 3]."""
    r = np.linalg.norm(x - y, axis=-1)
    return green(r, a_y, c_y)[0]


def remainder_c(x, n, H, a_x, g_x, c_x, y, a_y, c_y):
    """R(x, y) of eq. explicit_remainder, term by term, for general a and c.

    g_x is the surface gradient of a at x; a_y, c_y are a and c at the
    sources y [..., 3].  b = 0.
    """
    rv = x - y
    r = np.linalg.norm(rv, axis=-1)
    G, G1, G2 = green(r, a_y, c_y)
    nr = rv @ n
    return ((rv @ g_x) / r * G1
            - a_x * G2 * nr ** 2 / r ** 2
            + a_x * G1 * nr ** 2 / r ** 3
            - 2.0 * a_x * H * (nr / r) * G1
            + (c_x - a_x * np.asarray(c_y) / np.asarray(a_y)) * G)


def remainder_constant_c(x, n, H, a0, c0, y):
    """R(x, y) for constant a = a0 and c = c0 != 0 (Corollary, eq. bdd_remainder_helm).

    R = (i c0 / (4 a0)) H2(k r) (n.r)^2 / r^2 - (i k / 2) H1(k r) H (n.r) / r,
    k = sqrt(c0 / a0) with the branch of wavenumber().
    """
    k = complex(wavenumber(c0, a0))
    rv = x - y
    r = np.linalg.norm(rv, axis=-1)
    nr = rv @ n
    return (0.25j * c0 / a0 * _hankel1(2, k * r) * nr ** 2 / r ** 2
            - 0.5j * k * _hankel1(1, k * r) * H * nr / r)


def scaled_pair_c(x, n, H, a_x, g_x, c_x, y, k_y):
    """(a(y) R(x, y), a(y) K(x, y)) with a(y) G = g(r; k_y): what the quadrature integrates.

    With k_y^2 = c(y)/a(y) every term of eq. explicit_remainder carries one
    factor 1/a(y), so a(y) R depends on the source only through k_y:
      a(y) R = grad_G a(x).r^ g' - a(x) (g'' - g'/r) (n.r)^2/r^2
               - 2 a(x) H(x) (n.r^) g' + (c(x) - a(x) k_y^2) g.
    One evaluation of g, g', g'' serves both kernels.
    """
    rv = x - y
    r = np.linalg.norm(rv, axis=-1)
    g, g1, g2 = green_scaled(r, k_y)
    nr = rv @ n
    aR = ((rv @ g_x) / r * g1
          - a_x * (g2 - g1 / r) * nr ** 2 / r ** 2
          - 2.0 * a_x * H * (nr / r) * g1
          + (c_x - a_x * np.asarray(k_y) ** 2) * g)
    return aR, g


def remainder_scaled_c(x, n, H, a_x, g_x, c_x, y, k_y):
    """a(y) R(x, y) (see scaled_pair_c)."""
    return scaled_pair_c(x, n, H, a_x, g_x, c_x, y, k_y)[0]


def parametrix_scaled_c(x, y, k_y):
    """a(y) K(x, y) = g(|x - y|; k_y)."""
    return green_scaled(np.linalg.norm(x - y, axis=-1), k_y)[0]


# ---------------------------------------------------------------------------
# Advection, b != 0 (Sec. 4.3, Thm. advectionparametrix, eq. adv_remainder)
#
# The parametrix is unchanged and the remainder gains the advection term:
#   R_b(x, y) = R(x, y) + b(x) . grad_Gamma K(x, y),
# with grad_Gamma = grad - n(x) (n(x) . grad) acting on x and grad K = G'(r) r^.
# (The theorem points at eq. bdd_remainder_helm for R; read as the general R of
# eq. explicit_remainder, of which that equation is the constant-coefficient case.)
# ---------------------------------------------------------------------------


def advection_term(x, n, b_x, y, a_y, c_y=None):
    """b(x) . grad_Gamma K(x, y) for sources y [..., 3] (c_y None: c = 0)."""
    rv = x - y
    r = np.linalg.norm(rv, axis=-1)
    if c_y is None:
        G1 = INV_2PI / (np.asarray(a_y) * r)
    else:
        G1 = green(r, a_y, c_y)[1]
    bt = b_x - n * (b_x @ n)
    return G1 * (rv @ bt) / r


def advection_scaled(x, n, b_x, y, k_y=None):
    """a(y) b(x) . grad_Gamma K(x, y) = g'(r; k_y) b_t . r^ (k_y None: c = 0)."""
    rv = x - y
    r = np.linalg.norm(rv, axis=-1)
    g1 = INV_2PI / r if k_y is None else green_scaled(r, k_y)[1]
    bt = b_x - n * (b_x @ n)
    return g1 * (rv @ bt) / r
