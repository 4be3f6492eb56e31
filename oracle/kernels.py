"""Parametrix and remainder kernels for div_Gamma(a grad_Gamma u) = f with c = 0.

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
