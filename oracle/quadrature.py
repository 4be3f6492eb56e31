"""The three quadrature classes of Sec. 6.1, restated for quad patches.

Smooth (Sec. 6.1.3): far patches use the nodes themselves,
sum_k w_k F(x, x_k) sigma_k with w_k = omega_i omega_j |y_u x y_v|; that is
the plain Nystrom sum and lives in operator.py.

Singular, self patch (Sec. 6.1.1, eq. radial_int): for a target at the
reference point (u0, v0) of its own patch, integrate in polar coordinates
(r, theta) centred there:

  int_0^{2 pi} int_0^{L(theta)} F(x, y~(u0 + r cos t, v0 + r sin t)) phi(...) r dr dt

with L(theta) the distance to the edge of the square along the ray.  Theta is
split at the four corner directions; each piece is divided into Gauss-Legendre
panels chosen adaptively so that L(theta)^2 is integrated to a tolerance (the
paper's criterion), then further split to a maximum angular width so that the
angular variation of the degree-(p-1) interpolation basis is resolved.  The
radial integral uses Gauss-Legendre panels graded dyadically toward r = 0,
[0, L 2^-M], [L 2^-M, L 2^-(M-1)], ..., [L/2, L] (resolving the r log r
behaviour of the parametrix), with panels longer than h_max split further.
All panels are 16-point rules (the paper's "16th-order panels").

Nearly singular, near patches (Sec. 6.1.2): the integrals
int R(x, y~(u,v)) l_k(u,v) J~(u,v) du dv of the basis functions are computed
by adaptive quadtree subdivision of [-1,1]^2 with a 16 x 16 tensor Gauss rule
on each square, splitting a square while its rule differs from the sum of its
four children's by more than the tolerance relative to the patch's weights.
(The paper uses the Koornwinder basis on triangles; on quads the Lagrange
basis on the tensor Gauss nodes is the interpolating basis, and
sum_k W_k sigma_k with W_k = int F l_k J equals int F sigma~ J.)

Near test (Sec. 6.1.2): a target is near a patch when its distance to the
patch centroid is strictly below 1.5 patch radii.
"""

from __future__ import annotations

from functools import lru_cache

import numpy as np
from numpy.polynomial.legendre import leggauss

from .kernels import (advection_scaled, parametrix_scaled, remainder_scaled, scaled_pair_c,
                      wavenumber)
from .patch import PatchInterpolant, lagrange_basis

_T16, _W16 = leggauss(16)

NEAR_FACTOR = 1.5


def gl_panel(a, b):
    """16-point Gauss-Legendre nodes and weights on [a, b]."""
    h = 0.5 * (b - a)
    return a + h * (_T16 + 1.0), h * _W16


def ray_length(u0, v0, theta):
    """L(theta): distance from (u0, v0) to the boundary of [-1,1]^2 along theta."""
    theta = np.asarray(theta, dtype=np.float64)
    c, s = np.cos(theta), np.sin(theta)
    big = np.inf
    with np.errstate(divide="ignore", invalid="ignore"):
        lu = np.where(c > 0, (1.0 - u0) / c, np.where(c < 0, (-1.0 - u0) / c, big))
        lv = np.where(s > 0, (1.0 - v0) / s, np.where(s < 0, (-1.0 - v0) / s, big))
    return np.minimum(lu, lv)


def corner_sectors(u0, v0):
    """The four angular sectors between the corner directions, as (start, end)."""
    cu = np.array([1.0, -1.0, -1.0, 1.0])
    cv = np.array([1.0, 1.0, -1.0, -1.0])
    ang = np.sort(np.mod(np.arctan2(cv - v0, cu - u0), 2 * np.pi))
    return [(ang[k], ang[k + 1] if k < 3 else ang[0] + 2 * np.pi) for k in range(4)]


def _l2_integral(u0, v0, a, b):
    th, w = gl_panel(a, b)
    return np.dot(w, ray_length(u0, v0, th) ** 2)


def theta_panels(u0, v0, tol=1e-14, max_width=np.pi / 24, max_depth=50):
    """Theta panels: adaptive on int L^2 (Sec. 6.1.1), then capped in width."""
    panels = []

    def split(a, b, whole, depth):
        m = 0.5 * (a + b)
        left, right = _l2_integral(u0, v0, a, m), _l2_integral(u0, v0, m, b)
        if depth >= max_depth or abs(whole - left - right) <= tol:
            panels.append((a, b))
            return
        split(a, m, left, depth + 1)
        split(m, b, right, depth + 1)

    for a, b in corner_sectors(u0, v0):
        split(a, b, _l2_integral(u0, v0, a, b), 0)
    out = []
    for a, b in sorted(panels):
        k = max(1, int(np.ceil((b - a) / max_width)))
        edges = np.linspace(a, b, k + 1)
        out.extend(zip(edges[:-1], edges[1:]))
    return out


def radial_breakpoints(L, levels=16, h_max=0.5):
    """Dyadic grading toward 0, then panels no longer than h_max."""
    br = [0.0] + [L * 2.0 ** (-k) for k in range(levels, -1, -1)]
    out = [0.0]
    for a, b in zip(br[:-1], br[1:]):
        k = max(1, int(np.ceil((b - a) / h_max)))
        out.extend(list(np.linspace(a, b, k + 1)[1:]))
    return np.array(out)


@lru_cache(maxsize=4096)
def _polar_rule(u0, v0, levels, h_max, max_width):
    """Points (u, v) and weights (omega_theta * omega_r * r) of the polar rule."""
    us, vs, ws = [], [], []
    for a, b in theta_panels(u0, v0, max_width=max_width):
        th, wth = gl_panel(a, b)
        for t_k, w_k in zip(th, wth):
            L = float(ray_length(u0, v0, t_k))
            br = radial_breakpoints(L, levels, h_max)
            ra, rb = br[:-1, None], br[1:, None]
            r = (ra + 0.5 * (rb - ra) * (_T16 + 1.0)).ravel()
            wr = (0.5 * (rb - ra) * _W16).ravel()
            us.append(u0 + r * np.cos(t_k))
            vs.append(v0 + r * np.sin(t_k))
            ws.append(w_k * wr * r)
    return np.concatenate(us), np.concatenate(vs), np.concatenate(ws)


def polar_rule(u0, v0, levels=16, h_max=0.5, max_width=np.pi / 24):
    return _polar_rule(float(u0), float(v0), int(levels), float(h_max), float(max_width))


def self_weights(patch: PatchInterpolant, u0, v0, x, n, H, a_x, g_x,
                 levels=16, h_max=0.5, max_width=np.pi / 24, c_x=None, q=None, b_x=None):
    """Singular-quadrature weights of the target's own patch (eq. radial_int).

    Returns (W_R, W_K), each [p*p] in node order a*p + b, with
    W_R[ab] = int a(y) R(x, y~) l_a(u) l_b(v) J~(u, v) du dv and
    W_K[ab] = int a(y) K(x, y~) l_a(u) l_b(v) J~(u, v) du dv
    (the a(y) factor is removed here and applied as sigma_k / a_k).

    x - y~ is formed from the node offsets (PatchInterpolant.offsets) so the
    kernel keeps its precision as y~ -> x.
    The integration surface is the interpolated patch y~, so the normal in
    q = n.r/r^2 is that patch's own unit normal at the target (the argument
    n serves only the advection term below).  With the exact parametrisation of Sec. 6.1.1 the
    two coincide; with an interpolated patch an O(delta) mismatch between the
    given normal and the patch would add a delta^2/r^2 term to R and make its
    polar integral diverge logarithmically.

    c != 0: c_x is c at the target and q [p, p] holds c/a at the patch's
    nodes; q is interpolated to each quadrature point and the kernels use
    k = sqrt(q) there (a(y) K = g(r; k(y)), see kernels.py).  The weights are
    then complex.

    b_x (b != 0, eq. adv_remainder): the advection field at the target; the
    remainder weights then integrate a(y) R_b = a(y) R + a(y) b . grad_G K.
    grad_G there is taken with the given normal n at the target (b is tangential
    to it): the advection term is a first derivative at x, so unlike the
    curvature terms it has no delta^2/r^2 sensitivity to the patch normal.
    """
    n_patch = patch.normal_at(u0, v0)
    u, v, w = polar_rule(u0, v0, levels, h_max, max_width)
    Lu, Lv = patch.basis(u, v)
    J = np.sum((Lu @ patch.J) * Lv, axis=1)
    # the kernels depend on y only through x - y; form it from node offsets
    p = patch.p
    D = (patch.X - x).reshape(p, 3 * p)
    r = -np.sum((Lu @ D).reshape(-1, p, 3) * Lv[:, :, None], axis=1)
    zero = np.zeros(3)
    k = None
    if q is None:
        fr = w * J * remainder_scaled(zero, n_patch, H, a_x, g_x, -r)
        fk = w * J * parametrix_scaled(zero, -r)
    else:
        k = wavenumber(np.sum((Lu @ q) * Lv, axis=1), 1.0)
        aR, aK = scaled_pair_c(zero, n_patch, H, a_x, g_x, c_x, -r, k)
        fr, fk = w * J * aR, w * J * aK
    if b_x is not None:
        fr = fr + w * J * advection_scaled(zero, n, b_x, -r, k)
    WR = (Lu * fr[:, None]).T @ Lv
    WK = (Lu * fk[:, None]).T @ Lv
    return WR.ravel(), WK.ravel()


def _square_rule(patch: PatchInterpolant, x, n, H, a_x, g_x, u0, u1, v0, v1,
                 c_x=None, q=None, b_x=None):
    """16 x 16 tensor Gauss rule for the weights over one sub-square."""
    uq, wu = gl_panel(u0, u1)
    vq, wv = gl_panel(v0, v1)
    Lu = lagrange_basis(patch.t, uq)
    Lv = lagrange_basis(patch.t, vq)
    y = np.einsum("qa,abc,rb->qrc", Lu, patch.X, Lv)
    J = np.einsum("qa,ab,rb->qr", Lu, patch.J, Lv)
    ww = wu[:, None] * wv[None, :] * J
    k = None
    if q is None:
        fr = ww * remainder_scaled(x, n, H, a_x, g_x, y)
        fk = ww * parametrix_scaled(x, y)
    else:
        k = wavenumber(np.einsum("qa,ab,rb->qr", Lu, q, Lv), 1.0)
        aR, aK = scaled_pair_c(x, n, H, a_x, g_x, c_x, y, k)
        fr, fk = ww * aR, ww * aK
    if b_x is not None:
        fr = fr + ww * advection_scaled(x, n, b_x, y, k)
    WR = np.einsum("qr,qa,rb->ab", fr, Lu, Lv)
    WK = np.einsum("qr,qa,rb->ab", fk, Lu, Lv)
    return np.stack([WR.ravel(), WK.ravel()])


def near_weights(patch: PatchInterpolant, x, n, H, a_x, g_x, tol=1e-13, max_depth=16,
                 c_x=None, q=None, b_x=None):
    """Nearly singular weights of a near (non-self) patch by adaptive subdivision.

    Returns (W_R, W_K) as in self_weights.  Also returns the number of
    accepted squares via the attribute-free tuple (W_R, W_K, nsq).
    c_x, q and b_x as in self_weights.
    """
    cq = {"c_x": c_x, "q": q, "b_x": b_x}
    root = _square_rule(patch, x, n, H, a_x, g_x, -1.0, 1.0, -1.0, 1.0, **cq)
    scale = np.maximum(np.max(np.abs(root), axis=1), 1e-300)[:, None]
    count = [0]

    def recurse(sq, est, depth):
        u0, u1, v0, v1 = sq
        um, vm = 0.5 * (u0 + u1), 0.5 * (v0 + v1)
        kids = ((u0, um, v0, vm), (um, u1, v0, vm), (u0, um, vm, v1), (um, u1, vm, v1))
        ests = [_square_rule(patch, x, n, H, a_x, g_x, *k, **cq) for k in kids]
        total = ests[0] + ests[1] + ests[2] + ests[3]
        if depth >= max_depth or np.max(np.abs(total - est) / scale) <= tol:
            count[0] += 4
            return total
        return sum(recurse(k, e, depth + 1) for k, e in zip(kids, ests))

    W = recurse((-1.0, 1.0, -1.0, 1.0), root, 1)
    return W[0], W[1], count[0]
