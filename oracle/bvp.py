"""Neumann boundary-value system on an open surface (Sec. 5.2, eq. NeuBVPsystem).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Unknowns: sigma at the N surface nodes of Gamma and mu at the M edge nodes of
gamma = boundary of Gamma.  With the parametrix K(x, x') = log|x - x'| / (2 pi a(x'))
and the remainder R of eq. explicit_remainder (c = 0), Sec. 5.2 gives

    sigma + R_Gamma[sigma] + R_gamma[mu]                = f        on Gamma
    -mu / (2 a) + K'_Gamma[sigma] + K'_gamma[mu]         = f_gamma  on gamma
    u = K_Gamma[sigma] + K_gamma[mu]                                (eq. BC_rep)

R_gamma, K_gamma: the kernels R and K with sources on gamma (eq. diff_repr);
K'_Gamma, K'_gamma: nu(x) . grad_x K(x, x') at x on gamma (Thm. NeumannBCsrep),
with nu the binormal; grad_x K = (x - x') / (2 pi a(x') |x - x'|^2) (nu is tangent).

Discretisation (Sec. 6.1.4 and the surface rules of Sec. 6.1):
* R_Gamma, K_Gamma: the closed-surface operators of operator.py on Gamma's patches.
* R_gamma, K_gamma: trapezoid rule on an oversampled grid (F points per edge node),
  mu carried there by trigonometric interpolation (the paper's Fourier
  oversampling), a(x') taken at the oversampled points.
* K'_gamma: trapezoid rule on the edge nodes; the kernel is smooth on gamma (Thm.
  kern_smth), and its diagonal value is the limit y -> x along gamma,
  nu . (x - y) / |x - y|^2 -> -nu . gamma'' / (2 |gamma'|^2).
* K'_Gamma: the smooth rule sum_j w_j K'(x_e, x_j) sigma_j plus corrections on the
  patches near the edge node x_e.  x_e lies on the outer edge of one patch (edge
  nodes avoid patch corners); there the rule is polar about x_e over the half of the
  directions that enter the patch, theta split at the two far corners, Gauss-Legendre
  in theta and in the radius (after the polar Jacobian the integrand is smooth); on
  the other near patches it is the adaptive subdivision of quadrature.near_weights.
  As for the surface operators, sigma / a is interpolated on the patch.

The operator has a one-dimensional null space (constants solve the homogeneous
Neumann problem; reading 31): the edge row takes the rank-one term
(sum_k w_k mu_k) so that the solution is unique; u is then compared up to an
additive constant.
"""

from __future__ import annotations

import numpy as np
from numpy.polynomial.legendre import leggauss

from .kernels import INV_2PI, INV_PI
from . import operator as _operator
from .operator import Discretization, NearField, apply_K, apply_R, spawn_map
from .patch import PatchInterpolant
from .quadrature import NEAR_FACTOR


# ---------------------------------------------------------------- edge interpolation
def trig_interp_matrix(M: int, F: int) -> np.ndarray:
    """[F M, M]: values at t_j = 2 pi j / (F M) of the trigonometric interpolant
    (degree < M/2, plus the symmetric Nyquist term for even M) of data at
    t_k = 2 pi (k + 1/2) / M."""
    t = 2 * np.pi * np.arange(F * M) / (F * M)
    tk = 2 * np.pi * (np.arange(M) + 0.5) / M
    d = t[:, None] - tk[None, :]
    out = np.ones_like(d)
    for m in range(1, (M - 1) // 2 + 1):
        out += 2 * np.cos(m * d)
    if M % 2 == 0:
        out += np.cos(M // 2 * d)
    return out / M


# ---------------------------------------------------------------- kernels
def remainder_from_sources(disc: Discretization, xs, a_src, rows=None):
    """R(x_i, x') [len(rows), S] for sources x' (c = 0, eq. explicit_remainder)."""
    rows = np.arange(disc.N) if rows is None else np.asarray(rows)
    x, n, H, a, g = disc.x[rows], disc.n[rows], disc.H[rows], disc.a[rows], disc.g[rows]
    r = x[:, None, :] - xs[None, :, :]
    r2 = np.sum(r * r, axis=2)
    nr = np.einsum("ijk,ik->ij", r, n) / r2
    gr = np.einsum("ijk,ik->ij", r, g) / r2
    return (a[:, None] * (INV_PI * nr * nr - H[:, None] * INV_PI * nr) + INV_2PI * gr) / a_src[None, :]


def parametrix_from_sources(x, xs, a_src):
    """K(x, x') = log|x - x'| / (2 pi a(x'))  [len(x), S]."""
    r2 = np.sum((x[:, None, :] - xs[None, :, :]) ** 2, axis=2)
    return INV_2PI * 0.5 * np.log(r2) / a_src[None, :]


def kprime_from_sources(xe, nue, xs, a_src):
    """nu(x_e) . (x_e - x') / (2 pi a(x') |x_e - x'|^2)  [len(xe), S]."""
    d = xe[:, None, :] - xs[None, :, :]
    r2 = np.sum(d * d, axis=2)
    r2 = np.where(r2 == 0.0, np.inf, r2)        # a coincident pair contributes 0 here
    return INV_2PI * np.einsum("ijk,ik->ij", d, nue) / r2 / a_src[None, :]


# ---------------------------------------------------------------- K'_Gamma corrections
def _edge_theta_rule(u0, v0, n_theta=16, max_width=np.pi / 32):
    """Directions entering [-1, 1]^2 from (u0, v0) on its boundary: Gauss-Legendre in
    theta on panels cut at the corner directions, at most max_width wide; returns
    (cos theta, sin theta, weights, ray length L(theta) to the boundary)."""
    corners = np.array([[1.0, 1.0], [-1.0, 1.0], [-1.0, -1.0], [1.0, -1.0]])
    if abs(u0 + 1) < 1e-14:
        lo, hi = -np.pi / 2, np.pi / 2
    elif abs(u0 - 1) < 1e-14:
        lo, hi = np.pi / 2, 3 * np.pi / 2
    elif abs(v0 + 1) < 1e-14:
        lo, hi = 0.0, np.pi
    else:
        lo, hi = np.pi, 2 * np.pi
    cuts = [lo, hi]
    for c in corners:
        th = np.arctan2(c[1] - v0, c[0] - u0)
        for k in (-1, 0, 1, 2):
            tt = th + 2 * np.pi * k
            if lo + 1e-12 < tt < hi - 1e-12:
                cuts.append(tt)
    cuts = np.sort(np.array(cuts))
    xt, wt = leggauss(n_theta)
    TH, WT = [], []
    for a, b in zip(cuts[:-1], cuts[1:]):
        nsub = max(1, int(np.ceil((b - a) / max_width)))
        edges = np.linspace(a, b, nsub + 1)
        for s0, s1 in zip(edges[:-1], edges[1:]):
            TH.append(0.5 * (s0 + s1) + 0.5 * (s1 - s0) * xt)
            WT.append(0.5 * (s1 - s0) * wt)
    th, wth = np.concatenate(TH), np.concatenate(WT)
    ct, st = np.cos(th), np.sin(th)
    with np.errstate(divide="ignore"):
        Lu = np.where(ct > 0, (1 - u0) / ct, np.where(ct < 0, (-1 - u0) / ct, np.inf))
        Lv = np.where(st > 0, (1 - v0) / st, np.where(st < 0, (-1 - v0) / st, np.inf))
    return ct, st, wth, np.minimum(Lu, Lv)


def _polar_points(u0, v0, ct, st, wth, L, panels, n_rho):
    """Points (u, v) and weights (omega_theta omega_rho rho) with the radius on the
    panels [a L, b L] of the given fractions."""
    xr, wr = leggauss(n_rho)
    U, V, W = [], [], []
    for a, b in panels:
        rho = (0.5 * (a + b) + 0.5 * (b - a) * xr)[None, :] * L[:, None]
        U.append((u0 + rho * ct[:, None]).ravel())
        V.append((v0 + rho * st[:, None]).ravel())
        W.append(((0.5 * (b - a) * wr)[None, :] * L[:, None] * rho * wth[:, None]).ravel())
    return np.concatenate(U), np.concatenate(V), np.concatenate(W)


def _edge_polar_points(u0, v0, n_theta=16, n_rho=20, max_width=np.pi / 32):
    """Polar rule about (u0, v0) on the boundary of [-1, 1]^2 over the directions that
    enter the square, one radial panel: points (u, v) and weights.  Theta panels at
    most pi/32: next to a corner direction the ray length varies fast (pi/8 panels left
    2e-11 errors in the weights of an edge node 1/16 of a patch from a corner).  With
    16 Gauss points a panel in theta and 20 in the radius (12 a dyadic panel for the
    log kernel) the weights agree with 3-4x finer rules to 7e-15."""
    return _polar_points(u0, v0, *_edge_theta_rule(u0, v0, n_theta, max_width), [(0.0, 1.0)], n_rho)


def _kp_integrand(patch: PatchInterpolant, u, v, xe, nue):
    """nu . (x_e - y) / (2 pi |x_e - y|^2) J(u, v) times the tensor basis, [Q, p*p]."""
    d = -patch.offsets(u, v, xe)                          # x_e - y, accurate near x_e
    r2 = np.sum(d * d, axis=1)
    _, J, Lu, Lv = patch.evaluate(u, v)
    k = INV_2PI * (d @ nue) / r2 * J
    return (k[:, None, None] * Lu[:, :, None] * Lv[:, None, :]).reshape(len(u), -1)


def _edge_polar_points_graded(u0, v0, levels=18, n_theta=16, n_rho=12, max_width=np.pi / 32):
    """As _edge_polar_points with the radius on dyadic panels [2^-(k+1), 2^-k] L,
    k < levels, and [0, 2^-levels L]: for integrands with a log r factor (pi/8 theta
    panels left 4e-11 errors in the weights next to a corner; pi/32 converge them to
    1e-16)."""
    edges = [0.0] + [2.0 ** (k - levels) for k in range(levels + 1)]
    return _polar_points(u0, v0, *_edge_theta_rule(u0, v0, n_theta, max_width),
                         list(zip(edges[:-1], edges[1:])), n_rho)


def _k_integrand(patch: PatchInterpolant, u, v, xt):
    """log|x_t - y| / (2 pi) J(u, v) times the tensor basis, [Q, p*p]."""
    d = patch.offsets(u, v, xt)
    r2 = np.sum(d * d, axis=1)
    _, J, Lu, Lv = patch.evaluate(u, v)
    k = INV_2PI * 0.5 * np.log(r2) * J
    return (k[:, None, None] * Lu[:, :, None] * Lv[:, None, :]).reshape(len(u), -1)


def k_edge_self_weights(patch: PatchInterpolant, u0, v0, **rule):
    """W_k = int_patch log|x - y| / (2 pi) l_k J du dv about the patch's edge point
    x = y~(u0, v0) (Dirichlet trace row, K_Gamma on gamma)."""
    xt = patch.evaluate(np.array([u0]), np.array([v0]))[0][0]
    u, v, w = _edge_polar_points_graded(u0, v0, **rule)
    return w @ _k_integrand(patch, u, v, xt)


def k_edge_near_weights(patch: PatchInterpolant, xe, tol=1e-13, max_depth=18):
    """Adaptive subdivision for the log kernel (16 x 16 Gauss per square)."""
    g, gw = leggauss(16)

    def square(u0, u1, v0, v1):
        uu = 0.5 * (u0 + u1) + 0.5 * (u1 - u0) * g
        vv = 0.5 * (v0 + v1) + 0.5 * (v1 - v0) * g
        U, V = np.meshgrid(uu, vv, indexing="ij")
        Wq = np.outer(gw, gw).ravel() * 0.25 * (u1 - u0) * (v1 - v0)
        return Wq @ _k_integrand(patch, U.ravel(), V.ravel(), xe)

    root = square(-1.0, 1.0, -1.0, 1.0)
    scale = max(np.max(np.abs(root)), 1e-300)

    def rec(sq, est, depth):
        u0, u1, v0, v1 = sq
        um, vm = 0.5 * (u0 + u1), 0.5 * (v0 + v1)
        kids = ((u0, um, v0, vm), (um, u1, v0, vm), (u0, um, vm, v1), (um, u1, vm, v1))
        ests = [square(*k) for k in kids]
        tot = ests[0] + ests[1] + ests[2] + ests[3]
        if depth >= max_depth or np.max(np.abs(tot - est)) <= tol * scale:
            return tot
        return sum(rec(k, e, depth + 1) for k, e in zip(kids, ests))

    return rec((-1.0, 1.0, -1.0, 1.0), root, 1)


def kp_self_weights(patch: PatchInterpolant, u0, v0, xe, nue, **rule):
    """W_k = int_patch nu . grad K l_k J du dv about the patch's own edge point
    y~(u0, v0) (without the 1/a: the density sigma/a is interpolated).  The target is
    the interpolant's point, not the curve point x_e: they differ by the patch's
    interpolation error, and about any point off y~(u0, v0) the polar integrand would
    not be smooth at rho = 0 (reading 32)."""
    xt = patch.evaluate(np.array([u0]), np.array([v0]))[0][0]
    u, v, w = _edge_polar_points(u0, v0, **rule)
    return w @ _kp_integrand(patch, u, v, xt, nue)


def kp_near_weights(patch: PatchInterpolant, xe, nue, tol=1e-13, max_depth=18):
    """Adaptive subdivision (16 x 16 Gauss per square, as quadrature.near_weights)."""
    g, gw = leggauss(16)

    def square(u0, u1, v0, v1):
        uu = 0.5 * (u0 + u1) + 0.5 * (u1 - u0) * g
        vv = 0.5 * (v0 + v1) + 0.5 * (v1 - v0) * g
        U, V = np.meshgrid(uu, vv, indexing="ij")
        Wq = np.outer(gw, gw).ravel() * 0.25 * (u1 - u0) * (v1 - v0)
        return Wq @ _kp_integrand(patch, U.ravel(), V.ravel(), xe, nue)

    root = square(-1.0, 1.0, -1.0, 1.0)
    scale = max(np.max(np.abs(root)), 1e-300)

    def rec(sq, est, depth):
        u0, u1, v0, v1 = sq
        um, vm = 0.5 * (u0 + u1), 0.5 * (v0 + v1)
        kids = ((u0, um, v0, vm), (um, u1, v0, vm), (u0, um, vm, v1), (um, u1, vm, v1))
        ests = [square(*k) for k in kids]
        tot = ests[0] + ests[1] + ests[2] + ests[3]
        if depth >= max_depth or np.max(np.abs(tot - est)) <= tol * scale:
            return tot
        return sum(rec(k, e, depth + 1) for k, e in zip(kids, ests))

    return rec((-1.0, 1.0, -1.0, 1.0), root, 1)


# ------------------------------------------------- edge-node correction rows
def edge_correction_row(d, kind, xe, nue, P0, u0, v0, polar):
    """One edge node's quadrature corrections over the surface nodes: on each patch
    near x_e, the patch's weights (the polar rule about y~(u0, v0) on the node's own
    patch P0, the adaptive near rule elsewhere) less the smooth rule's node terms.
    kind "kp": K'_Gamma (Neumann edge rows); "k": K~ (Dirichlet edge rows)."""
    pp = d.p * d.p
    row = np.zeros(d.N)
    dist = np.linalg.norm(d.centroid - xe, axis=1)
    near = sorted(set([P0] + [int(P) for P in np.nonzero(dist < NEAR_FACTOR * d.radius)[0]]))
    for P in near:
        k = np.arange(P * pp, (P + 1) * pp)
        if kind == "kp":
            if P == P0:
                W = kp_self_weights(d.patches[P], u0, v0, xe, nue, **polar)
            else:
                W = kp_near_weights(d.patches[P], xe, nue)
            smooth = kprime_from_sources(xe[None], nue[None], d.x[k], d.a[k])[0]
        else:
            if P == P0:
                W = k_edge_self_weights(d.patches[P], u0, v0)
            else:
                W = k_edge_near_weights(d.patches[P], xe)
            smooth = parametrix_from_sources(xe[None], d.x[k], d.a[k])[0]
        row[k] += W / d.a[k] - d.w[k] * smooth
    return row


def _edge_rows_worker(tasks):
    return [edge_correction_row(_operator._WORKER_DISC, *t) for t in tasks]


def edge_correction_rows(disc, tasks, processes=None):
    """edge_correction_row for every task (kind, xe, nue, P0, u0, v0, polar), over
    spawned processes when processes > 1 (rows are independent: same values)."""
    if not processes or processes <= 1 or len(tasks) < 2:
        return [edge_correction_row(disc, *t) for t in tasks]
    nch = min(len(tasks), processes * 2)
    size = (len(tasks) + nch - 1) // nch
    chunks = [tasks[k:k + size] for k in range(0, len(tasks), size)]
    return [r for rr in spawn_map(disc, _edge_rows_worker, chunks, processes) for r in rr]


# ---------------------------------------------------------------- the system
class NeumannBVP:
    """Dense operators of eq. NeuBVPsystem for an OpenSurface (workloads.bvp)."""

    def __init__(self, osurf, coeff, a_edge, a_over, near: NearField | None = None,
                 processes=None, polar=None):
        s = osurf.surface
        self.osurf = osurf
        self.disc = Discretization(s.nodes, s.normals, s.tangents, s.curvature, s.weights,
                                   coeff.a, coeff.grad_a, s.npatch, s.p)
        self.near = near if near is not None else NearField(self.disc, processes=processes)
        self.processes = processes
        self.N, self.M = self.disc.N, osurf.M
        self.curves = osurf.curves
        self.a_edge = np.asarray(a_edge, dtype=np.float64)
        self.a_over = np.asarray(a_over, dtype=np.float64)
        self.xe = np.concatenate([c.x for c in self.curves])
        self.nue = np.concatenate([c.nu for c in self.curves])
        self.we = np.concatenate([c.w for c in self.curves])
        self.polar = dict(polar or {})
        self._build_edge()

    # edge-sourced operators, curve blocks through the interpolation matrices
    def _build_edge(self):
        N, M = self.N, self.M
        d = self.disc
        self.Rg = np.zeros((N, M))
        self.Kg = np.zeros((N, M))
        off, offo = 0, 0
        for c in self.curves:
            I = trig_interp_matrix(c.M, c.F)
            ao = self.a_over[offo:offo + c.F * c.M]
            self.Rg[:, off:off + c.M] = (remainder_from_sources(d, c.xo, ao) * c.wo) @ I
            self.Kg[:, off:off + c.M] = (parametrix_from_sources(d.x, c.xo, ao) * c.wo) @ I
            off += c.M
            offo += c.F * c.M
        # K'_gamma on the edge nodes (trapezoid; diagonal limit)
        Kp = kprime_from_sources(self.xe, self.nue, self.xe, self.a_edge) if M else np.zeros((0, 0))
        diag = []
        for c in self.curves:
            sp2 = np.sum(c.d1 * c.d1, 1)
            diag.append(-np.sum(c.nu * c.d2, 1) / (2 * sp2))
        Kp[np.diag_indices(M)] = INV_2PI * np.concatenate(diag) / self.a_edge
        self.Kpg = Kp * self.we[None, :]
        # K'_Gamma: smooth rule + corrections
        KpG = kprime_from_sources(self.xe, self.nue, d.x, d.a) * d.w[None, :]
        self.KpG = KpG + self._kp_corrections()

    def edge_patch(self, e):
        """(patch index, u0, v0) of the patch whose outer edge holds edge node e."""
        s = self.osurf.surface
        nb, nphi = s.params["n_band"], s.params["n_phi"]
        ci, k = (0, e) if e < self.curves[0].M else (1, e - self.curves[0].M)
        c = self.curves[ci]
        dph = 2 * np.pi / nphi
        b = int(np.floor(c.t[k] / dph))
        v0 = (c.t[k] - (b + 0.5) * dph) / (0.5 * dph)
        a = 0 if ci == 0 else nb - 1
        return a * nphi + b, (-1.0 if ci == 0 else 1.0), v0

    def _edge_tasks(self, kind, polar):
        return [(kind, self.xe[e], self.nue[e], *self.edge_patch(e), polar)
                for e in range(self.M)]

    def _kp_corrections(self):
        rows = edge_correction_rows(self.disc, self._edge_tasks("kp", self.polar), self.processes)
        return np.array(rows).reshape(self.M, self.N)

    # dense system with the rank-one term in the edge row
    def matrix(self):
        N, M = self.N, self.M
        A = np.zeros((N + M, N + M))
        A[:N, :N] = self.disc.smooth_matrix("R") + self.near.dense("R") + np.eye(N)
        A[:N, N:] = self.Rg
        A[N:, :N] = self.KpG
        A[N:, N:] = self.Kpg - np.diag(0.5 / self.a_edge) + np.outer(np.ones(M), self.we)
        return A

    def apply(self, sigma, mu):
        """The system's operator on (sigma, mu), rank-one term included."""
        top = sigma + apply_R(self.disc, self.near, sigma) + self.Rg @ mu
        bot = (self.KpG @ sigma + self.Kpg @ mu - 0.5 * mu / self.a_edge
               + np.dot(self.we, mu))
        return top, bot

    def represent(self, sigma, mu):
        """u = K_Gamma[sigma] + K_gamma[mu] at the surface nodes."""
        return apply_K(self.disc, self.near, sigma) + self.Kg @ mu

    def solve(self, f, f_gamma):
        A = self.matrix()
        z = np.linalg.solve(A, np.concatenate([f, f_gamma]))
        sigma, mu = z[:self.N], z[self.N:]
        return sigma, mu, self.represent(sigma, mu)


# ---------------------------------------------------------------- Dirichlet (Sec. 5.3)
def double_layer_from_sources(x, xs, nus, a):
    """nu(x') . grad_x' K(x, x') = -nu(x') . (x - x') / (2 pi a |x - x'|^2), constant a."""
    d = x[:, None, :] - xs[None, :, :]
    r2 = np.sum(d * d, axis=2)
    r2 = np.where(r2 == 0.0, np.inf, r2)
    return -INV_2PI * np.einsum("ijk,jk->ij", d, nus) / r2 / a


def t_kernel_from_sources(disc: Discretization, xs, nus):
    """T(x, x') = nu(x') . grad_x' R(x, x') for constant a (the a's of R cancel):
    R = [(n.r)^2 / r^4 - H (n.r) / r^2] / pi with r = x - x', grad_x' = -grad_r."""
    x, n, H = disc.x, disc.n, disc.H
    r = x[:, None, :] - xs[None, :, :]
    r2 = np.sum(r * r, axis=2)
    nr = np.einsum("ijk,ik->ij", r, n)
    nnu = n @ nus.T
    rnu = np.einsum("ijk,jk->ij", r, nus)
    return -INV_PI * (2 * nr * nnu / r2 ** 2 - 4 * nr ** 2 * rnu / r2 ** 3
                      - H[:, None] * nnu / r2 + 2 * H[:, None] * nr * rnu / r2 ** 2)


class DirichletBVP(NeumannBVP):
    """Dense operators of the Dirichlet system of Sec. 5.3 for constant a:

        sigma + R_Gamma[sigma] + T_gamma[mu]             = f        on Gamma
        +mu / (2a) + K_Gamma[sigma] + N_gamma[mu]        = f_gamma  on gamma
        u = K_Gamma[sigma] + N_gamma[mu]

    (reading 28: the trace of the double layer from inside is +mu/(2a) plus its value
    on gamma, and the system's second row has K_Gamma, as the trace theorem states).
    T_gamma and N_gamma off gamma: oversampled trapezoid rule; N_gamma on gamma:
    trapezoid rule with the diagonal limit -nu . gamma'' / (4 pi a |gamma'|^2); K_Gamma
    at an edge node: smooth rule plus corrections, the graded polar rule on the edge
    patch and the adaptive rule on the other near patches."""

    def __init__(self, osurf, coeff, a_edge, a_over, near=None, processes=None, polar=None):
        a0 = float(coeff.a[0])
        if (np.max(np.abs(coeff.a - a0)) > 1e-14 * a0 or np.max(np.abs(coeff.grad_a)) > 0
                or np.max(np.abs(np.asarray(a_edge) - a0)) > 1e-14 * a0):
            raise ValueError("the Dirichlet system is built for a constant coefficient")
        self.a0 = a0
        super().__init__(osurf, coeff, a_edge, a_over, near=near, processes=processes, polar=polar)

    def _build_edge(self):
        N, M = self.N, self.M
        d = self.disc
        self.Tg = np.zeros((N, M))
        self.Ng = np.zeros((N, M))
        off = 0
        for c in self.curves:
            I = trig_interp_matrix(c.M, c.F)
            self.Tg[:, off:off + c.M] = (t_kernel_from_sources(d, c.xo, c.nuo) * c.wo) @ I
            self.Ng[:, off:off + c.M] = (double_layer_from_sources(d.x, c.xo, c.nuo, self.a0) * c.wo) @ I
            off += c.M
        Nd = double_layer_from_sources(self.xe, self.xe, self.nue, self.a0)
        diag = []
        for c in self.curves:
            diag.append(-np.sum(c.nu * c.d2, 1) / (2 * np.sum(c.d1 * c.d1, 1)))
        Nd[np.diag_indices(M)] = INV_2PI * np.concatenate(diag) / self.a0
        self.Ngg = Nd * self.we[None, :]
        KG = parametrix_from_sources(self.xe, d.x, d.a) * d.w[None, :]
        self.KG = KG + self._k_corrections()

    def _k_corrections(self):
        rows = edge_correction_rows(self.disc, self._edge_tasks("k", {}), self.processes)
        return np.array(rows).reshape(self.M, self.N)

    def matrix(self):
        N, M = self.N, self.M
        A = np.zeros((N + M, N + M))
        A[:N, :N] = self.disc.smooth_matrix("R") + self.near.dense("R") + np.eye(N)
        A[:N, N:] = self.Tg
        A[N:, :N] = self.KG
        A[N:, N:] = self.Ngg + np.diag(0.5 / self.a_edge)
        return A

    def apply(self, sigma, mu):
        top = sigma + apply_R(self.disc, self.near, sigma) + self.Tg @ mu
        bot = self.KG @ sigma + self.Ngg @ mu + 0.5 * mu / self.a_edge
        return top, bot

    def represent(self, sigma, mu):
        return apply_K(self.disc, self.near, sigma) + self.Ng @ mu
