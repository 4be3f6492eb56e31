"""Triangle-patch inputs, the library's host triangle basis and the oracle's
node-interpolated triangle operators (CPU only).

* workloads.trirule builds the Vioreanu-Rokhlin rule independently of the
  oracle (tensor-Legendre spanning set, QR); its nodes and weights equal the
  oracle's (Koornwinder basis) as sets, for p = 2..8.
* pm_selftest_tri_basis: the library's Lagrange basis of the nodes (its own
  Koornwinder recurrences and inverse) and its derivative matrices equal the
  oracle's basis U^T K and U^T grad K; the basis is exact on the nodes.
* The oracle's exact Koornwinder derivatives against a five-point difference
  quotient.
* TriNodeDiscretization (geometry interpolated from the nodes): the interpolant
  reproduces the nodes, and on the icosphere R~ 1 = -1, R~ Y = 0 and
  K~ Y_l = -Y_l / (l (l + 1)) hold to discretisation error, which falls under
  refinement.
"""

import numpy as np
import pytest

from conftest import oracle_processes
from workloads.trirule import vioreanu_rokhlin_rule

ORDERS = [2, 3, 4, 5, 6, 7, 8]


def _match(a_uv, b_uv):
    """Permutation taking the rows of b to those of a (nearest neighbour)."""
    d = np.linalg.norm(a_uv[:, None, :] - b_uv[None, :, :], axis=2)
    return np.argmin(d, axis=1), d.min(axis=1).max()


@pytest.mark.parametrize("p", ORDERS)
def test_workload_rule_equals_oracle_rule(p):
    from oracle.triangle import vioreanu_rokhlin
    u, v, w = vioreanu_rokhlin_rule(p)
    ou, ov, ow = vioreanu_rokhlin(p)
    perm, dist = _match(np.stack([u, v], 1), np.stack([ou, ov], 1))
    assert len(u) == p * (p + 1) // 2
    assert dist < 1e-12
    assert sorted(perm) == list(range(len(u)))
    assert np.abs(w - ow[perm]).max() < 1e-12
    assert abs(w.sum() - 0.5) < 1e-14


@pytest.fixture(scope="module")
def lib():
    from paper_2401_12501_gb300 import build, _lib
    build.build()
    return _lib.load()


@pytest.mark.parametrize("p", [2, 4, 6, 8])
def test_library_triangle_basis_equals_oracle(lib, p):
    from paper_2401_12501_gb300._lib import ptr
    from oracle.triangle import koornwinder, koornwinder_grad
    u, v, w = vioreanu_rokhlin_rule(p)
    nt = len(u)
    ref = np.ascontiguousarray(np.stack([u, v, w], 1))
    rng = np.random.default_rng(p)
    qu, qv = rng.uniform(0, 1, 64), rng.uniform(0, 1, 64)
    flip = qu + qv > 1
    qu[flip], qv[flip] = 1 - qu[flip], 1 - qv[flip]
    qu = np.concatenate([qu, u])
    qv = np.concatenate([qv, v])
    n = len(qu)
    l, Du, Dv = np.empty((n, nt)), np.empty((nt, nt)), np.empty((nt, nt))
    assert lib.pm_selftest_tri_basis(p, ptr(ref), n, ptr(qu), ptr(qv), ptr(l), ptr(Du),
                                     ptr(Dv)) == 0
    U = np.linalg.inv(koornwinder(p - 1, u, v).T)
    assert np.abs(l - (U.T @ koornwinder(p - 1, qu, qv)).T).max() < 1e-13
    assert np.abs(l[64:] - np.eye(nt)).max() < 1e-13          # Lagrange on the nodes
    gu, gv = koornwinder_grad(p - 1, u, v)
    assert np.abs(Du - (U.T @ gu).T).max() < 1e-11
    assert np.abs(Dv - (U.T @ gv).T).max() < 1e-11
    # derivatives of the interpolant of a linear function are its slopes
    assert np.abs(Du @ (3 * u - 2 * v) - 3).max() < 1e-11
    assert np.abs(Dv @ (3 * u - 2 * v) + 2).max() < 1e-11


def test_library_rejects_bad_triangle_rules(lib):
    from paper_2401_12501_gb300._lib import ptr
    u, v, w = vioreanu_rokhlin_rule(3)
    out = np.empty((6, 6))
    bad = np.ascontiguousarray(np.stack([u, v, w], 1))
    bad[0, :2] = (0.7, 0.6)                                      # outside T0
    assert lib.pm_selftest_tri_basis(3, ptr(bad), 0, None, None, None, ptr(out), ptr(out)) == 1
    dup = np.ascontiguousarray(np.stack([u, v, w], 1))
    dup[1, :2] = dup[0, :2]                                      # not unisolvent
    assert lib.pm_selftest_tri_basis(3, ptr(dup), 0, None, None, None, ptr(out), ptr(out)) == 1
    assert lib.pm_surface_create_tri(None, 1, 3, None, None, None, None, None, None, None,
                                     None) == 1


@pytest.mark.parametrize("n", [1, 3, 7])
def test_koornwinder_gradient_against_differences(n):
    from oracle.triangle import koornwinder, koornwinder_grad
    rng = np.random.default_rng(n)
    u, v = rng.uniform(0.05, 0.45, 30), rng.uniform(0.05, 0.45, 30)
    du, dv = koornwinder_grad(n, u, v)
    h = 1e-3

    def d5(f, x, y, ax):
        e = np.array([h, 0.0]) if ax == 0 else np.array([0.0, h])
        g = [f(x + k * e[0], y + k * e[1]) for k in (-2, -1, 1, 2)]
        return (g[0] - 8 * g[1] + 8 * g[2] - g[3]) / (12 * h)

    K = lambda x, y: koornwinder(n, x, y)
    scale = np.abs(du).max() + np.abs(dv).max() + 1.0
    assert np.abs(du - d5(K, u, v, 0)).max() < 1e-7 * scale
    assert np.abs(dv - d5(K, u, v, 1)).max() < 1e-7 * scale


def test_node_interpolated_operators_on_the_icosphere():
    """Unit sphere from triangle node data: R~ 1 = -1 (so R~ sigma = -(1/4 pi) sum w sigma),
    R~ Y_3^2 = 0 and K~ Y_3^2 = -Y_3^2/12 at sampled rows; the errors fall by ~100x from
    20 to 80 patches (p = 6)."""
    from oracle.operator import apply_K, apply_R
    from oracle.triangle_nodes import TriNodeDiscretization
    from oracle.triangle_operator import tri_near_field
    from workloads import real_sph_harm
    from workloads.trisurfaces import tri_ellipsoid
    errs = []
    for level in (0, 1):
        s = tri_ellipsoid(level, 6)
        d = TriNodeDiscretization.from_surface(s)
        L = d.lagrange(d.tu, d.tv)
        assert np.abs(L - np.eye(d.pp)).max() < 1e-12               # exact on the nodes
        rows = np.arange(0, s.N, max(1, s.N // 20))
        nf = tri_near_field(d, rows=rows, processes=oracle_processes())
        Y = real_sph_harm(3, 2, s.nodes)
        e = max(np.abs(apply_R(d, nf, np.ones(s.N), rows) + 1.0).max(),
                np.abs(apply_R(d, nf, Y, rows)).max(),
                np.abs(apply_K(d, nf, Y, rows) + Y[rows] / 12).max())
        errs.append(e)
    assert errs[0] < 1e-3 and errs[1] < 1e-5 and errs[1] < errs[0] / 30, errs
