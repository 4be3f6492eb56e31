"""Chebyshev FMM far field (PM_PREC_FMM) against the direct sums and the oracle.

The FMM replaces the far part of the smooth sums by 8x8x8-point Chebyshev
interpolation between boxes; its error against the exact sum is bounded by
the per-config tolerance for float32-class applies (at most 1e-5 relative).
The M2L step runs as per-offset-class operator GEMMs on the library's tcgen05
tensor-core kernel (float32 operands as two float16 parts) by default, or
evaluated directly on the float32 pipe.
"""

import numpy as np
import pytest

from conftest import oracle_processes
from workloads import make_workload

pytestmark = pytest.mark.gpu

TOL_FMM = 1e-5


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_12501_gb300 as pm
    c = pm.Context(0)
    yield c
    c.close()


_S = {}


def surf(ctx, name):
    import paper_2401_12501_gb300 as pm
    if name not in _S:
        wl = make_workload(name)
        s = pm.Surface.from_fixture(ctx, wl.surface)
        s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
        _S[name] = (wl, s)
    return _S[name]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name", ["torus_98304", "ellipsoid_9600"])
def test_fmm_matches_direct_sum(ctx, name):
    import paper_2401_12501_gb300 as pm
    wl, s = surf(ctx, name)
    st = s.fmm_stats()
    assert st["depth"] >= 2 and st["boxes"] > 8
    rng = np.random.default_rng(12)
    sigma = rng.standard_normal(wl.N) + 1.0
    for part in (pm.PM_PART_SMOOTH_R, pm.PM_PART_SMOOTH_K):
        exact = s.apply_part(part, sigma, "ff")
        fmm = s.apply_part(part, sigma, "fmm")
        assert rel(fmm, exact) < TOL_FMM, (part, rel(fmm, exact), st)


def test_fmm_full_apply_against_oracle_rows(ctx):
    from oracle.operator import Discretization, NearField, apply_K, apply_R
    wl, s = surf(ctx, "torus_98304")
    rng = np.random.default_rng(13)
    rows = sorted(set([0, wl.N - 1] + [int(i) for i in rng.integers(0, wl.N, 14)]))
    d = Discretization.from_workload(wl)
    nf = NearField(d, rows=rows, processes=oracle_processes())
    sigma = rng.standard_normal(wl.N) + 1.0
    oR = apply_R(d, nf, sigma, rows)
    oK = apply_K(d, nf, sigma, rows)
    yR = s.apply_R(sigma, "fmm")[rows]
    yK = s.apply_K(sigma, "fmm")[rows]
    assert np.abs(yR - oR).max() <= TOL_FMM * np.abs(oR).max()
    assert np.abs(yK - oK).max() <= TOL_FMM * np.abs(oK).max()


def test_fmm_operator_in_refined_solve(ctx):
    """GMRES with FMM applies + float-float refinement reaches the same solution."""
    wl, s = surf(ctx, "ellipsoid_9600")
    u_fmm, i_fmm = s.solve(wl.f, tol=1e-10, prec="fmm")
    u_32, _ = s.solve(wl.f, tol=1e-10, prec="fp32")
    w = wl.surface.weights
    assert i_fmm[0].residual <= 1e-10
    assert np.sqrt(np.dot(w, (u_fmm - u_32) ** 2) / np.dot(w, u_32 ** 2)) < 1e-8


def test_batched_fmm_solve(ctx):
    """Several right-hand sides in one FMM solve: the lockstep solver applies the FMM
    per right-hand side (the batched float32 kernels refuse other precisions, so a
    silent direct-sum fallback would fail here) and matches the one-at-a-time solves."""
    wl, s = surf(ctx, "ellipsoid_9600")
    w = wl.surface.weights
    F = np.stack([np.roll(wl.f, 97 * k) for k in range(3)])
    F -= (F @ w)[:, None] / w.sum()
    U, info = s.solve(F, tol=1e-10, prec="fmm")
    for k in range(3):
        alone, _ = s.solve(F[k], tol=1e-10, prec="fmm")
        assert info[k].residual <= 1e-10
        assert np.sqrt(np.dot(w, (U[k] - alone) ** 2) / np.dot(w, alone ** 2)) < 1e-8


@pytest.mark.parametrize("name", ["torus_98304", "ellipsoid_9600"])
def test_tensor_core_m2l_matches_direct_m2l(ctx, name):
    """The M2L step as per-offset GEMMs (unit-box operators scaled per level)
    against the M2L evaluated directly between the Chebyshev points: the two
    differ only by float32 rounding in the far field (the near field is shared)."""
    import paper_2401_12501_gb300 as pm
    wl = make_workload(name)
    out = {}
    for tc in (0, 1):
        o = pm.default_opts()
        o.fmm_tensor_m2l = tc
        s = pm.Surface.from_fixture(ctx, wl.surface, o)
        s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
        sigma = np.random.default_rng(14).standard_normal(wl.N) + 1.0
        out[tc] = (s.apply_part(pm.PM_PART_SMOOTH_R, sigma, "fmm"),
                   s.apply_part(pm.PM_PART_SMOOTH_K, sigma, "fmm"),
                   s.apply_part(pm.PM_PART_SMOOTH_R, sigma, "fmm"))
        s.close()
    # the two far fields differ by float32 rounding (~1e-7 per value, summed over the
    # V lists) plus the dropped split product (2^-22 per term): a few 1e-6 relative
    for k in (0, 1):
        assert rel(out[1][k], out[0][k]) < 5e-6, (k, rel(out[1][k], out[0][k]))
    assert np.array_equal(out[1][0], out[1][2])            # deterministic


@pytest.mark.parametrize("name", ["torus_98304", "ellipsoid_9600"])
def test_far_field_stream_changes_no_bit(ctx, name):
    """The far field (P2M, M2M, M2L, L2L) on its own stream beside the P2P (knob
    fmm_streams = 2, the built-in choice) and every launch on one stream (1) run the
    same kernels on the same data: applies and a graph-driven solve agree bit for bit."""
    import paper_2401_12501_gb300 as pm
    wl, s = surf(ctx, name)
    sigma = np.random.default_rng(21).standard_normal(wl.N) + 1.0
    out = {}
    for k in (1, 2):
        s.set_knobs(fmm_streams=k)
        assert s.knobs()["fmm_streams"] == k
        out[k] = (s.apply_part(pm.PM_PART_SMOOTH_R, sigma, "fmm"),
                  s.apply_part(pm.PM_PART_SMOOTH_K, sigma, "fmm"),
                  s.solve(wl.f, tol=1e-8, prec="fmm")[0])
    s.set_knobs(fmm_streams=0)
    for a, b in zip(out[1], out[2]):
        assert np.array_equal(a, b)
