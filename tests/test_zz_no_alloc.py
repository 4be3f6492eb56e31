"""The allocation-free smooth remainder sum (pm_smooth_remainder_f32_noalloc).

It serves callers that cannot allocate device memory.  Called twice in a row
through the C ABI, with different densities, it must reproduce the regular
float32 smooth remainder sum of a surface (pm_apply_part with
PM_PART_SMOOTH_R) within the float32 tolerance used by the other GPU tests;
the second call also shows that nothing stale survives in the shared static
scratch.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""

import ctypes as C

import numpy as np
import pytest

from workloads import make_workload

pytestmark = pytest.mark.gpu


def test_noalloc_matches_surface_smooth_sum_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_12501_gb300 as pm
    from paper_2401_12501_gb300 import _lib

    wl = make_workload("ellipsoid_9600")
    sf, co = wl.surface, wl.coeff
    N = sf.N
    ctx = pm.Context(0)
    surf = pm.Surface.from_fixture(ctx, sf)
    surf.set_coeff(co.a, co.grad_a)
    dev = torch.device("cuda", 0)

    def f32(v):
        return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).to(dev)

    x, n, H = f32(sf.nodes), f32(sf.normals), f32(sf.curvature)
    a, g = f32(co.a), f32(co.grad_a)
    stream = torch.cuda.current_stream(dev)
    lib = _lib.lib()
    rng = np.random.default_rng(11)
    for call in range(2):
        sigma = rng.standard_normal(N) + (1.0 if call == 0 else -0.5)
        s = f32(sf.weights * sigma / co.a)
        out = torch.empty(N, dtype=torch.float64, device=dev)
        st = lib.pm_smooth_remainder_f32_noalloc(
            N, C.c_void_p(x.data_ptr()), C.c_void_p(n.data_ptr()), C.c_void_p(H.data_ptr()),
            C.c_void_p(a.data_ptr()), C.c_void_p(g.data_ptr()), C.c_void_p(s.data_ptr()),
            C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        _lib.check(st, "pm_smooth_remainder_f32_noalloc")
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = surf.apply_part(pm.PM_PART_SMOOTH_R, sigma, "fp32")
        assert np.isfinite(got).all()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-6, call

    # sizes beyond the static scratch are rejected with a clear status
    big = lib.pm_smooth_remainder_f32_noalloc(
        40000, C.c_void_p(x.data_ptr()), C.c_void_p(n.data_ptr()), C.c_void_p(H.data_ptr()),
        C.c_void_p(a.data_ptr()), C.c_void_p(g.data_ptr()), C.c_void_p(s.data_ptr()),
        C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert big == 1                                  # PM_ERR_INVALID_ARG
    assert b"32768" in lib.pm_last_error()
    surf.close()
    ctx.close()


def _noalloc(lib, torch, dev, x, n, H, a, g, s):
    """Call the allocation-free sum on float32 copies of host arrays; float64 result."""
    from paper_2401_12501_gb300 import _lib

    def f32(v):
        return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32).ravel()).to(dev)

    args = [f32(v) for v in (x, n, H, a, g, s)]
    N = len(H)
    out = torch.full((N,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    st = lib.pm_smooth_remainder_f32_noalloc(
        N, *[C.c_void_p(t.data_ptr()) for t in args], C.c_void_p(out.data_ptr()),
        C.c_void_p(stream.cuda_stream))
    _lib.check(st, "pm_smooth_remainder_f32_noalloc")
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _oracle_rows(x, n, H, a, g, s, rows):
    """sum_{j != i} s_j a_j R(x_i, x_j) in float64 from the oracle's kernel (the
    allocation-free entry point's definition: strengths s_j = w_j sigma_j / a_j)."""
    from oracle.kernels import remainder_scaled
    out = []
    for i in rows:
        k = np.arange(len(H)) != i
        out.append(np.dot(s[k], remainder_scaled(x[i], n[i], H[i], a[i], g[i], x[k])))
    return np.array(out)


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_12501_gb300 import _lib
    return torch, torch.device("cuda", 0), _lib.lib()


def test_noalloc_elementwise_against_oracle_on_the_sphere(gpu):
    """Every row of the 1,536-node sphere (config 1 geometry) against the float64
    oracle, element by element at the float32 tolerance (1e-5 of the largest row)."""
    torch, dev, lib = gpu
    wl = make_workload("sphere_1536")
    sf = wl.surface
    from workloads import smooth_random_coefficient
    co = smooth_random_coefficient(sf, 2)          # a variable coefficient exercises grad a
    sigma = np.random.default_rng(4).standard_normal(sf.N) + 0.3
    s = sf.weights * sigma / co.a
    args = (sf.nodes.reshape(-1, 3), sf.normals.reshape(-1, 3), sf.curvature, co.a,
            co.grad_a.reshape(-1, 3), s)
    got = _noalloc(lib, torch, dev, *args)
    ref = _oracle_rows(*args, range(sf.N))
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_noalloc_edge_sizes(gpu):
    """N = 1 (no pair: exactly zero), a small random cloud (N = 37, one source split),
    strengths of 1e12 (the self pair stays an exact zero, no overflow), and N = 32,768,
    the largest size the static scratch holds (a 32 x 16-patch torus, sampled rows
    against the oracle)."""
    torch, dev, lib = gpu
    rng = np.random.default_rng(8)
    one = _noalloc(lib, torch, dev, np.array([[0.3, -0.2, 0.9]]), np.array([[0.0, 0.0, 1.0]]),
                   np.array([1.0]), np.array([1.2]), np.array([[0.1, 0.0, 0.0]]), np.array([2.0]))
    assert one.shape == (1,) and one[0] == 0.0

    N = 37
    x = rng.standard_normal((N, 3))
    x /= np.linalg.norm(x, axis=1)[:, None]
    n = x.copy()
    H, a = rng.uniform(0.5, 1.5, N), rng.uniform(0.7, 1.3, N)
    g = 0.1 * rng.standard_normal((N, 3))
    s = rng.standard_normal(N)
    got = _noalloc(lib, torch, dev, x, n, H, a, g, s)
    ref = _oracle_rows(x, n, H, a, g, s, range(N))
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    big = _noalloc(lib, torch, dev, x, n, H, a, g, 1e12 * s)
    assert np.isfinite(big).all()
    assert np.abs(big - 1e12 * ref).max() <= 1e-5 * 1e12 * np.abs(ref).max()

    from workloads import smooth_random_coefficient, torus
    sf = torus(32, 16, 8)
    assert sf.N == 32768
    co = smooth_random_coefficient(sf, 5)
    sigma = rng.standard_normal(sf.N)
    s = sf.weights * sigma / co.a
    args = (sf.nodes.reshape(-1, 3), sf.normals.reshape(-1, 3), sf.curvature, co.a,
            co.grad_a.reshape(-1, 3), s)
    got = _noalloc(lib, torch, dev, *args)
    assert np.isfinite(got).all()
    rows = [0, 1, 4095, 16384, 32767] + [int(i) for i in rng.integers(0, sf.N, 11)]
    ref = _oracle_rows(*args, rows)
    assert np.abs(got[rows] - ref).max() <= 1e-5 * np.abs(ref).max()
