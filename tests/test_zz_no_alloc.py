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
