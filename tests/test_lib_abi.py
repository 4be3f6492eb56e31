"""The C-ABI library loads and exports every symbol include/parametrix.h declares
(no compute calls: this runs without a GPU)."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "parametrix.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(pm_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2401_12501_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    from paper_2401_12501_gb300 import _lib
    declared = declared_symbols()
    assert len(declared) >= 14
    assert set(declared) == set(_lib.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\sT\s(pm_\w+)", out))
    for name in declared:
        assert name in exported, name
        assert hasattr(lib, name)


def test_status_strings_and_defaults(lib):
    import ctypes as C
    from paper_2401_12501_gb300 import _lib
    for st in range(10):
        assert lib.pm_status_str(st)
    o = _lib.default_opts()
    assert o.near_factor == 1.5 and o.near_max_leaves <= 512


def test_null_arguments_are_rejected_without_gpu(lib):
    import ctypes as C
    assert lib.pm_ctx_create(0, None) == 1           # PM_ERR_INVALID_ARG
    assert lib.pm_surface_info(None, None, None) == 1
    assert lib.pm_profile_enable(None, 1) == 1
    assert lib.pm_surface_set_knobs(None, None) == 1
    assert lib.pm_surface_get_knobs(None, None) == 1
    assert lib.pm_surface_autotune(None, 1, 1, 5, None) == 1
    assert lib.pm_ctx_info(None, None, 0, None) == 1
    assert lib.pm_surface_clone(None, None) == 1
    assert lib.pm_surface_set_coeff_c(None, None, None, None) == 1
    assert lib.pm_apply_c(None, 0, None, None, 0, None) == 1
    assert lib.pm_solve_c(None, None, None, 1e-8, 10, None, None) == 1
    assert lib.pm_surface_store_ff(None, 3) == 1
    assert lib.pm_surface_stored_ff(None) == 0
    h = C.c_void_p()
    assert lib.pm_bvp_create(None, 0, 1, None, None, None, None, None, None, None, None, None,
                             None, None, None, None, C.byref(h)) == 1
    assert lib.pm_bvp_create(None, 0, 0, None, None, None, None, None, None, None, None, None,
                             None, None, None, None, None) == 1
    assert lib.pm_bvp_apply(None, None, None, None, None) == 1
    assert lib.pm_bvp_solve(None, None, None, 1e-10, 10, None, None, None, None) == 1
    lib.pm_bvp_destroy(None)                          # no-op


def _header_struct_fields(name):
    src = open(os.path.join(ROOT, "include", "parametrix.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = dict((n, b) for b, n in re.findall(r"typedef struct \{([^{}]*)\}\s*(\w+)\s*;", src))[name]
    return re.findall(r"\b(int|double|size_t|pm_knobs)\s+(\w+)\s*;", body)


@pytest.mark.parametrize("cname,pyname", [("pm_opts", "PmOpts"), ("pm_solve_info", "PmSolveInfo"),
                                          ("pm_knobs", "PmKnobs"),
                                          ("pm_tune_result", "PmTuneResult")])
def test_struct_layouts_match_header(cname, pyname):
    """The ctypes mirrors of the option and info structs list the header's fields
    in the same order with the same C types (no compute calls)."""
    import ctypes as C
    from paper_2401_12501_gb300 import _lib
    ctype = {"int": C.c_int, "double": C.c_double, "size_t": C.c_size_t,
             "pm_knobs": _lib.PmKnobs}
    fields = _header_struct_fields(cname)
    py = getattr(_lib, pyname)._fields_
    assert [n for _, n in fields] == [n for n, _ in py]
    assert [ctype[t] for t, _ in fields] == [t for _, t in py]


def test_fmm_offset_classes(lib):
    """The FMM's M2L symmetry reduction (host code, no GPU): the 316 V-list offsets of
    [-3, 3]^3 (max |d_i| in {2, 3}) fall into 16 classes; for each offset the returned
    signed axis permutation g maps the class's canonical offset d_c onto it,
    (g v)_a = s_a v_pi(a); every class holds exactly the orbit of d_c under the 48
    signed permutations of the cube; other offsets are rejected."""
    import itertools
    import numpy as np
    from paper_2401_12501_gb300._lib import ptr
    cls = np.zeros(343, np.int32)
    sym = np.zeros(343, np.int32)
    canon = np.zeros(48, np.int32)
    assert lib.pm_selftest_fmm_classes(ptr(cls), ptr(sym), ptr(canon)) == 0
    canon = canon.reshape(16, 3)
    assert len({tuple(c) for c in canon}) == 16
    assert all(c[0] >= c[1] >= c[2] >= 0 and c[0] in (2, 3) for c in canon)
    members = {c: set() for c in range(16)}
    for d in itertools.product(range(-3, 4), repeat=3):
        k = ((d[0] + 3) * 7 + (d[1] + 3)) * 7 + (d[2] + 3)
        if max(map(abs, d)) < 2:
            assert cls[k] == -1
            continue
        c = int(cls[k])
        assert 0 <= c < 16
        g = int(sym[k])
        pi = [(g >> (2 * a)) & 3 for a in range(3)]
        s = [-1 if (g >> (6 + a)) & 1 else 1 for a in range(3)]
        assert sorted(pi) == [0, 1, 2]
        assert tuple(s[a] * canon[c][pi[a]] for a in range(3)) == d
        members[c].add(d)
    assert sum(len(m) for m in members.values()) == 316
    for c, m in members.items():
        orbit = {tuple(sg[a] * canon[c][p[a]] for a in range(3))
                 for p in itertools.permutations(range(3))
                 for sg in itertools.product((1, -1), repeat=3)}
        assert m == orbit, c


def test_green_function_c_nonzero(lib):
    """The library's double-precision g, g', g'' for c != 0 (pm_green.cuh, host code,
    no GPU) against the oracle's scipy evaluation: Helmholtz (q > 0, J/Y from the
    math library) and modified Helmholtz (q < 0, the library's own K0/K1: ascending
    series up to 2, trapezoid rule on the integral representation above), across
    both K0/K1 branches and far into the decay; invalid arguments are rejected."""
    import numpy as np
    from oracle.kernels import green_scaled
    from paper_2401_12501_gb300._lib import ptr
    r = np.concatenate([np.geomspace(1e-6, 60.0, 301), [0.5, 0.999, 1.0, 1.001, 2.0]])
    for q in (4.0, 0.37, -4.0, -1.0, -0.05, -30.0):
        out = np.zeros((len(r), 6))
        assert lib.pm_selftest_green(ptr(r), len(r), q, ptr(out)) == 0
        k = np.sqrt(complex(q))
        ref = green_scaled(r, k)
        for m, (g, name) in enumerate(zip(ref, ("g", "g'", "g''"))):
            got = out[:, 2 * m] + 1j * out[:, 2 * m + 1]
            # relative to |g| where it is not near a zero of J or Y, absolute otherwise
            scale = np.maximum(np.abs(g), 1e-3 * np.abs(g).max() if q > 0 else 0.0)
            err = np.abs(got - g) / np.maximum(scale, 1e-300)
            assert err.max() < 1e-12, (q, name, err.max(), r[err.argmax()])
    out = np.zeros(6)
    bad = [(np.array([1.0]), 0.0), (np.array([1.0]), np.inf), (np.array([0.0]), 1.0),
           (np.array([-1.0]), -1.0), (np.array([np.nan]), 2.0)]
    for rr, q in bad:
        assert lib.pm_selftest_green(ptr(rr), 1, q, ptr(out)) == 1
    assert lib.pm_selftest_green(None, 1, 1.0, ptr(out)) == 1


def test_green_function_complex_c(lib):
    """Complex q = c/a (the library's K0/K1 at complex argument: series below |w| = 2,
    deformed contour above) against the oracle's scipy Hankel functions, on the
    branch arg q in (-pi/2, 3pi/2] (reading 21): q in every quadrant, near the real
    axes and with large |k r|."""
    import numpy as np
    from oracle.kernels import green_scaled, wavenumber
    from paper_2401_12501_gb300._lib import ptr
    r = np.concatenate([np.geomspace(1e-5, 12.0, 161), [0.3, 1.0, 2.5]])
    for q in (4 + 1j, 4 - 1j, -4 + 0.5j, -4 - 0.5j, 2j, -2j, 0.3 + 2j, 4 + 1e-3j, -1 - 1e-3j,
              9 + 3j, 0.01 + 0.02j):
        out = np.zeros((len(r), 6))
        assert lib.pm_selftest_green_c(ptr(r), len(r), q.real, q.imag, ptr(out)) == 0
        ref = green_scaled(r, wavenumber(q, 1.0))
        for m, name in enumerate(("g", "g'", "g''")):
            got = out[:, 2 * m] + 1j * out[:, 2 * m + 1]
            err = np.abs(got - ref[m]) / np.abs(ref[m])
            assert err.max() < 1e-12, (q, name, err.max(), r[err.argmax()])
    out = np.zeros(6)
    assert lib.pm_selftest_green_c(ptr(np.array([1.0])), 1, 0.0, 0.0, ptr(out)) == 1


def test_green_function_c_nonzero_float32(lib):
    """The float32 evaluation the per-pair sums use (pm_green.cuh, host code, no GPU)
    against the oracle at the float32 radii: 2e-6 relative (absolute near the zeros of
    J and Y) plus 1.5e-7 z for the float32 rounding of z = sqrt(|q|) r, which the
    exponential decay and the oscillation turn into a relative error of about
    z * 6e-8; across the K0/K1 series/trapezoid switch at 2 and up to the float32
    underflow of K0; invalid arguments are rejected."""
    import numpy as np
    from oracle.kernels import green_scaled
    from paper_2401_12501_gb300._lib import ptr
    r = np.concatenate([np.geomspace(1e-5, 40.0, 401), [0.999, 1.0, 1.001]]).astype(np.float32)
    for q in (4.0, 0.37, -4.0, -0.05, -30.0):
        out = np.zeros((len(r), 6), np.float32)
        assert lib.pm_selftest_green_f32(ptr(r), len(r), q, ptr(out)) == 0
        q32 = float(np.float32(q))
        ref = green_scaled(r.astype(np.float64), np.sqrt(complex(q32)))
        z = np.sqrt(abs(q32)) * r.astype(np.float64)
        for m, (g, name) in enumerate(zip(ref, ("g", "g'", "g''"))):
            got = out[:, 2 * m].astype(np.float64) + 1j * out[:, 2 * m + 1]
            live = z < 85.0                       # K0 underflows float32 beyond
            scale = np.maximum(np.abs(g), 1e-3 * np.abs(g).max() if q > 0 else 0.0)
            err = np.abs(got - g)[live] / np.maximum(scale[live], 1e-30)
            bound = 2e-6 + 1.5e-7 * z[live]
            assert np.all(err < bound), (q, name, err.max(), r[live][err.argmax()])
    out = np.zeros(6, np.float32)
    for rr, q in [(np.array([1.0], np.float32), 0.0), (np.array([0.0], np.float32), 1.0),
                  (np.array([np.inf], np.float32), -1.0)]:
        assert lib.pm_selftest_green_f32(ptr(rr), 1, q, ptr(out)) == 1


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_smooth_sum_c_nonzero_pair_arithmetic(lib, sign):
    """The float32 per-pair arithmetic of the c != 0 smooth sums (host loop, no GPU)
    against the oracle's smooth sums Sum_{j != i} w_j R(x_i, x_j) sigma_j and the same
    for K, on the 384-node ellipsoid with variable a, a tangential advection field
    added to grad_G a, variable real c of one sign (Helmholtz or modified Helmholtz)
    and a complex sigma: 1e-6 relative L2 (measured 3.5e-7 for R, 2.6e-7 for K)."""
    import numpy as np
    from oracle.operator import Discretization
    from paper_2401_12501_gb300._lib import ptr
    from workloads import cubed_sphere
    from workloads.coefficients import ellipsoid_coefficient
    s = cubed_sphere(1, 8, axes=(1.0, 1.5, 2.0))
    co = ellipsoid_coefficient(s)
    N = len(s.weights)
    c = sign * (2.0 + np.exp(s.nodes[:, 0] / 2))
    b = np.cross(s.normals, np.array([0.3, -0.2, 1.0]))
    d = Discretization(s.nodes, s.normals, s.tangents, s.curvature, s.weights,
                       co.a, co.grad_a, s.npatch, s.p, c=c, b=b)
    rng = np.random.default_rng(8)
    sigma = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    refR = d.smooth_apply("R", sigma)
    refK = d.smooth_apply("K", sigma)
    f32 = lambda v: np.ascontiguousarray(v, dtype=np.float32)
    sw = s.weights * sigma / co.a
    sc = f32(np.stack([sw.real, sw.imag], 1))
    out = np.zeros((N, 4))
    # the library reads these during the call: keep every buffer referenced
    bufs = [f32(v) for v in (s.nodes, s.normals, s.curvature, co.a, co.grad_a + b, c)]
    assert lib.pm_selftest_smooth_c_f32(N, *[ptr(v) for v in bufs], ptr(sc), ptr(out)) == 0
    gotR = out[:, 0] + 1j * out[:, 1]
    gotK = out[:, 2] + 1j * out[:, 3]
    rel = lambda u, v: np.linalg.norm(u - v) / np.linalg.norm(v)
    assert rel(gotR, refR) < 1e-6, rel(gotR, refR)
    assert rel(gotK, refK) < 1e-6, rel(gotK, refK)


def test_bounds_checked_build_compiles(tmp_path):
    """The -DPM_BOUNDS_CHECK variant of the apply path compiles for sm_103a (no GPU
    needed): pm_api.cu, where every apply is bracketed by pm_surface_check and a
    finite scan of its result."""
    import subprocess
    from paper_2401_12501_gb300 import build
    src = os.path.join(build.CSRC, "pm_api.cu")
    r = subprocess.run([build.nvcc(), *build.ARCH, *build.FLAGS, "-DPM_BOUNDS_CHECK", "-c", src,
                        "-o", str(tmp_path / "pm_api_checked.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
