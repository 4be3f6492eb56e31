"""GB300-native parametrix solver for div_G(a grad_G u) = f on closed surfaces.

The compute path is the CUDA library ``libparametrix.so`` (C ABI in
``include/parametrix.h``); this package only marshals arguments.  Host arrays
are numpy float64; device arrays are contiguous float64 torch CUDA tensors.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib, tunecache
from ._lib import (PM_PART_NEAR_K, PM_PART_NEAR_R, PM_PART_SMOOTH_K,  # noqa: F401
                   PM_PART_SMOOTH_R, PM_PREC_FF, PM_PREC_FMM, PM_PREC_FP32, PM_PREC_FP32_TC, PM_PREC_FP64,
                   PM_SOLVE_DEVICE_PTRS, PM_SOLVE_INITIAL_GUESS, PM_SOLVE_PROJECT_RHS,
                   PmError, PmSolveInfo,
                   check, default_opts, ptr)

PRECISIONS = {"fp64": PM_PREC_FP64, "fp32": PM_PREC_FP32, "fp32_tc": PM_PREC_FP32_TC,
              "ff": PM_PREC_FF, "fmm": PM_PREC_FMM}


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


class Context:
    """pm_ctx: one CUDA device."""

    def __init__(self, device: int = 0):
        h = C.c_void_p()
        check(_lib.lib().pm_ctx_create(int(device), C.byref(h)), "pm_ctx_create")
        self.handle = h
        self.device = int(device)

    def info(self):
        """(device name, SM count) of the context's GPU."""
        buf = C.create_string_buffer(256)
        sms = C.c_int()
        check(_lib.lib().pm_ctx_info(self.handle, buf, len(buf), C.byref(sms)), "pm_ctx_info")
        return buf.value.decode(errors="replace"), sms.value

    def selftest_tc_gemm(self, A, B, bf16: bool = False, reps: int = 0):
        """C = A B^T on the library's tcgen05 GEMM (pm_selftest_tc_gemm).  A [rows, K]
        and B [ncols, K] are uint16 arrays of float16 (or bfloat16) bit patterns;
        returns C as float32 [ncols, rows] and, with reps > 0, the mean ms per launch."""
        A = np.ascontiguousarray(A, dtype=np.uint16)
        B = np.ascontiguousarray(B, dtype=np.uint16)
        rows, K = A.shape
        ncols = B.shape[0]
        if B.shape[1] != K:
            raise ValueError("A and B need the same K")
        out = np.empty((ncols, rows), dtype=np.float32)
        ms = C.c_double(0.0)
        check(_lib.lib().pm_selftest_tc_gemm(self.handle, ptr(A), ptr(B), ptr(out), rows, K,
                                             ncols, int(bool(bf16)), int(reps), C.byref(ms)),
              "pm_selftest_tc_gemm")
        return out, ms.value

    def close(self):
        if self.handle:
            _lib.lib().pm_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surface:
    """pm_surface: discretised closed surface, near field and coefficient."""

    def __init__(self, ctx: Context, npatch: int, p: int, nodes, normals, tangents,
                 curvature, weights, opts=None):
        N = npatch * p * p
        self.ctx, self.npatch, self.p, self.N = ctx, npatch, p, N
        arrs = [_f64(nodes, 3 * N), _f64(normals, 3 * N), _f64(tangents, 6 * N),
                _f64(curvature, N), _f64(weights, N)]
        h = C.c_void_p()
        o = C.byref(opts) if opts is not None else None
        check(_lib.lib().pm_surface_create(ctx.handle, npatch, p, *[ptr(a) for a in arrs],
                                           o, C.byref(h)), "pm_surface_create")
        self.handle = h

    @classmethod
    def from_fixture(cls, ctx, surf, opts=None):
        if hasattr(surf, "ref_u"):
            return cls.create_tri(ctx, surf.npatch, surf.p, surf.ref_u, surf.ref_v, surf.ref_w,
                                  surf.nodes, surf.normals, surf.tangents, surf.curvature,
                                  surf.weights, opts)
        return cls(ctx, surf.npatch, surf.p, surf.nodes, surf.normals, surf.tangents,
                   surf.curvature, surf.weights, opts)

    @classmethod
    def create_tri(cls, ctx, npatch, p, ref_u, ref_v, ref_w, nodes, normals, tangents,
                   curvature, weights, opts=None):
        """Triangle patches (pm_surface_create_tri): the order-p rule (ref_u, ref_v, ref_w)
        on T0 and the node data, N = npatch * p (p + 1) / 2."""
        nt = p * (p + 1) // 2
        N = npatch * nt
        ref = np.ascontiguousarray(np.stack([ref_u, ref_v, ref_w], 1), dtype=np.float64)
        if ref.shape != (nt, 3):
            raise ValueError(f"the rule has {ref.shape[0]} nodes, order {p} needs {nt}")
        arrs = [_f64(nodes, 3 * N), _f64(normals, 3 * N), _f64(tangents, 6 * N),
                _f64(curvature, N), _f64(weights, N)]
        h = C.c_void_p()
        o = C.byref(opts) if opts is not None else None
        check(_lib.lib().pm_surface_create_tri(ctx.handle, npatch, p, ptr(ref),
                                               *[ptr(a) for a in arrs], o, C.byref(h)),
              "pm_surface_create_tri")
        s = object.__new__(cls)
        s.ctx, s.npatch, s.p, s.N = ctx, npatch, p, N
        s.handle = h
        return s

    def clone(self) -> "Surface":
        """A surface on the same geometry sharing the near-field quadrature
        (pm_surface_clone): set its own coefficient with set_coeff."""
        h = C.c_void_p()
        check(_lib.lib().pm_surface_clone(self.handle, C.byref(h)), "pm_surface_clone")
        c = object.__new__(Surface)
        c.ctx, c.npatch, c.p, c.N = self.ctx, self.npatch, self.p, self.N
        c.handle = h
        return c

    def close(self):
        if self.handle:
            _lib.lib().pm_surface_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def selftest_fflog(self, xh, xl):
        """The library's float-float logarithm of xh + xl (float32 arrays)."""
        xh = np.ascontiguousarray(xh, dtype=np.float32)
        xl = np.ascontiguousarray(xl, dtype=np.float32)
        out = np.empty(xh.size)
        check(_lib.lib().pm_selftest_fflog(self.handle, ptr(xh), ptr(xl), xh.size, ptr(out)),
              "pm_selftest_fflog")
        return out

    def fmm_stats(self):
        """(near pairs, far box pairs, depth, boxes) of the FMM tree (built on first use)."""
        st = np.zeros(4)
        check(_lib.lib().pm_surface_fmm_stats(self.handle, ptr(st)), "pm_surface_fmm_stats")
        return {"p2p_pairs": st[0], "m2l_box_pairs": st[1], "depth": int(st[2]), "boxes": int(st[3])}

    def tune(self, direct_tpt=0, direct_blocks_per_sm=0):
        check(_lib.lib().pm_surface_tune(self.handle, int(direct_tpt), int(direct_blocks_per_sm)),
              "pm_surface_tune")

    def knobs(self) -> dict:
        """The surface's launch-shape knobs (pm_knobs; 0 = built-in choice)."""
        k = _lib.PmKnobs()
        check(_lib.lib().pm_surface_get_knobs(self.handle, C.byref(k)), "pm_surface_get_knobs")
        return {f: getattr(k, f) for f in tunecache.KNOB_FIELDS}

    def set_knobs(self, **kw):
        """Set knobs by name; the others keep their current values."""
        cur = self.knobs()
        unknown = set(kw) - set(cur)
        if unknown:
            raise ValueError(f"unknown knobs {sorted(unknown)}")
        cur.update({k: int(v) for k, v in kw.items()})
        k = _lib.PmKnobs(**cur)
        check(_lib.lib().pm_surface_set_knobs(self.handle, C.byref(k)), "pm_surface_set_knobs")

    def autotune(self, nrhs: int = 1, prec: str = "fp32", reps: int = 5, cache: str | None = None):
        """Time the candidate launch shapes of this surface's remainder apply
        (pm_surface_autotune) and keep the fastest.  With a cache path, a stored
        result for the same (GPU, size bucket, nrhs, precision) is applied
        instead of timing, and a new result is stored."""
        gpu, _ = self.ctx.info()
        key = tunecache.tune_key(gpu, self.N, nrhs, prec)
        if cache is not None:
            hit = tunecache.load(cache).get(key)
            if tunecache.valid_entry(hit):
                self.set_knobs(**hit["knobs"])
                return dict(hit, cached=True, key=key)
        r = _lib.PmTuneResult()
        check(_lib.lib().pm_surface_autotune(self.handle, int(nrhs), PRECISIONS[prec], int(reps),
                                             C.byref(r)), "pm_surface_autotune")
        entry = {"knobs": {f: getattr(r.best, f) for f in tunecache.KNOB_FIELDS},
                 "best_ms": r.best_ms, "default_ms": r.default_ms, "candidates": r.candidates,
                 "N": self.N}
        if cache is not None:
            tunecache.store(cache, key, entry)
        return dict(entry, cached=False, key=key)

    def info(self):
        n, nb = C.c_int(), C.c_int()
        check(_lib.lib().pm_surface_info(self.handle, C.byref(n), C.byref(nb)), "pm_surface_info")
        return n.value, nb.value

    def set_coeff(self, a, grad_a=None):
        a = _f64(a, self.N)
        g = None if grad_a is None else _f64(grad_a, 3 * self.N)
        check(_lib.lib().pm_surface_set_coeff(self.handle, ptr(a), ptr(g)),
              "pm_surface_set_coeff")

    def store_ff(self, which: str = "RK"):
        """pm_surface_store_ff: keep the float-float matrices of the remainder ("R") and/or
        parametrix ("K") smooth sums in device memory, so that every "ff" apply of them
        (solves' residuals and representation included) streams the matrix; "" releases
        both.  6 bytes per entry (to 2^-40 relative): N x ceil(N / 128) * 128 entries for
        R; for K the upper triangle of 128 x 128 tiles where the surface uses the symmetric
        sums, else N x ld."""
        bits = (1 if "R" in which else 0) | (2 if "K" in which else 0)
        if set(which) - {"R", "K"}:
            raise ValueError(f"which must name R and/or K, got {which!r}")
        check(_lib.lib().pm_surface_store_ff(self.handle, bits), "pm_surface_store_ff")

    def stored_ff(self) -> str:
        """The kernels whose float-float matrices are stored ("", "R", "K" or "RK")."""
        b = _lib.lib().pm_surface_stored_ff(self.handle)
        return ("R" if b & 1 else "") + ("K" if b & 2 else "")

    def check(self):
        """pm_surface_check: the near-field indices and stored data are consistent and finite."""
        check(_lib.lib().pm_surface_check(self.handle), "pm_surface_check")

    def set_coeff_c(self, a, grad_a, c):
        """a, grad_a as in set_coeff, and c [N] real or complex (div(a grad u) + c u = f)."""
        a = _f64(a, self.N)
        g = None if grad_a is None else _f64(grad_a, 3 * self.N)
        cz = np.asarray(c, dtype=np.complex128) * np.ones(self.N)
        cc = np.ascontiguousarray(np.stack([cz.real, cz.imag], 1))
        check(_lib.lib().pm_surface_set_coeff_c(self.handle, ptr(a), ptr(g), ptr(cc)),
              "pm_surface_set_coeff_c")

    def apply_c(self, sigma, which="R"):
        """R~ sigma or K~ sigma of a c != 0 surface (complex128 [N])."""
        sg = np.ascontiguousarray(np.asarray(sigma, dtype=np.complex128).reshape(self.N))
        out = np.empty_like(sg)
        check(_lib.lib().pm_apply_c(self.handle, 1 if which == "K" else 0, ptr(sg), ptr(out), 0,
                                    None), "pm_apply_c")
        return out

    def solve_c(self, f, tol=1e-10, maxit=2000, return_sigma=False):
        """u with div(a grad u) + c u = f on a c != 0 surface; returns (u, info[, sigma])."""
        fc = np.ascontiguousarray(np.asarray(f, dtype=np.complex128).reshape(self.N))
        u = np.empty_like(fc)
        sig = np.empty_like(fc) if return_sigma else None
        info = PmSolveInfo()
        check(_lib.lib().pm_solve_c(self.handle, ptr(fc), ptr(u), float(tol), int(maxit),
                                    ptr(sig), C.byref(info)), "pm_solve_c")
        out = (u, info)
        return out + (sig,) if return_sigma else out

    def _apply(self, fn, args, sigma, prec, stream, out=None):
        prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        dev = _is_device(sigma)
        if dev:
            import torch
            if sigma.dtype != torch.float64 or not sigma.is_contiguous():
                raise ValueError("device sigma must be a contiguous float64 tensor")
            nrhs = sigma.numel() // self.N
            if out is None:
                out = torch.empty_like(sigma)
            st = C.c_void_p(stream if stream is not None else
                            torch.cuda.current_stream(sigma.device).cuda_stream)
        else:
            sigma = np.ascontiguousarray(sigma, dtype=np.float64)
            nrhs = sigma.size // self.N
            out = np.empty_like(sigma) if out is None else out
            st = C.c_void_p(stream)
        if nrhs * self.N != (sigma.numel() if dev else sigma.size):
            raise ValueError("sigma size is not a multiple of N")
        check(fn(self.handle, *args, ptr(sigma), ptr(out), nrhs, prec, 1 if dev else 0, st),
              fn.__name__)
        return out

    def apply_R(self, sigma, prec="fp32", stream=None, out=None):
        return self._apply(_lib.lib().pm_apply_R, (), sigma, prec, stream, out)

    def apply_K(self, sigma, prec="fp32", stream=None, out=None):
        return self._apply(_lib.lib().pm_apply_K, (), sigma, prec, stream, out)

    def apply_part(self, part, sigma, prec="fp32", stream=None, out=None):
        return self._apply(_lib.lib().pm_apply_part, (int(part),), sigma, prec, stream, out)

    def get_near(self, corrections=True):
        """(row_ptr [N+1], blk_patch [nblk], corr_R, corr_K [nblk, nodes per patch])."""
        N, nb = self.info()
        pp = N // self.npatch
        rp = np.empty(N + 1, dtype=np.int32)
        bp = np.empty(nb, dtype=np.int32)
        cr = np.empty((nb, pp)) if corrections else None
        ck = np.empty((nb, pp)) if corrections else None
        check(_lib.lib().pm_surface_get_near(self.handle, ptr(rp), ptr(bp), ptr(cr), ptr(ck)),
              "pm_surface_get_near")
        return rp, bp, cr, ck

    def profile(self, enable=True):
        check(_lib.lib().pm_profile_enable(self.handle, 1 if enable else 0), "pm_profile_enable")

    def profile_read(self, phase, reset=False):
        """(milliseconds, launches) of one phase since the last reset."""
        ms, n = C.c_double(), C.c_int()
        check(_lib.lib().pm_profile_read(self.handle, int(phase), C.byref(ms), C.byref(n),
                                         1 if reset else 0), "pm_profile_read")
        return ms.value, n.value

    def solve(self, f, tol=1e-10, maxit=2000, prec="fp32", project_rhs=False,
              return_sigma=False, stream=None, sigma0=None):
        """u (mean zero) with div(a grad u) = f; returns (u, info[, sigma]).  sigma0
        (same shape and place as f): start from this density (PM_SOLVE_INITIAL_GUESS)."""
        prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        dev = _is_device(f)
        flags = ((PM_SOLVE_PROJECT_RHS if project_rhs else 0) | (PM_SOLVE_DEVICE_PTRS if dev else 0)
                 | (PM_SOLVE_INITIAL_GUESS if sigma0 is not None else 0))
        want_sig = return_sigma or sigma0 is not None
        if dev:
            import torch
            nrhs = f.numel() // self.N
            u = torch.empty_like(f)
            sig = torch.empty_like(f) if want_sig else None
            if sigma0 is not None:
                sig.copy_(sigma0.reshape(f.shape))
                torch.cuda.current_stream(f.device).synchronize()   # before a caller's stream
            st = C.c_void_p(stream if stream is not None else
                            torch.cuda.current_stream(f.device).cuda_stream)
        else:
            f = np.ascontiguousarray(f, dtype=np.float64)
            nrhs = f.size // self.N
            u = np.empty_like(f)
            sig = np.empty_like(f) if want_sig else None
            if sigma0 is not None:
                sig[...] = np.asarray(sigma0, dtype=np.float64).reshape(f.shape)
            st = C.c_void_p(stream)
        infos = (PmSolveInfo * nrhs)()
        check(_lib.lib().pm_solve(self.handle, ptr(f), ptr(u), nrhs, float(tol), int(maxit),
                                  prec, flags, ptr(sig), infos, st), "pm_solve")
        out = (u, list(infos))
        return out + (sig,) if return_sigma else out


class BoundaryValueProblem:
    """pm_bvp_*: the Neumann (Sec. 5.2) or, for constant a, Dirichlet (Sec. 5.3)
    boundary-value system of an open surface; kind "neumann" or "dirichlet".

    surface: a Surface built from the open surface's patches, with its coefficient set.
    curves: boundary curves, each with attributes M, F (edge nodes and oversampling
    factor), x, d1, d2, nu [M, 3] (point, dgamma/dt, d2gamma/dt2, binormal at
    t_k = 2 pi (k + 1/2) / M), xo, nuo [F M, 3], speedo [F M] (point, binormal and
    |dgamma/dt| at t_j = 2 pi j / (F M)); edge_a [Me], over_a [Fo]: a at the edge nodes
    and the oversampled points; edge_patch [Me], edge_uv [Me, 2]: each edge node's
    patch and reference coordinates on that patch's edge."""

    KINDS = {"neumann": 0, "dirichlet": 1}

    def __init__(self, surface: "Surface", curves, edge_a, over_a, edge_patch, edge_uv,
                 kind: str = "neumann"):
        cat = lambda name: np.ascontiguousarray(                     # noqa: E731
            np.concatenate([np.asarray(getattr(c, name), np.float64).reshape(-1) for c in curves]))
        self.surface = surface
        self.Me = int(sum(c.M for c in curves))
        self._keep = dict(
            M=np.ascontiguousarray([c.M for c in curves], dtype=np.int32),
            F=np.ascontiguousarray([c.F for c in curves], dtype=np.int32),
            x=cat("x"), d1=cat("d1"), d2=cat("d2"), nu=cat("nu"),
            a=_f64(edge_a, self.Me), patch=np.ascontiguousarray(edge_patch, dtype=np.int32),
            uv=_f64(edge_uv, 2 * self.Me), xo=cat("xo"), nuo=cat("nuo"), so=cat("speedo"),
            ao=np.ascontiguousarray(over_a, dtype=np.float64))
        k = self._keep
        h = C.c_void_p()
        self.handle = None
        check(_lib.lib().pm_bvp_create(surface.handle, self.KINDS[kind], len(curves), ptr(k["M"]),
                                       ptr(k["F"]), ptr(k["x"]), ptr(k["d1"]), ptr(k["d2"]),
                                       ptr(k["nu"]), ptr(k["a"]), ptr(k["patch"]), ptr(k["uv"]),
                                       ptr(k["xo"]), ptr(k["nuo"]), ptr(k["so"]), ptr(k["ao"]),
                                       C.byref(h)), "pm_bvp_create")
        self.handle = h
        self.kind = kind

    def apply(self, sigma, mu):
        sigma = _f64(sigma, self.surface.N)
        mu = _f64(mu, self.Me)
        out_s, out_e = np.empty(self.surface.N), np.empty(self.Me)
        check(_lib.lib().pm_bvp_apply(self.handle, ptr(sigma), ptr(mu), ptr(out_s), ptr(out_e)),
              "pm_bvp_apply")
        return out_s, out_e

    def solve(self, f, f_gamma, tol=1e-12, maxit=1000):
        """(u [N], info, sigma [N], mu [Me])."""
        f = _f64(f, self.surface.N)
        fg = _f64(f_gamma, self.Me)
        u, sig, mu = np.empty(self.surface.N), np.empty(self.surface.N), np.empty(self.Me)
        info = PmSolveInfo()
        check(_lib.lib().pm_bvp_solve(self.handle, ptr(f), ptr(fg), float(tol), int(maxit),
                                      ptr(u), ptr(sig), ptr(mu), C.byref(info)), "pm_bvp_solve")
        return u, info, sig, mu

    def close(self):
        if self.handle:
            _lib.lib().pm_bvp_destroy(self.handle)
            self.handle = None


NeumannBVP = BoundaryValueProblem      # the default kind


def solve_multi(surfaces, rhs, tol=1e-10, maxit=2000, project_rhs=False, stream=None):
    """Solve several operators' systems in one lockstep batch (pm_solve_multi).

    surfaces: list of Surface (distinct, one context); rhs: list of arrays, rhs[k] of
    shape [nrhs_k, N_k] (or [N_k]) -- numpy (host) or CUDA torch tensors (all device or
    all host).  Returns (list of u with the shapes of rhs, list of info per instance)."""
    n = len(surfaces)
    if n != len(rhs) or n == 0:
        raise ValueError("one right-hand-side array per surface")
    dev = _is_device(rhs[0])
    fs, us, nr = [], [], []
    for s, f in zip(surfaces, rhs):
        if dev:
            import torch
            f = f.contiguous().to(torch.float64)
            k = f.numel() // s.N
            u = torch.empty_like(f)
        else:
            f = np.ascontiguousarray(f, dtype=np.float64)
            k = f.size // s.N
            u = np.empty_like(f)
        if k * s.N != (f.numel() if dev else f.size) or k < 1:
            raise ValueError("right-hand sides must be [nrhs, N] of their surface")
        fs.append(f)
        us.append(u)
        nr.append(k)
    ops = (C.c_void_p * n)(*[s.handle.value for s in surfaces])
    fp = (C.c_void_p * n)(*[ptr(f).value for f in fs])
    up = (C.c_void_p * n)(*[ptr(u).value for u in us])
    nrc = (C.c_int * n)(*nr)
    infos = (PmSolveInfo * sum(nr))()
    flags = (PM_SOLVE_PROJECT_RHS if project_rhs else 0) | (PM_SOLVE_DEVICE_PTRS if dev else 0)
    if dev and stream is None:
        import torch
        stream = torch.cuda.current_stream(fs[0].device).cuda_stream
    check(_lib.lib().pm_solve_multi(ops, n, nrc, fp, up, float(tol), int(maxit), PM_PREC_FP32,
                                    flags, infos, C.c_void_p(stream)), "pm_solve_multi")
    out_info, c = [], 0
    for k in nr:
        out_info.append(list(infos[c:c + k]))
        c += k
    return us, out_info


class Server:
    """pm_server: continuous batching of solve requests over many operators."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int, max_batch: int = 64, n_workers: int = 4):
        h = C.c_void_p()
        check(_lib.lib().pm_server_create(ctx.handle, int(hbm_budget_bytes), int(max_batch),
                                          int(n_workers), C.byref(h)), "pm_server_create")
        self.handle = h
        self._sizes = {}

    def submit(self, op: Surface, f, tol=1e-8, prec="fp32"):
        f = _f64(f, op.N)
        t = C.c_ulonglong()
        prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        check(_lib.lib().pm_server_submit(self.handle, op.handle, ptr(f), float(tol), prec,
                                          C.byref(t)), "pm_server_submit")
        self._sizes[t.value] = op.N
        return t.value

    def submit_desc(self, geometry_id: int, coeff_id: int, surface, a, grad_a, f, tol=1e-8,
                    prec="fp32", opts=None):
        """Submit a request on an operator the server builds (or reuses) itself from a
        surface fixture (npatch, p, nodes, normals, tangents, curvature, weights) and a
        coefficient, keyed by the caller's geometry and coefficient ids."""
        N = surface.npatch * surface.p ** 2
        arrs = [_f64(surface.nodes, 3 * N), _f64(surface.normals, 3 * N),
                _f64(surface.tangents, 6 * N), _f64(surface.curvature, N),
                _f64(surface.weights, N), _f64(a, N),
                None if grad_a is None else _f64(grad_a, 3 * N)]
        d = _lib.PmOperatorDesc(int(geometry_id), int(coeff_id), int(surface.npatch),
                                int(surface.p), *[ptr(x) for x in arrs],
                                C.pointer(opts) if opts is not None else None)
        f = _f64(f, N)
        t = C.c_ulonglong()
        prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        check(_lib.lib().pm_server_submit_desc(self.handle, C.byref(d), ptr(f), float(tol), prec,
                                               C.byref(t)), "pm_server_submit_desc")
        self._sizes[t.value] = N
        return t.value

    def poll(self, ticket):
        d = C.c_int()
        check(_lib.lib().pm_server_poll(self.handle, C.c_ulonglong(ticket), C.byref(d)),
              "pm_server_poll")
        return bool(d.value)

    def wait(self, ticket, timeout_ms=-1):
        """(u, info, latency_seconds) of a finished request."""
        u, info, t = self.wait_ex(ticket, timeout_ms)
        return u, info, t["latency_s"]

    def wait_ex(self, ticket, timeout_ms=-1):
        """(u, info, times) of a finished request; times holds latency_s, build_s
        (building its operator while it waited), solve_s and queue_s."""
        u = np.empty(self._sizes[ticket])
        info = PmSolveInfo()
        tm = _lib.PmRequestTimes()
        st = _lib.lib().pm_server_wait_ex(self.handle, C.c_ulonglong(ticket), ptr(u),
                                          C.byref(info), C.byref(tm), int(timeout_ms))
        if st != _lib.PM_ERR_TIMEOUT:
            self._sizes.pop(ticket, None)
        check(st, "pm_server_wait")
        return u, info, {f: getattr(tm, f) for f, _ in tm._fields_}

    def configure(self, max_batch: int, active_workers: int):
        """Batch limit and number of working workers for batches formed from now on."""
        check(_lib.lib().pm_server_configure(self.handle, int(max_batch), int(active_workers)),
              "pm_server_configure")

    def stats(self):
        b, s, m = C.c_longlong(), C.c_longlong(), C.c_longlong()
        used = C.c_size_t()
        check(_lib.lib().pm_server_stats(self.handle, C.byref(b), C.byref(s), C.byref(m),
                                         C.byref(used)), "pm_server_stats")
        nb, res, mar, nop = C.c_longlong(), C.c_size_t(), C.c_size_t(), C.c_int()
        check(_lib.lib().pm_server_stats_ex(self.handle, C.byref(nb), C.byref(res), C.byref(mar),
                                            C.byref(nop)), "pm_server_stats_ex")
        return {"batches": b.value, "solved": s.value, "max_batch": m.value,
                "bytes_in_use": used.value, "builds": nb.value, "margin_bytes": mar.value,
                "operators": nop.value}

    def close(self):
        if self.handle:
            _lib.lib().pm_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
