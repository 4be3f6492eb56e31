"""Benchmark of the parametrix hot path on one GB300 (or N independent replicas).

Default workload: the 98,304-node torus (R = 2, r = 0.7, 64 x 24 patches of
8 x 8 nodes) with a = exp(0.3 cos(theta) sin(2 phi)) and f = cos(3 phi) sin(theta)
projected to mean zero.  One step is one full solve of div(a grad u) = f to a
relative residual of 1e-10 (so that u matches a plain float64 GPU solve to well
within 1e-8; the line reports the measured difference): device GMRES whose
operator applies use the Chebyshev FMM (tensor-core M2L) plus the float32
near-field correction, float-float true residuals, u = K~ sigma in float-float
and the mean projection.  The float-float sums read the operator's float-float
matrices, stored in HBM once per operator before the timed region (their build
time and size are reported; --no-store-ff evaluates the pairs instead, and the
line also reports that step's time).  --workload ellipsoid_9600 times the 9,600-node
ellipsoid with direct float32 applies instead.  The near field is built once
per surface, before the timed region (its time is reported).  Inputs are
resident in HBM; L2 is flushed between steps.

Prints one JSON line (rank 0).  --impl reference times the float64 CPU oracle
(every host core, one process per core) on a bounded sample of the same
workload instead.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "R-apply Gpairs/s; solves/s at 1e-8 rel err vs plain GPU solve; p50/p99 latency"
UNIT = "Gpairs/s"
FLOPS_PER_PAIR_R = 26      # variable-a remainder pair (algorithmic count)
FLOPS_PER_PAIR_K = 10      # parametrix pair
M2L_FLOPS_PER_BOX_PAIR = 2 * 9 * 512 * 512   # remainder M2L, 9 kernels on 8^3-point grids
FP32_LANES_PER_SM = 128    # FP32 lanes of one sm_100-family SM
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# of the current kernel versions on a workload; set to None whenever the kernel changes
# until it is captured again.
TRAFFIC_BYTES = {("k_direct_R32", "ellipsoid_9600"): 625408,
                 ("k_sym_ff_R", "ellipsoid_9600"): 1849856,
                 ("k_sym_ff_K", "ellipsoid_9600"): 356608,
                 ("k_sym_ff_R", "torus_98304"): 567848192,
                 ("k_sym_ff_K", "torus_98304"): 548400640,
                 ("k_tc_gemm", "torus_98304"): 446360320,
                 ("k_fmm_p2p", "torus_98304"): 6932992,
                 # stored-matrix GEMVs: captured on the 9,600-node ellipsoid, scaled to the
                 # torus by entries (row layout) and tiles (symmetric layout), since their
                 # traffic per entry does not depend on N (None until captured)
                 ("k_ffmat_gemv", "ellipsoid_9600"): 556227840,
                 ("k_ffmat_symK_gemv", "ellipsoid_9600"): 287151616,
                 ("k_ffmat_gemv", "torus_98304"): 58324716356,
                 ("k_ffmat_symK_gemv", "torus_98304"): 29752534596}
SYM_PARTIAL_CAP = 1024 ** 3             # the library's cap on symmetric-sum partial slices
DEFAULT_PREC = {"torus_98304": "fmm"}   # operator precision of the solve step per workload


def _measured_peaks():
    """HBM GB/s and bf16 TFLOP/s measured on the GB300s (generated file)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        return {"hbm_gbs": m.get("hbm_gbs"), "bf16_tflops": m.get("bf16_tflops"),
                "bf16_tflops_sustained": m.get("bf16_tflops_sustained"),
                "basis": "of measured (MEASURED_PEAKS.json)"}
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "basis": "of fallback (no MEASURED_PEAKS.json)"}


def _max_sm_mhz(device_index=0):
    """The GPU's maximum SM clock read from the device (nvidia-smi), else None."""
    try:
        r = subprocess.run(["nvidia-smi", f"--id={device_index}",
                            "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                           capture_output=True, text=True, timeout=30)
        return float(r.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return None


def fp32_peak_tflops(sms, mhz):
    """Non-tensor float32 peak from unit counts: SMs x FP32 lanes x 2 flops (FMA) x clock."""
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle leg
# The float64 oracle's remainder apply, timed on a bounded sample of target rows: one
# process per host core (spawned, each with one BLAS thread), every process evaluating
# disjoint row chunks of the smooth sum over all N sources for a fixed wall time, plus
# the near-field correction of a few rows (built once, untimed; its apply is timed).
_ORC = {}


def _orc_init(workload):
    import numpy as np
    from oracle.operator import Discretization
    from workloads import make_workload
    d = Discretization.from_workload(make_workload(workload))
    _ORC["d"] = d
    _ORC["sigma"] = np.random.default_rng(0).standard_normal(d.N)


def _orc_rows(task):
    import numpy as np
    rank, nproc, seconds, chunk = task
    d, sigma = _ORC["d"], _ORC["sigma"]
    N = d.N
    rows_done, k = 0, rank
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        r0 = (k * 7919 * chunk) % max(1, N - chunk)
        d.smooth_apply("R", sigma, np.arange(r0, min(N, r0 + chunk)), chunk=chunk)
        rows_done += min(N, r0 + chunk) - r0
        k += nproc
    return rows_done, time.perf_counter() - t0


class OracleRunner:
    """A pool of oracle processes for one workload (spawned: no process forks after a
    CUDA context exists) and the near-field corrections of a few sampled rows."""

    def __init__(self, workload: str, processes: int):
        import multiprocessing as mp
        import numpy as np
        from oracle.operator import Discretization, NearField
        from workloads import make_workload
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        self.workload, self.P = workload, max(1, processes)
        d = Discretization.from_workload(make_workload(workload))
        self.N = d.N
        self.chunk = 32 if d.N > 50000 else 128
        rng = np.random.default_rng(0)
        self.sigma = rng.standard_normal(d.N)
        self.near_rows = [int(i) for i in rng.integers(0, d.N, 8)]
        self.nf = NearField(d, rows=self.near_rows)          # one-time corrections, untimed
        self.pool = mp.get_context("spawn").Pool(self.P, initializer=_orc_init,
                                                 initargs=(workload,))

    def rate(self, seconds: float, processes: int | None = None):
        """(Gpairs/s, description) of the oracle's remainder apply on `processes` cores."""
        P = self.P if processes is None else max(1, min(processes, self.P))
        res = self.pool.map(_orc_rows, [(r, P, seconds, self.chunk) for r in range(P)])
        rows = sum(r[0] for r in res)
        wall = max(r[1] for r in res)
        ts = time.perf_counter()
        self.nf.apply("R", self.sigma, self.near_rows)
        t_near = (time.perf_counter() - ts) / len(self.near_rows)
        t_row = wall / rows + t_near / P        # per-row time with P cores working
        desc = (f"{rows} target rows of {self.workload} (float64 smooth sum over all {self.N} "
                f"sources, numpy) on {P} process(es) x {seconds:.1f} s + near-field "
                f"correction of {len(self.near_rows)} rows")
        return self.N / t_row / 1e9, desc

    def close(self):
        self.pool.terminate()
        self.pool.join()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def reference_line(args, vals, desc, cores):
    """The reference arm's JSON line: the oracle's rate (mean over the timed steps)."""
    v = statistics.mean(vals[args.warmup:]) if len(vals) > args.warmup else vals[-1]
    return {
        "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "impl": "reference",
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_oracle_subprocess(workload: str, seconds: float):
    """cpu_baseline of the GPU arm: the oracle on every host core and on one core, in a
    fresh process that never touches the GPU."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-leg",
                        "--workload", workload, "--oracle-seconds", str(seconds)],
                       capture_output=True, text=True, env=env, timeout=900)
    for ln in r.stdout.splitlines()[::-1]:
        if ln.startswith("{"):
            return json.loads(ln)
    raise RuntimeError("oracle leg failed: " + r.stdout[-2000:] + r.stderr[-2000:])


# ----------------------------------------------------------------------------- GPU arm
PHASES = ["prep", "direct_R", "direct_K", "near", "vec", "accurate_R", "fmm_m2l_gemm",
          "fmm_p2p", "accurate_K"]


def max_over_ranks(value, world, device=None):
    """The largest value over the ranks of the job (a replica job takes as long as
    its slowest replica); the value itself for one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, pairs_per_step, ms_per_step):
    """Whole-job smooth-sum pairs per second (Gpairs/s): every replica runs the same
    step, so the job evaluates world * pairs_per_step pairs per step time."""
    return world * pairs_per_step / (ms_per_step * 1e-3) / 1e9


def _nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def _nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def _phase_totals(surf, reset=True):
    out = {}
    for k, nm in enumerate(PHASES):
        out[nm] = surf.profile_read(k)
    out["launches_all"] = surf.profile_read(len(PHASES))     # every kernel the library launched
    surf.profile_read(0, reset=reset)
    return out


def _alu_roofline(kernel, flops_per_launch, ms_per_launch, peak, step_share, traffic, **extra):
    ach = flops_per_launch / (ms_per_launch * 1e-3) / 1e12
    d = {"bound": "alu", "kernel": kernel, "achieved": round(ach, 3), "peak": round(peak, 2),
         "unit": "TFLOP/s", "frac": round(ach / peak, 4), "traffic": traffic,
         "kernel_ms": round(ms_per_launch, 5), "step_time_share": round(step_share, 4)}
    d.update(extra)
    return d


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_2401_12501_gb300 as pm
    from workloads import make_workload

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prec = args.prec or DEFAULT_PREC.get(args.workload, "fp32")
    wl = make_workload(args.workload)
    N = wl.N
    pairs = float(N) * N
    ctx = pm.Context(local_rank)
    gpu_name, sms = ctx.info()
    max_mhz = _max_sm_mhz(local_rank)
    peak_fp32 = fp32_peak_tflops(sms, max_mhz or 2070.0)
    mp_peaks = _measured_peaks()
    t0 = time.perf_counter()
    surf = pm.Surface.from_fixture(ctx, wl.surface)
    t_build = time.perf_counter() - t0
    surf.set_coeff(wl.coeff.a, wl.coeff.grad_a)
    nblk = surf.info()[1]
    # launch shapes picked by the autotuner (untimed, before warm-up): the FMM's octree
    # depth for FMM applies, the float32 sums' shape otherwise
    tune = (surf.autotune(nrhs=1, prec=prec, reps=3 if prec == "fmm" else 5)
            if not args.no_autotune else _builtin(surf))
    fmm = surf.fmm_stats() if prec == "fmm" else None
    # float-float matrices of both smooth kernels kept in HBM (pm_surface_store_ff): the
    # refinement residual and u = K sigma then stream them instead of evaluating pairs
    store = None
    if not args.no_store_ff:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        t0 = time.perf_counter()
        try:
            surf.store_ff("RK")
            t_store = time.perf_counter() - t0
            store = {"kernels": surf.stored_ff(), "build_s": round(t_store, 4),
                     "device_bytes": int(free0 - torch.cuda.mem_get_info(dev)[0])}
        except pm._lib.PmError as e:
            store = {"unavailable": str(e)}
    stored = bool(store and store.get("kernels"))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    f_h = torch.from_numpy(wl.f.copy()).pin_memory()
    f_d = f_h.to(dev)
    tol = args.tol

    def step():
        return surf.solve(f_d, tol=tol, prec=prec)

    # the accuracy the timed solves reach: u against a plain float64 solve (float64
    # operator applies and Krylov basis, direct sums) of the same system to 1e-12
    t0 = time.perf_counter()
    u_ref, _ = surf.solve(wl.f, tol=1e-12, prec="fp64")
    t_fp64 = time.perf_counter() - t0
    u_chk, _ = surf.solve(wl.f, tol=tol, prec=prec)
    wq = wl.surface.weights
    err_vs_fp64 = float(np.sqrt(np.dot(wq, (u_chk - u_ref) ** 2) / np.dot(wq, u_ref ** 2)))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    infos = []
    surf.profile_read(len(PHASES), reset=True)          # zero the launch counter
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))                   # evict L2 between timed steps
            evs[k][0].record(stream)
            _, info = step()
            evs[k][1].record(stream)
            infos.append(info[0])
        torch.cuda.synchronize()
    launches_timed = surf.profile_read(len(PHASES))[1]
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    clocks = clk.summary()

    # phase split: the same steps again with per-phase events recorded by the library
    # on the launching stream (event records cannot sit inside the graph-driven GMRES
    # cycle, so this pass issues its launches from the host; the kernels are the same)
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    surf.profile(True)
    surf.profile_read(0, reset=True)
    _nvtx_push("solve_profiled_pass")           # ncu --nvtx-include selects these launches
    for k in range(args.steps):
        flush.fill_(float(k))
        pev[k][0].record(stream)
        step()
        pev[k][1].record(stream)
    torch.cuda.synchronize()
    _nvtx_pop()
    surf.profile(False)
    ph = _phase_totals(surf)
    prof_total_ms = sum(a.elapsed_time(b) for a, b in pev)
    ms_per_step = total_ms / args.steps
    # operator applies per solve: one R apply per Arnoldi step, one accurate R apply
    # per refinement, one accurate K apply for u
    it = statistics.mean(i.iterations for i in infos)
    rf = statistics.mean(i.refinements for i in infos)
    applies = it + rf + 1
    value = job_throughput(world, applies * pairs, ms_per_step)
    solves_per_s = world * 1e3 / ms_per_step
    per_step = lambda nm: (ph[nm][0] / args.steps, ph[nm][1] / args.steps)   # noqa: E731
    acc_R_ms, acc_R_n = per_step("accurate_R")
    acc_K_ms, acc_K_n = per_step("accurate_K")
    fast_R_ms, fast_R_n = per_step("direct_R")
    # operator applies that did work: the profiled pass issues a cycle's steps from the
    # host in chunks of 4 between reads of the done flag, so up to 3 launches a cycle
    # after convergence return at once; per-launch times divide by the applies with work
    # (one per Arnoldi step and one per residual update after the first refinement)
    fast_R_eff = it + max(0.0, rf - 1)
    actual_pairs = ((fast_R_eff * fmm["p2p_pairs"] if fmm else fast_R_eff * pairs)
                    + (acc_R_n + acc_K_n) * pairs)

    # end-to-end through the C ABI with host (pinned) buffers: f in, u out
    for _ in range(2):
        surf.solve(f_h.numpy(), tol=tol, prec=prec)
    torch.cuda.synchronize()
    n_e2e = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        surf.solve(f_h.numpy(), tol=tol, prec=prec)
    e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e_value = job_throughput(world, applies * pairs, e2e_s * 1e3)

    # per-launch kernel times: every operator apply of the step, back to back on the
    # launching stream, with per-phase events (the host enqueues ahead of the device, so
    # no launch gap falls inside an event pair, unlike the host-issued profiled pass;
    # no launch there returns early); the shares stay those of the profiled pass
    reps = 10
    sig_k = torch.from_numpy(np.random.default_rng(5).standard_normal(N) + 1.0).to(dev)

    def per_launch(fn, names):
        fn()
        torch.cuda.synchronize()
        surf.profile(True)
        surf.profile_read(0, reset=True)
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        surf.profile(False)
        p2 = _phase_totals(surf)
        return {nm: p2[nm][0] / p2[nm][1] for nm in names if p2[nm][1]}

    klt = {}
    in_step = {}
    if fmm:
        # in the step the far field runs on a second stream beside the P2P; the kernels'
        # own times come from applies with every launch on one stream (knob fmm_streams)
        in_step = per_launch(lambda: surf.apply_R(sig_k, prec),
                             ["direct_R", "fmm_p2p", "fmm_m2l_gemm"])
        surf.set_knobs(fmm_streams=1)
    klt.update(per_launch(lambda: surf.apply_R(sig_k, prec), ["direct_R", "fmm_p2p", "fmm_m2l_gemm"]))
    if fmm:
        surf.set_knobs(fmm_streams=0)
    klt.update(per_launch(lambda: surf.apply_R(sig_k, "ff"), ["accurate_R"]))
    klt.update(per_launch(lambda: surf.apply_K(sig_k, "ff"), ["accurate_K"]))

    # the same step with the float-float sums evaluated pair by pair (matrices released)
    computed_ff = None
    if stored:
        surf.store_ff("")
        for _ in range(2):
            step()
        n_cmp = max(3, min(args.steps, 5))
        cev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(n_cmp)]
        torch.cuda.synchronize()
        for k in range(n_cmp):
            flush.fill_(float(k))
            cev[k][0].record(stream)
            step()
            cev[k][1].record(stream)
        torch.cuda.synchronize()
        computed_ff = {"ms_per_step": round(sum(a.elapsed_time(b) for a, b in cev) / n_cmp, 4),
                       "steps": n_cmp,
                       "note": "the float-float residual and representation sums evaluated pair "
                               "by pair (symmetric tile-pair kernels) instead of read from the "
                               "stored matrices; untimed build excluded either way"}

    # rooflines of the step's kernels, per launch from the back-to-back applies
    nt = -(-N // 128)
    sym = N >= 256 and nt * N * 8 <= SYM_PARTIAL_CAP
    ff_name = "k_sym_ff" if sym else "k_direct_ff"
    roofs = {}
    hbm_peak = mp_peaks["hbm_gbs"]
    ld = -(-N // 128) * 128
    if stored and acc_R_n:
        byt = N * ld * 6 + 8 * ld + 8 * N
        ms = klt["accurate_R"]
        ach = byt / (ms * 1e-3) / 1e9
        roofs["accurate_R"] = {
            "bound": "hbm", "kernel": "k_ffmat_gemv (stored float-float remainder matrix, "
                                      "6 bytes an entry, float-float GEMV)",
            "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(ach / hbm_peak, 4),
            "traffic": TRAFFIC_BYTES.get(("k_ffmat_gemv", args.workload)),
            "algorithmic_bytes": byt, "kernel_ms": round(ms, 5),
            "peak_basis": "HBM copy bandwidth " + mp_peaks["basis"],
            "step_time_share": round(acc_R_ms * args.steps / prof_total_ms, 4)}
    if stored and acc_K_n:
        ntk = -(-N // 128)
        sym_k = N >= 256 and ntk * N * 8 <= SYM_PARTIAL_CAP
        mat = ntk * (ntk + 1) // 2 * 128 * 128 * 6 if sym_k else N * ld * 6
        byt = mat + 8 * ld + 8 * N
        ms = klt["accurate_K"]
        ach = byt / (ms * 1e-3) / 1e9
        roofs["accurate_K"] = {
            "bound": "hbm",
            "kernel": ("k_ffmat_symK_gemv (stored symmetric float-float parametrix matrix, "
                       "upper-triangle tiles; row and column sums per tile)" if sym_k else
                       "k_ffmat_gemv (stored float-float parametrix matrix)"),
            "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(ach / hbm_peak, 4),
            "traffic": TRAFFIC_BYTES.get(("k_ffmat_symK_gemv" if sym_k else "k_ffmat_gemv_K",
                                          args.workload)),
            "algorithmic_bytes": byt, "kernel_ms": round(ms, 5),
            "peak_basis": "HBM copy bandwidth " + mp_peaks["basis"],
            "step_time_share": round(acc_K_ms * args.steps / prof_total_ms, 4)}
    if acc_R_n and not stored:
        roofs["accurate_R"] = _alu_roofline(
            ff_name + "<R> (float-float remainder sum" + (", each unordered pair once)" if sym else ")"),
            FLOPS_PER_PAIR_R * pairs, klt["accurate_R"], peak_fp32, acc_R_ms * args.steps / prof_total_ms,
            TRAFFIC_BYTES.get((ff_name + "_R", args.workload)),
            note="algorithmic flops of the float64-class sum (26 per ordered pair); float-float "
                 "arithmetic costs ~10 float32 instructions per algorithmic flop (274 per "
                 "unordered pair), so the sum is bound by FP32 instruction issue")
    if acc_K_n and not stored:
        roofs["accurate_K"] = _alu_roofline(
            ff_name + "<K> (float-float parametrix sum)", FLOPS_PER_PAIR_K * pairs,
            klt["accurate_K"], peak_fp32, acc_K_ms * args.steps / prof_total_ms,
            TRAFFIC_BYTES.get((ff_name + "_K", args.workload)))
    if fmm and ph["fmm_m2l_gemm"][1]:
        g_ms = klt["fmm_m2l_gemm"]
        alg = M2L_FLOPS_PER_BOX_PAIR * fmm["m2l_box_pairs"]
        peak_tc = mp_peaks["bf16_tflops_sustained"] or mp_peaks["bf16_tflops"]
        ach = alg / (g_ms * 1e-3) / 1e12
        roofs["fmm_m2l_gemm"] = {
            "bound": "tensor", "kernel": "k_tc_gemm (FMM M2L, float16 parts, tcgen05)",
            "achieved": round(ach, 2), "peak": peak_tc, "unit": "TFLOP/s",
            "frac": round(ach / peak_tc, 4), "traffic": TRAFFIC_BYTES.get(("k_tc_gemm", args.workload)),
            "kernel_ms": round(g_ms, 5), "executed_flops_factor": 3,
            "executed_frac": round(3 * ach / peak_tc, 4),
            "peak_basis": "float16 dense rate = bf16 rate (nominal ratio 1); sustained bf16 "
                          + mp_peaks["basis"],
            "step_time_share": round(ph["fmm_m2l_gemm"][0] / prof_total_ms, 4)}
        if "fmm_m2l_gemm" in in_step:
            roofs["fmm_m2l_gemm"]["kernel_ms_in_step"] = round(in_step["fmm_m2l_gemm"], 5)
    if fmm and ph["fmm_p2p"][1]:
        p_ms = klt["fmm_p2p"]
        roofs["fmm_p2p"] = _alu_roofline(
            "k_fmm_p2p<R> (FMM adjacent-leaf float32 sums)", FLOPS_PER_PAIR_R * fmm["p2p_pairs"],
            p_ms, peak_fp32, ph["fmm_p2p"][0] / prof_total_ms,
            TRAFFIC_BYTES.get(("k_fmm_p2p", args.workload)))
        if "fmm_p2p" in in_step:
            roofs["fmm_p2p"]["kernel_ms_in_step"] = round(in_step["fmm_p2p"], 5)
            roofs["fmm_p2p"]["timing"] = (
                "kernel_ms: the P2P alone (every launch of the apply on one stream, back to "
                "back); kernel_ms_in_step: its event time inside the step's applies, where the "
                "far field (P2M, M2M, M2L GEMM, L2L) runs beside it on a higher-priority "
                "stream and shares its SMs; step_time_share from the latter")
    if not fmm and fast_R_n:
        roofs["direct_R"] = _alu_roofline(
            "k_direct_R32 (float32 remainder sum)", FLOPS_PER_PAIR_R * pairs, klt["direct_R"],
            peak_fp32, fast_R_ms * args.steps / prof_total_ms,
            TRAFFIC_BYTES.get(("k_direct_R32", args.workload)))
    dom = max(roofs, key=lambda k: roofs[k]["step_time_share"]) if roofs else None
    peak_basis = (f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                  f"{max_mhz or 2070.0:g} MHz (unit counts; SM count from the device, clock "
                  + ("from nvidia-smi)" if max_mhz else "assumed: nvidia-smi unavailable)"))
    for r in roofs.values():
        if r["bound"] == "alu":
            r["peak_basis"] = peak_basis
    step_desc = ("one solve of div(a grad u) = f to relative residual "
                 f"{tol:g}: device GMRES with "
                 + ("Chebyshev-FMM applies (tensor-core M2L)" if prec == "fmm" else
                    "float32 direct-sum applies")
                 + " + float32 near field, float-float refinement residuals, u = K sigma in "
                   "float-float"
                 + (" (both read from the operator's stored float-float matrices)" if stored
                    else "") + ", mean projection")
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32",
        "dtype_detail": ("f32 operator applies (FMM: float16-part tensor-core M2L with float32 "
                         "accumulation; float32 P2P, P2M/L2P and near field) + float-float "
                         "residuals/representation + f64 Krylov basis" if prec == "fmm" else
                         "f32 operator applies (compensated sums) + float-float residuals/"
                         "representation + f64 Krylov basis and near field"),
        "data": "synthetic", "impl": "gb300",
        "config": {"workload": args.workload, "N": N, "gpu": gpu_name, "operator_prec": prec,
                   "step": step_desc,
                   "value_definition": "equivalent smooth-sum pairs per second over the solve "
                                       "step = (Arnoldi steps + refinements + 1) * N^2 / time",
                   "near_blocks": nblk, "near_build_s": round(t_build, 3),
                   "stored_ff_matrices": store,
                   "autotune": {"knobs": {k: v for k, v in tune["knobs"].items() if v},
                                "apply_ms": _r(tune["best_ms"], 4),
                                "builtin_apply_ms": _r(tune["default_ms"], 4),
                                "candidates": tune["candidates"]},
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "solves_per_s": round(solves_per_s, 3),
        "computed_ff_step": computed_ff,
        "actual_pairs_gpairs_per_s": round(world * actual_pairs / (ms_per_step * 1e-3) / 1e9, 3),
        "actual_pairs_definition": ("pairs evaluated pair by pair per step: FMM applies count "
                                    "their adjacent-leaf (P2P) pairs, accurate (float-float) "
                                    "applies N^2 (each pair's stored entry read once, or its "
                                    "kernel evaluated); the far field is not pairs" if fmm else
                                    "every apply evaluates (or reads the stored entry of) "
                                    "N^2 pairs"),
        "solve": {"iterations": it, "refinements": rf, "applies_per_solve": applies,
                  "operator_applies_with_work": fast_R_eff,
                  "residual_max": max(i.residual for i in infos),
                  "rel_err_vs_fp64_solve": err_vs_fp64, "fp64_solve_s": round(t_fp64, 3),
                  "profiled_ms_per_step": round(prof_total_ms / args.steps, 4),
                  "phase_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in ph.items()
                                        if k != "launches_all"},
                  "phase_launches_per_step": {k: v[1] / args.steps for k, v in ph.items()
                                              if k != "launches_all"}},
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": 8 * N,
                "d2h_bytes_per_step": 8 * N, "solves_per_s": round(world / e2e_s, 3)},
        "gpu_launches": int(launches_timed),
        "roofline": roofs.get(dom),
        "roofline_other": {k: v for k, v in roofs.items() if k != dom},
        "clocks": clocks,
    }
    if fmm:
        line["config"]["fmm"] = {
            "tree": fmm, "interp_points": "8^3 Chebyshev (first kind) per box",
            "leaf": "uniform-depth octree of occupied boxes, depth by a cost model / autotuner",
            "note": ("deviation from the config text (leaf <= 256 points, 6^3 points): 6^3 "
                     "points do not reach the 1e-5 apply tolerance, and at 8^3 points a "
                     "deeper tree (smaller leaves) costs more in M2L than it saves in P2P")}
    surf.close()
    ctx.close()
    return line


def _builtin(s):
    """The autotuner's report for the built-in launch shapes (used with --no-autotune)."""
    return {"knobs": s.knobs(), "best_ms": None, "default_ms": None,
            "candidates": 0, "cached": False, "key": "built-in"}


def _r(v, nd):
    return None if v is None else round(v, nd)


def run_ellipsoid(args, dev):
    """The 9,600-node ellipsoid solve with direct float32 applies (the whole solve
    step of the headline, on the smaller surface whose float32 sums dominate)."""
    sub = argparse.Namespace(**vars(args))
    sub.workload, sub.prec = "ellipsoid_9600", "fp32"
    ln = run_gpu(sub, 0, 1, dev.index or 0)
    keep = ("value", "unit", "ms_per_step", "solves_per_s", "solve", "e2e", "roofline",
            "roofline_other", "clocks", "gpu_launches")
    out = {k: ln[k] for k in keep}
    out["config"] = {k: ln["config"][k] for k in ("workload", "N", "step", "near_blocks",
                                                  "near_build_s", "autotune")}
    return out


def run_batched(args, dev):
    """24,576-node star with 8 coefficient fields and 64 right-hand sides (RHS r on
    field r mod 8): 8 operators on one geometry (one near-field build, 7 clones),
    solved one at a time, as per-field lockstep batches, and through the
    continuous-batching server with all 64 requests at once; plus all 64 RHS on
    one field (the most sharing one operator allows)."""
    import torch
    import paper_2401_12501_gb300 as pm
    from workloads import star_batch
    n_field, n_rhs = 8, 64
    s_surf, coeffs, F = star_batch(n_rhs=n_rhs, n_coeff=n_field)
    ctx = pm.Context(dev.index or 0)
    t0 = time.perf_counter()
    s0 = pm.Surface.from_fixture(ctx, s_surf)
    t_build = time.perf_counter() - t0
    s0.set_coeff(coeffs[0].a, coeffs[0].grad_a)
    # launch shapes picked by the autotuner (copied to the clones): one right-hand
    # side, 8 per field; the 64-RHS shape is tuned on its own below
    tune1 = s0.autotune(nrhs=1, prec="fp32", reps=3) if not args.no_autotune else _builtin(s0)
    tune8 = (s0.autotune(nrhs=n_rhs // n_field, prec="fp32", reps=3) if not args.no_autotune
             else _builtin(s0))
    t0 = time.perf_counter()
    ops = [s0] + [s0.clone() for _ in range(n_field - 1)]
    t_clone = time.perf_counter() - t0
    for k in range(1, n_field):
        ops[k].set_coeff(coeffs[k].a, coeffs[k].grad_a)
    Fd = torch.from_numpy(F).to(dev)
    field_rows = [list(range(k, n_rhs, n_field)) for k in range(n_field)]
    Fk = [Fd[rows].contiguous() for rows in field_rows]

    # one at a time (8 sample solves, one per field)
    ops[0].solve(Fd[0], tol=args.tol, prec="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(n_field):
        ops[k].solve(Fk[k][0], tol=args.tol, prec="fp32")
    torch.cuda.synchronize()
    t_plain = (time.perf_counter() - t0) / n_field

    # per-field lockstep batches, one field after another
    for k in range(n_field):
        ops[k].solve(Fk[k], tol=args.tol, prec="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = []
    for k in range(n_field):
        _, info = ops[k].solve(Fk[k], tol=args.tol, prec="fp32")
        res += [i.residual for i in info]
    torch.cuda.synchronize()
    t_fields = time.perf_counter() - t0

    # all 8 fields x 8 right-hand sides in one multi-instance lockstep batch: every
    # field's applies in the same launches, each GMRES cycle one CUDA graph
    # its launch shape (fields of a geometry per smooth-sum item = right-hand sides per
    # block / 8, blocks per SM) picked by timing a few candidates on the whole solve;
    # the per-field knobs are restored afterwards
    knobs0 = ops[0].knobs()
    multi_tune = {}
    for rbk, bps in ((8, 8), (16, 8), (16, 12), (32, 8)):
        if args.no_autotune and (rbk, bps) != (16, 8):
            continue
        ops[0].set_knobs(batch_rhs_per_block=rbk, batch_blocks_per_sm=bps)
        pm.solve_multi(ops, Fk, tol=args.tol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pm.solve_multi(ops, Fk, tol=args.tol)
        torch.cuda.synchronize()
        multi_tune[(rbk, bps)] = time.perf_counter() - t0
    best = min(multi_tune, key=multi_tune.get)
    ops[0].set_knobs(batch_rhs_per_block=best[0], batch_blocks_per_sm=best[1])
    pm.solve_multi(ops, Fk, tol=args.tol)
    torch.cuda.synchronize()
    reps_m = 3
    t0 = time.perf_counter()
    for _ in range(reps_m):
        _, minfo = pm.solve_multi(ops, Fk, tol=args.tol)
    torch.cuda.synchronize()
    t_multi = (time.perf_counter() - t0) / reps_m
    res += [i.residual for inf in minfo for i in inf]
    ops[0].set_knobs(**knobs0)

    # continuous-batching server, all 64 requests at t = 0 (operators overlap)
    F_host = [F[r] for r in range(n_rhs)]

    def serve_all(max_batch, n_workers):
        sv = pm.Server(ctx, hbm_budget_bytes=16 << 30, max_batch=max_batch, n_workers=n_workers)
        t0 = time.perf_counter()
        tickets = [sv.submit(ops[r % n_field], F_host[r], tol=args.tol) for r in range(n_rhs)]
        out = [sv.wait(t) for t in tickets]
        wall = time.perf_counter() - t0
        sv.close()
        return wall, max(o[1].residual for o in out)

    serve_all(64, 4)
    t_served, res_served = serve_all(64, 4)

    # all 64 right-hand sides on field 0
    tune64 = (ops[0].autotune(nrhs=n_rhs, prec="fp32", reps=3) if not args.no_autotune
              else _builtin(ops[0]))
    ops[0].solve(Fd, tol=args.tol, prec="fp32")
    torch.cuda.synchronize()
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        U, info = ops[0].solve(Fd, tol=args.tol, prec="fp32")
    torch.cuda.synchronize()
    t_one_field = (time.perf_counter() - t0) / reps
    for op in ops:
        op.close()
    knobs = lambda r: {"knobs": {k: v for k, v in r["knobs"].items() if v},
                       "apply_ms": _r(r["best_ms"], 3),
                       "builtin_apply_ms": _r(r["default_ms"], 3)}
    return {"workload": "star_24576: 8 coefficient fields a = 1 + 0.4 tanh(g) (seeds 0-7) x "
                        "64 right-hand sides (seeds 0-63), RHS r on field r mod 8",
            "N": s_surf.N, "near_build_s": round(t_build, 3),
            "clone_s_7_operators": round(t_clone, 3), "tol": args.tol,
            "plain_solves_per_s": round(1.0 / t_plain, 2),
            "batched_solves_per_s": round(n_rhs / t_fields, 2),
            "batched_form": "each field's 8 right-hand sides in one lockstep batched solve "
                            "(multi-RHS sums sharing each pair's geometry), fields one after "
                            "another",
            "speedup_vs_plain": round(t_plain * n_rhs / t_fields, 2),
            "multi_instance_solves_per_s": round(n_rhs / t_multi, 2),
            "multi_instance_form": "pm_solve_multi: the 8 operators' 64 right-hand sides in one "
                                   "lockstep GMRES, each Arnoldi step's float32 applies of all "
                                   "operators in one persistent smooth-sum launch over a work "
                                   "list + one near-field launch, each cycle one CUDA graph",
            "multi_instance_speedup_vs_plain": round(t_plain * n_rhs / t_multi, 2),
            "multi_instance_tuned": {"fields_per_item": best[0] // 8, "blocks_per_sm": best[1],
                                     "candidates_ms": {f"{k[0] // 8}x{k[1]}": round(v * 1e3, 2)
                                                       for k, v in multi_tune.items()}},
            "served_all_at_once_solves_per_s": round(n_rhs / t_served, 2),
            "one_field_64_rhs_solves_per_s": round(n_rhs / t_one_field, 2),
            "max_residual": max(max(res), res_served, max(i.residual for i in info)),
            "autotune": {"nrhs_1": knobs(tune1), "nrhs_8": knobs(tune8),
                         "nrhs_64": knobs(tune64)}}


def run_paper(args, dev):
    """The paper's own test problems (Sec. 7), a = 1: error of the solution against
    the exact one and time per solve at the finest resolution of each; the N-body
    accuracy test of the fast apply on the 58,752-node wavy torus (Sec. 6.2)."""
    import numpy as np
    import torch
    import paper_2401_12501_gb300 as pm
    from workloads import paper_problem
    ctx = pm.Context(dev.index or 0)
    out = {"tol": args.tol, "problems": {}}
    for name, precs in (("sphere_paper_6144", ("fp32",)), ("ellipsoid_paper_24576", ("fp32",)),
                        ("wavy_torus_58752", ("fp32", "fmm"))):
        wl, uex = paper_problem(name)
        t0 = time.perf_counter()
        s = pm.Surface.from_fixture(ctx, wl.surface)
        t_build = time.perf_counter() - t0
        s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
        w = wl.surface.weights
        fd = torch.from_numpy(wl.f.copy()).to(dev)
        row = {"N": wl.N, "near_build_s": round(t_build, 3), "description": wl.description}
        for prec in precs:
            s.solve(fd, tol=args.tol, prec=prec)
            torch.cuda.synchronize()
            reps = 3
            t0 = time.perf_counter()
            for _ in range(reps):
                u, info = s.solve(fd, tol=args.tol, prec=prec)
            torch.cuda.synchronize()
            t = (time.perf_counter() - t0) / reps
            u = u.cpu().numpy()
            row[prec] = {"solve_ms": round(t * 1e3, 3), "iterations": info[0].iterations,
                         "residual": info[0].residual,
                         "rel_l2_error_vs_exact": float(np.sqrt(np.dot(w, (u - uex) ** 2) /
                                                                np.dot(w, uex ** 2)))}
        if name == "wavy_torus_58752":
            sig = torch.from_numpy(wl.surface.nodes[:, 0] +
                                   np.random.default_rng(0).standard_normal(wl.N)).to(dev)
            nb = {}
            for part, key in ((pm.PM_PART_SMOOTH_K, "parametrix"), (pm.PM_PART_SMOOTH_R, "remainder")):
                ex = s.apply_part(part, sig, "ff").cpu().numpy()
                res = {}
                for prec in ("fmm", "fp32"):
                    y = s.apply_part(part, sig, prec)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    for _ in range(3):
                        y = s.apply_part(part, sig, prec)
                    torch.cuda.synchronize()
                    y = y.cpu().numpy()
                    res[prec] = {"ms": round((time.perf_counter() - t0) / 3 * 1e3, 3),
                                 "rel_l2_error_vs_float_float":
                                     float(np.linalg.norm(y - ex) / np.linalg.norm(ex))}
                nb[key] = res
            out["nbody_wavy_torus_58752"] = {"sigma": "x_1 + N(0,1) (seed 0)", **nb,
                                             "fmm_tree": s.fmm_stats()}
        out["problems"][name] = row
        s.close()
    return out


def run_bvp(args, dev):
    """Open-surface problems (Sec. 5): torus bands (R = 2, r = 0.7, theta in [0, n_band
    pi/8]), the manufactured Newtonian solution u = -1/|x - x0|; Neumann with
    a = exp(0.2 x + 0.3 z) and Fourier oversampling F = 16, Dirichlet with a = 1 and
    F = 32; edge nodes M per circle.  Reports the edge quadrature build, the float64
    GMRES solve to 1e-12 and u's error against the exact solution (Neumann: up to the
    additive constant)."""
    import numpy as np
    import paper_2401_12501_gb300 as pm
    from workloads.bvp import (band_coefficient, constant_band_coefficient, edge_a, edge_patches,
                               newtonian_dirichlet, newtonian_neumann, torus_band)
    ctx = pm.Context(dev.index or 0)
    out = {"problem": "Neumann (eq. NeuBVPsystem, a = exp(0.2 x + 0.3 z)) and Dirichlet "
                      "(eq. DirBVPsystem, a = 1); float64", "cases": {}}
    for kind, F in (("neumann", 16), ("dirichlet", 32)):
      for nb, nphi, p, M in ((2, 4, 8, 32), (4, 8, 8, 64), (8, 16, 8, 128)):
        os_ = torus_band(nb, nphi, p, M, F)
        co = band_coefficient(os_) if kind == "neumann" else constant_band_coefficient(os_)
        t0 = time.perf_counter()
        s = pm.Surface.from_fixture(ctx, os_.surface)
        s.set_coeff(co.a, co.grad_a)
        t1 = time.perf_counter()
        patch, uv = edge_patches(os_)
        if kind == "neumann":
            ae, ao = edge_a(os_), edge_a(os_, True)
        else:
            ae, ao = np.ones(os_.M), np.ones(F * os_.M)
        b = pm.BoundaryValueProblem(s, os_.curves, ae, ao, patch, uv, kind=kind)
        t2 = time.perf_counter()
        if kind == "neumann":
            f, fg, v = newtonian_neumann(os_, co)
        else:
            f, fg, v = newtonian_dirichlet(os_)
        b.solve(f, fg, tol=1e-12)
        t3 = time.perf_counter()
        u, info, _, _ = b.solve(f, fg, tol=1e-12)
        t4 = time.perf_counter()
        w = os_.surface.weights
        if kind == "neumann":
            e = (u - v) - np.dot(w, u - v) / w.sum()
            vv = v - np.dot(w, v) / w.sum()
        else:
            e, vv = u - v, v
        out["cases"][f"{kind}_band_{s.N}_edge_{b.Me}"] = {
            "N": s.N, "edge_nodes": b.Me, "oversampled": F * b.Me,
            "surface_build_s": round(t1 - t0, 3), "edge_build_s": round(t2 - t1, 4),
            "solve_s": round(t4 - t3, 4), "iterations": info.iterations,
            "residual": info.residual,
            "rel_l2_error_vs_exact": float(np.sqrt(np.dot(w, e * e) / np.dot(w, vv * vv)))}
        b.close()
        s.close()
    ctx.close()
    return out


def run_triangles(args, dev):
    """Triangle patches (Sec. 6.1, the paper's own discretisation): the unit sphere
    from 320 and 1,280 icosahedral triangles at the order-8 Vioreanu-Rokhlin nodes
    (11,520 and 46,080 nodes), f = Y_3^2: near-field build time, solve time to 1e-10
    (float32 direct applies; FMM applies on the larger surface as well) and the error
    against u = -f/12; the smooth-sum kernels are those of the quadrilateral surfaces."""
    import numpy as np
    import torch
    import paper_2401_12501_gb300 as pm
    from workloads import real_sph_harm
    from workloads.trisurfaces import tri_ellipsoid
    ctx = pm.Context(dev.index or 0)
    out = {"tol": args.tol, "rule": "Vioreanu-Rokhlin order 8 (36 nodes a triangle)",
           "problems": {}}
    for level, precs in ((2, ("fp32",)), (3, ("fp32", "fmm"))):
        sf = tri_ellipsoid(level, 8)
        t0 = time.perf_counter()
        s = pm.Surface.from_fixture(ctx, sf)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        s.set_coeff(np.ones(sf.N))
        Y = real_sph_harm(3, 2, sf.nodes)
        fd = torch.from_numpy(Y.copy()).to(dev)
        w = sf.weights
        row = {"N": sf.N, "triangles": sf.npatch, "near_build_s": round(t_build, 3),
               "near_blocks": s.info()[1]}
        for prec in precs:
            s.solve(fd, tol=args.tol, prec=prec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                u, info = s.solve(fd, tol=args.tol, prec=prec)
            torch.cuda.synchronize()
            t = (time.perf_counter() - t0) / 3
            u = u.cpu().numpy()
            row[prec] = {"solve_ms": round(t * 1e3, 3), "iterations": info[0].iterations,
                         "residual": info[0].residual,
                         "rel_l2_error_vs_exact": float(np.sqrt(np.dot(w, (u + Y / 12) ** 2) /
                                                                np.dot(w, (Y / 12) ** 2)))}
        out["problems"][f"tri_sphere_{sf.N}"] = row
        s.close()
    ctx.close()
    return out


def run_micro_ffmat(args):
    """The stored float-float matrices of one surface (default the 9,600-node ellipsoid:
    a 737 MB remainder matrix and a 369 MB symmetric parametrix matrix, both larger than
    L2): the store, then one float-float remainder and one parametrix apply, the
    launches an ncu capture of k_ffmat_gemv / k_ffmat_symK_gemv looks at."""
    import numpy as np
    import torch
    import paper_2401_12501_gb300 as pm
    from workloads import make_workload
    name = args.workload if args.workload != "torus_98304" else "ellipsoid_9600"
    wl = make_workload(name)
    ctx = pm.Context(0)
    s = pm.Surface.from_fixture(ctx, wl.surface)
    s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
    s.store_ff("RK")
    sig = torch.from_numpy(np.random.default_rng(2).standard_normal(wl.N) + 1.0).to("cuda:0")
    y = s.apply_R(sig, "ff")
    z = s.apply_K(sig, "ff")
    torch.cuda.synchronize()
    print(json.dumps({"micro": "ffmat", "workload": name, "N": wl.N,
                      "finite": bool(torch.isfinite(y).all() and torch.isfinite(z).all())}))
    s.close()
    ctx.close()


def run_micro_fmm(args):
    """One FMM remainder and one parametrix apply on the 98,304-node torus (built
    without stored matrices, ~2 GB on the device): the launches an ncu capture of the
    FMM kernels (k_fmm_p2p, k_tc_gemm, ...) looks at."""
    import numpy as np
    import torch
    import paper_2401_12501_gb300 as pm
    from workloads import make_workload
    wl = make_workload("torus_98304")
    ctx = pm.Context(0)
    s = pm.Surface.from_fixture(ctx, wl.surface)
    s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
    sig = torch.from_numpy(np.random.default_rng(3).standard_normal(wl.N) + 1.0).to("cuda:0")
    y = s.apply_R(sig, "fmm")
    z = s.apply_K(sig, "fmm")
    torch.cuda.synchronize()
    print(json.dumps({"micro": "fmm", "workload": "torus_98304", "N": wl.N,
                      "finite": bool(torch.isfinite(y).all() and torch.isfinite(z).all()),
                      "tree": s.fmm_stats()}))
    s.close()
    ctx.close()


def run_micro_tri(args):
    """One triangle-patch surface build (the unit sphere from 80 triangles at the order-8
    Vioreanu-Rokhlin nodes, 2,880 nodes): the launches an ncu capture of the triangle
    near-field kernels looks at."""
    import paper_2401_12501_gb300 as pm
    from workloads.trisurfaces import tri_ellipsoid
    ctx = pm.Context(0)
    sf = tri_ellipsoid(1, 8)
    t0 = time.perf_counter()
    s = pm.Surface.from_fixture(ctx, sf)
    print(json.dumps({"micro": "tri", "N": sf.N, "near_blocks": s.info()[1],
                      "build_s": round(time.perf_counter() - t0, 3)}))
    s.close()
    ctx.close()


def run_micro_helmholtz(args):
    """Three float64 c != 0 remainder applies on the 1,536-node unit sphere (a = 1,
    c = --micro-c): the launches an ncu capture of k_direct_c64 looks at."""
    import numpy as np
    import paper_2401_12501_gb300 as pm
    from workloads import cubed_sphere
    ctx = pm.Context(0)
    sf = cubed_sphere(2, 8)
    s = pm.Surface.from_fixture(ctx, sf)
    s.set_coeff_c(np.ones(sf.N), np.zeros((sf.N, 3)), np.full(sf.N, args.micro_c))
    sig = np.random.default_rng(1).standard_normal(sf.N) + 0j
    for _ in range(3):
        y = s.apply_c(sig, "R")
    print(json.dumps({"micro": "helmholtz", "c": args.micro_c, "N": sf.N,
                      "max_abs": float(np.abs(y).max())}))
    s.close()
    ctx.close()


def run_helmholtz(args, dev):
    """c != 0 (Sec. 4.2) on the device in float64: the paper's sphere test with c
    added (Sec. 7.1: four harmonics incl. l = 10, u = sum f_lm Y / (c - l(l+1))) and
    its variable-coefficient examples (Sec. 7.4: a linear in z, c = -4 - e^{x/2}; and
    complex c = 4 (1 + 0.2 y + 0.2 i sin x) with a = 1 + e^z; manufactured
    v = -1/|x - x0|) on cubed-sphere ellipsoids; near-field build and
    solve times, error against the exact solution, and the float64 smooth sum's
    pair rate (the dominant kernel, k_direct_c64)."""
    import numpy as np
    import torch
    import paper_2401_12501_gb300 as pm
    from workloads import cubed_sphere, four_harmonic_problem, real_sph_harm
    from workloads.coefficients import _tangential
    ctx = pm.Context(dev.index or 0)
    out = {"tol": 1e-12, "arithmetic": "complex float64", "problems": {}}

    def e4(x, n):
        ga = np.tile([0.0, 0.0, 0.5], (len(x), 1))
        return 2.0 + 0.5 * x[:, 2], _tangential(ga, n), -4.0 - np.exp(x[:, 0] / 2)

    def manufactured(sf, a, ga, c):
        x0 = np.array([-3.0, -3.0, 4.0])
        dx = sf.nodes - x0
        rho = np.linalg.norm(dx, axis=1)
        v = -1.0 / rho
        grad = dx / rho[:, None] ** 3
        dn = np.sum(grad * sf.normals, 1)
        dnn = 1.0 / rho ** 3 - 3 * np.sum(dx * sf.normals, 1) ** 2 / rho ** 5
        return (np.sum(ga * (grad - sf.normals * dn[:, None]), 1) +
                a * (-2 * sf.curvature * dn - dnn) + c * v), v

    cases = []
    for cval in (-4.0, 4.0):
        sf = cubed_sphere(4, 8)
        f, _ = four_harmonic_problem(sf, seed=0)
        coef = np.random.default_rng(0).standard_normal(4)
        uex = sum(cf * real_sph_harm(l, m, sf.nodes) / (cval - l * (l + 1))
                  for cf, (l, m) in zip(coef, [(1, 0), (3, 3), (10, 6), (10, 7)]))
        N = sf.N
        cases.append((f"sphere_{N}_c{cval:+g}", sf, np.ones(N), np.zeros((N, 3)),
                      np.full(N, cval), f, uex))
    for m in (3, 5):
        sf = cubed_sphere(m, 8, axes=(1.0, 1.5, 2.0))
        a, ga, c = e4(sf.nodes, sf.normals)
        f, v = manufactured(sf, a, ga, c)
        cases.append((f"ellipsoid_{sf.N}_sec74", sf, a, ga, c, f, v))
    # the paper's complex example: a = 1 + e^z, c = 4 (1 + 0.2 y + 0.2 i sin x)
    sf = cubed_sphere(3, 8, axes=(1.0, 1.5, 2.0))
    ez = np.exp(sf.nodes[:, 2])
    a = 1.0 + ez
    ga = _tangential(np.stack([0 * ez, 0 * ez, ez], 1), sf.normals)
    c = 4.0 * (1 + 0.2 * sf.nodes[:, 1] + 0.2j * np.sin(sf.nodes[:, 0]))
    f, v = manufactured(sf, a, ga, c)
    cases.append((f"ellipsoid_{sf.N}_sec74_complex", sf, a, ga, c, f, v))
    for name, sf, a, ga, c, f, uex in cases:
        s = pm.Surface.from_fixture(ctx, sf)
        t0 = time.perf_counter()
        s.set_coeff_c(a, ga, c)
        t_near = time.perf_counter() - t0
        s.solve_c(f, tol=1e-12)
        t0 = time.perf_counter()
        reps = 2
        for _ in range(reps):
            u, info = s.solve_c(f, tol=1e-12)
        t_solve = (time.perf_counter() - t0) / reps
        w = sf.weights
        err = float(np.sqrt(np.dot(w, np.abs(u - uex) ** 2) / np.dot(w, np.abs(uex) ** 2)))
        # the float64 smooth sum alone (profile phases around its launches)
        sig = np.random.default_rng(1).standard_normal(sf.N) + 0j
        s.profile(True)
        s.profile_read(0, reset=True)
        for _ in range(3):
            s.apply_c(sig, "R")
        s.profile(False)
        ms, nl = s.profile_read(pm._lib.PM_PHASE_DIRECT64)
        near_ms, nn = s.profile_read(pm._lib.PM_PHASE_NEAR)
        s.profile_read(0, reset=True)
        pairs = sf.N * (sf.N - 1)
        out["problems"][name] = {
            "N": sf.N, "near_build_c_s": round(t_near, 3), "solve_ms": round(t_solve * 1e3, 2),
            "iterations": info.iterations, "residual": info.residual,
            "rel_l2_error_vs_exact": err,
            "k_direct_c64_ms": round(ms / max(1, nl), 4),
            "k_direct_c64_gpairs_per_s": round(pairs / (ms / max(1, nl)) / 1e6, 3),
            "near_c_ms": round(near_ms / max(1, nn), 4)}
        s.close()
    ctx.close()
    return out


def run_fmm(args, dev):
    """98,304-node torus: float32 apply with the Chebyshev FMM vs the direct sum."""
    import numpy as np
    import torch
    import paper_2401_12501_gb300 as pm
    from workloads import make_workload
    wl = make_workload("torus_98304")
    ctx = pm.Context(dev.index or 0)
    t0 = time.perf_counter()
    s = pm.Surface.from_fixture(ctx, wl.surface)
    t_build = time.perf_counter() - t0
    s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
    # octree depth and direct-sum launch shape picked by the autotuner
    tune_fmm = s.autotune(nrhs=1, prec="fmm", reps=3) if not args.no_autotune else _builtin(s)
    tune_32 = s.autotune(nrhs=1, prec="fp32", reps=3) if not args.no_autotune else _builtin(s)
    st = s.fmm_stats()
    sig = torch.from_numpy(np.random.default_rng(3).standard_normal(wl.N)).to(dev)
    out = {}
    for prec in ("fp32", "fmm", "ff"):
        y = torch.empty_like(sig)
        s.apply_R(sig, prec, out=y)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 3
        _nvtx_push("fmm_torus_" + prec)
        for _ in range(reps):
            s.apply_R(sig, prec, out=y)
        torch.cuda.synchronize()
        _nvtx_pop()
        out[prec] = ((time.perf_counter() - t0) / reps, y.cpu().numpy())
    ex = out["ff"][1]
    # whole solves (tol 1e-8): GMRES with FMM applies vs with direct float32 applies,
    # float-float refinement and representation in both
    solves = {}
    for prec in ("fmm", "fp32"):
        s.solve(wl.f, tol=1e-8, prec=prec)                  # warm (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u, info = s.solve(wl.f, tol=1e-8, prec=prec)
        solves[prec] = (time.perf_counter() - t0, u, info[0])
    w = wl.surface.weights
    du = solves["fmm"][1] - solves["fp32"][1]
    m2l_pairs = st["m2l_box_pairs"]
    res = {"workload": "torus_98304", "N": wl.N, "near_build_s": round(t_build, 3),
           "m2l": "one operator GEMM per offset class (16 classes of the 316 offsets under the "
                  "cube's signed axis permutations), all classes in one launch of the library's "
                  "tcgen05 kernel (TMEM accumulators, TMA-staged tiles) with float32 "
                  "accumulation: float32 operands scaled by powers of two and split in two "
                  "float16 parts, the three products of order <= 2^-11 as one GEMM over K = 1536",
           "m2l_gemm_flops_per_apply": 2.0 * 9 * 512 * 512 * m2l_pairs,
           "m2l_f16_flops_executed_per_apply": 3 * 2.0 * 9 * 512 * 512 * m2l_pairs,
           "m2l_operator_bytes_per_apply": 16 * 9 * 512 * 1536 * 2,
           "solve_tol_1e-8": {p: {"ms": round(v[0] * 1e3, 2), "iterations": v[2].iterations,
                                  "refinements": v[2].refinements,
                                  "residual": v[2].residual} for p, v in solves.items()},
           "solve_u_rel_diff_fmm_vs_fp32": float(np.sqrt(np.dot(w, du * du) /
                                                         np.dot(w, solves["fp32"][1] ** 2))),
           "autotune": {t: {"knobs": {k: v for k, v in r["knobs"].items() if v},
                            "apply_ms": _r(r["best_ms"], 3),
                            "builtin_apply_ms": _r(r["default_ms"], 3),
                            "candidates": r["candidates"]}
                        for t, r in (("fmm", tune_fmm), ("fp32", tune_32))},
           "fmm_tree": st, "apply_R_ms": {k: round(v[0] * 1e3, 3) for k, v in out.items()},
           "rel_err_vs_float_float": {k: float(np.linalg.norm(v[1] - ex) / np.linalg.norm(ex))
                                      for k, v in out.items() if k != "ff"},
           "direct_gpairs_per_s": round(wl.N ** 2 / out["fp32"][0] / 1e9, 1)}
    s.close()
    return res


# Served geometries: a ladder over 1.5k-400k nodes, both patch orders and all four
# families (family, p, surface parameters, N).  A request's size is drawn
# log-uniformly over [1,500, 400,000] and snapped to the nearest rung in log N, so
# the rung fixes its family and p; two coefficient fields per geometry.
SERVE_LADDER = [("sphere", 8, 2, 1536), ("ellipsoid", 10, 4, 9600), ("star", 8, 8, 24576),
                ("torus", 10, (32, 12), 38400), ("ellipsoid", 8, 16, 98304),
                ("star", 10, 16, 153600), ("torus", 8, (128, 48), 393216)]


def _ladder_surface(rung):
    from workloads import cubed_sphere, star_surface, torus
    fam, p, par, _ = rung
    if fam == "sphere":
        return cubed_sphere(par, p)
    if fam == "ellipsoid":
        return cubed_sphere(par, p, axes=(1.0, 1.5, 2.0))
    if fam == "star":
        return star_surface(par, p)
    return torus(par[0], par[1], p)


def run_served(args, dev):
    """Poisson arrivals of solve requests on operators the server builds itself from
    their descriptions (near field per geometry, clone per further coefficient), FMM
    applies from serve_fmm_min nodes, GMRES to serve_tol on the apply-precision
    operator (no float-float refinement: float32/FMM applies + float64 GMRES).
    One server: a cold run (operators built as their first requests arrive; build
    time reported apart), then on the resident operators continuous batching vs one
    request at a time, at the arrival rate and with every request at t = 0."""
    import threading as th
    import numpy as np
    import paper_2401_12501_gb300 as pm
    from workloads import random_harmonic_rhs, smooth_random_coefficient
    rng = np.random.default_rng(0)
    n_req, rate = args.serve_requests, args.serve_rate
    lo, hi = np.log(1500.0), np.log(float(args.serve_nmax))
    logs = np.log([r[3] for r in SERVE_LADDER])
    draws = []
    for _ in range(n_req):
        n = float(np.exp(rng.uniform(lo, hi)))
        k = int(np.argmin(np.abs(logs - np.log(n))))
        draws.append((k, int(rng.integers(0, 2)), int(rng.integers(0, 1 << 30))))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    used = sorted({d[0] for d in draws})
    surfs = {k: _ladder_surface(SERVE_LADDER[k]) for k in used}
    coeffs = {(k, c): smooth_random_coefficient(surfs[k], c) for k in used for c in (0, 1)}
    rhs = [random_harmonic_rhs(surfs[k], fs % 1000, n_terms=20, lmax=12) for k, _, fs in draws]
    opts = pm.default_opts()
    opts.residual_prec = pm.PM_PREC_FP32                # GMRES on the apply-precision operator
    prec = ["fmm" if surfs[k].N >= args.serve_fmm_min else "fp32" for k, _, _ in draws]
    ctx = pm.Context(dev.index or 0)
    sv = pm.Server(ctx, hbm_budget_bytes=int(args.serve_budget_gb * 2 ** 30), max_batch=64,
                   n_workers=4)

    def submit(i):
        k, c, _ = draws[i]
        co = coeffs[(k, c)]
        return sv.submit_desc(k, c, surfs[k], co.a, co.grad_a, rhs[i], tol=args.serve_tol,
                              prec=prec[i], opts=opts)

    keep = {next(j for j, d in enumerate(draws) if d[0] == k): None for k in used}

    def serve(max_batch, n_workers, arr, keep_u=False):
        sv.configure(max_batch, n_workers)
        b0 = sv.stats()["batches"]
        tickets = [None] * n_req
        t_start = time.perf_counter()

        def client():
            for i in range(n_req):
                dt = arr[i] - (time.perf_counter() - t_start)
                if dt > 0:
                    time.sleep(dt)
                tickets[i] = submit(i)

        c = th.Thread(target=client)
        c.start()
        lat, lat_nb, builds, res, sizes = [], [], [], [], []
        for i in range(n_req):
            while tickets[i] is None:
                time.sleep(0.0005)
            u, info, tm = sv.wait_ex(tickets[i])
            if keep_u and i in keep:
                keep[i] = u
            lat.append(tm["latency_s"])
            lat_nb.append(tm["latency_s"] - tm["build_s"])
            builds.append(tm["build_s"])
            res.append(info.residual)
        c.join()
        wall = time.perf_counter() - t_start
        st = sv.stats()
        lat, lat_nb = np.array(lat), np.array(lat_nb)
        out = {"p50_latency_ms": round(float(np.percentile(lat, 50)) * 1e3, 2),
               "p99_latency_ms": round(float(np.percentile(lat, 99)) * 1e3, 2),
               "solves_per_s": round(n_req / wall, 2), "wall_s": round(wall, 3),
               "batches": st["batches"] - b0, "max_batch_seen": st["max_batch"],
               "max_residual": float(max(res))}
        if max(builds) > 0:
            out["build_wait_s_total"] = round(float(sum(builds)), 3)
            out["requests_waiting_on_a_build"] = int(sum(b > 0 for b in builds))
            out["p50_latency_ms_excluding_build_wait"] = round(float(np.percentile(lat_nb, 50)) * 1e3, 2)
            out["p99_latency_ms_excluding_build_wait"] = round(float(np.percentile(lat_nb, 99)) * 1e3, 2)
        return out

    t0 = time.perf_counter()
    cold = serve(64, 4, arrivals)
    t_cold = time.perf_counter() - t0
    n_builds = sv.stats()["builds"]
    served = serve(64, 4, arrivals, keep_u=True)
    plain = serve(1, 1, arrivals)
    zero = np.zeros(n_req)
    sat_served = serve(64, 4, zero)
    sat_plain = serve(1, 1, zero)
    sv.close()
    # accuracy of the served apply-precision solutions (one request per rung up to
    # 100k nodes, from the continuous-batching run) against float-float refined
    # solves of the same systems on caller-built operators
    acc = {}
    for i, u_op in keep.items():
        k, c, _ = draws[i]
        if surfs[k].N > 100000:
            continue
        co = coeffs[(k, c)]
        s = pm.Surface.from_fixture(ctx, surfs[k])
        s.set_coeff(co.a, co.grad_a)
        u_ff, _ = s.solve(rhs[i], tol=1e-10, prec=prec[i])
        s.close()
        w = surfs[k].weights
        acc[f"{SERVE_LADDER[k][0]}_{SERVE_LADDER[k][3]}_p{SERVE_LADDER[k][1]}"] = float(
            np.sqrt(np.dot(w, (u_op - u_ff) ** 2) / np.dot(w, u_ff ** 2)))
    ctx.close()
    counts = {f"{SERVE_LADDER[k][0]}_{SERVE_LADDER[k][3]}_p{SERVE_LADDER[k][1]}":
              sum(d[0] == k for d in draws) for k in used}
    return {"requests": n_req, "arrival_rate_per_s": rate, "seed": 0,
            "geometries": len(used), "operators": 2 * len(used),
            "node_range": [min(surfs[k].N for k in used), max(surfs[k].N for k in used)],
            "patch_orders": sorted({SERVE_LADDER[k][1] for k in used}),
            "requests_per_geometry": counts, "n_max_drawn": args.serve_nmax,
            "tol": args.serve_tol, "fmm_applies_from_n": args.serve_fmm_min,
            "solve": "GMRES (float64 basis) to tol on the float32 / FMM operator, "
                     "no float-float refinement (opts.residual_prec = PM_PREC_FP32)",
            "u_rel_err_vs_float_float_refined_solve": acc,
            "admission": "by free HBM: cudaMemGetInfo less a margin, modelled bytes per "
                         "build and batch, budget cap %.0f GiB" % args.serve_budget_gb,
            "cold_run_with_in_server_builds": {**cold, "operator_builds_near_field_or_clone": n_builds,
                                               "run_s": round(t_cold, 3)},
            "continuous_batching": served, "one_at_a_time": plain,
            "solves_per_s_ratio": round(served["solves_per_s"] / plain["solves_per_s"], 2),
            "saturated": {"continuous_batching": sat_served, "one_at_a_time": sat_plain,
                          "solves_per_s_ratio": round(sat_served["solves_per_s"]
                                                      / sat_plain["solves_per_s"], 2)}}


def run_micro_tc_gemm(args):
    """The M2L product of the 98,304-node torus at its full size on the library's
    tcgen05 GEMM alone: A = the remainder operators' 9 x 512 rows, K = 3 x 512
    (two float16 parts, three products), 11,392 columns (the torus's V-list box
    pairs at depth 3), seeded normal operands."""
    import numpy as np
    import paper_2401_12501_gb300 as pm
    rows, K, ncols = 4608, 1536, 11392
    rng = np.random.default_rng(1)
    A = rng.standard_normal((rows, K)).astype(np.float16).view(np.uint16)
    B = rng.standard_normal((ncols, K)).astype(np.float16).view(np.uint16)
    ctx = pm.Context(0)
    _, ms = ctx.selftest_tc_gemm(A, B, reps=max(1, args.steps))
    ctx.close()
    fl = 2.0 * rows * K * ncols
    print(json.dumps({"micro": "tc_gemm", "shape": [rows, ncols, K], "dtype": "f16",
                      "ms": ms, "tflops": fl / (ms * 1e-3) / 1e12}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="torus_98304")
    ap.add_argument("--prec", default=None, choices=["fp32", "fmm"],
                    help="operator precision of the solve step (default: FMM for the torus, "
                         "float32 direct sums otherwise)")
    ap.add_argument("--oracle-leg", action="store_true")
    ap.add_argument("--oracle-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-store-ff", action="store_true",
                    help="evaluate the float-float sums pair by pair instead of storing the "
                         "operator's float-float matrices in HBM")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in launch shapes (for profiler runs, whose timings "
                         "would mislead the autotuner)")
    ap.add_argument("--extras", default="ellipsoid,batched,fmm,served,paper,helmholtz,triangles,bvp",
                    help="comma-separated extra measurements to run (ellipsoid, batched, fmm, "
                         "served, paper, helmholtz, triangles, bvp)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched, FMM and served measurements")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-nmax", type=int, default=400000)
    ap.add_argument("--serve-tol", type=float, default=1e-8)
    ap.add_argument("--serve-budget-gb", type=float, default=200.0)
    ap.add_argument("--serve-fmm-min", type=int, default=40000,
                    help="served operators with at least this many nodes use FMM applies")
    ap.add_argument("--micro", choices=["tc_gemm", "helmholtz", "tri", "ffmat", "fmm"], default=None,
                    help="time one kernel alone instead of the solve step (profiling aid)")
    ap.add_argument("--micro-c", type=float, default=-4.0,
                    help="c of --micro helmholtz (1,536-node unit sphere, a = 1)")
    args = ap.parse_args()

    if args.micro == "tc_gemm":
        run_micro_tc_gemm(args)
        return
    if args.micro == "helmholtz":
        run_micro_helmholtz(args)
        return
    if args.micro == "tri":
        run_micro_tri(args)
        return
    if args.micro == "ffmat":
        run_micro_ffmat(args)
        return
    if args.micro == "fmm":
        run_micro_fmm(args)
        return
    if args.oracle_leg:
        P = host_cores()
        runner = OracleRunner(args.workload, P)
        rate_all, desc_all = runner.rate(args.oracle_seconds)
        rate_1, desc_1 = runner.rate(max(2.0, args.oracle_seconds / 2), processes=1)
        runner.close()
        print(json.dumps({"value": rate_all, "sample": desc_all, "cores": P,
                          "value_1core": rate_1, "sample_1core": desc_1}))
        return

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))

    if args.impl == "reference":
        if rank != 0:
            return
        P = host_cores()
        runner = OracleRunner(args.workload, P)
        per_step = max(1.0, min(8.0, 120.0 / max(1, args.steps + args.warmup)))
        vals, desc = [], ""
        for _ in range(args.warmup + args.steps):
            v, desc = runner.rate(per_step)
            vals.append(v)
        runner.close()
        print(json.dumps(reference_line(args, vals, desc, P)))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    line = run_gpu(args, rank, world, local_rank)
    if rank == 0 and not args.no_extra:
        import torch
        dev = torch.device("cuda", local_rank)
        want = set(args.extras.split(","))
        for name, key, fn in (("ellipsoid", "ellipsoid_9600", run_ellipsoid),
                              ("batched", "batched_star_24576", run_batched),
                              ("fmm", "fmm_torus_98304", run_fmm), ("served", "served", run_served),
                              ("paper", "paper_problems", run_paper),
                              ("helmholtz", "helmholtz_c_nonzero", run_helmholtz),
                              ("triangles", "triangle_patches", run_triangles),
                              ("bvp", "boundary_value_problems", run_bvp)):
            if name not in want:
                continue
            try:
                line[key] = fn(args, dev)
            except Exception as e:  # report, do not hide
                line[key] = {"error": str(e)[:400]}
    if rank == 0:
        if not args.no_cpu_baseline:
            try:
                r = run_oracle_subprocess(args.workload, args.oracle_seconds)
                line["cpu_baseline"] = {"value": r["value"], "unit": UNIT, "cores": r["cores"],
                                        "kind": "oracle", "sample": r["sample"],
                                        "value_1core": r["value_1core"],
                                        "sample_1core": r["sample_1core"]}
            except Exception as e:  # report, do not hide
                line["cpu_baseline"] = {"value": None, "error": str(e)[:300]}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
