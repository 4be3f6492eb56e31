"""Benchmark of the parametrix hot path on one GB300 (or N independent replicas).

Default workload: the 9,600-node ellipsoid (1, 1.5, 2) with
a = 1 + 0.5 sin(2x) cos(3y) and a seeded mean-zero right-hand side.  One step
is one full solve of div(a grad u) = f to a relative residual of 1e-10 (so
that u matches a plain float64 solve to 1e-8; the line reports the measured
difference): source prep, float32 smooth sums,
near-field correction, device GMRES, float-float true residuals, u = K~ sigma
and the mean projection.  The near field is built once per surface, before
the timed region (its time is reported).  Inputs are resident in HBM; L2 is
flushed between steps.

Prints one JSON line (rank 0).  --impl reference times the float64 CPU oracle
on a bounded sample of the same workload instead.
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
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# of the current kernel versions on this workload (profiles/k_direct_*_ellipsoid_9600.md);
# set to None whenever the kernel changes until it is captured again.
TRAFFIC_BYTES = {("k_direct_R32", "ellipsoid_9600"): 624128,
                 ("k_direct_ff_R", "ellipsoid_9600"): 1236224,
                 ("k_sym_ff_R", "ellipsoid_9600"): 1299712}
SYM_PARTIAL_CAP = 1024 ** 3             # the library's cap on symmetric-sum partial slices
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0


def fp32_peak_tflops(mhz=SM_MAX_MHZ):
    """Non-tensor float32 peak from unit counts: SMs x FP32 lanes x 2 flops (FMA) x clock."""
    return SM_COUNT * FP32_LANES * 2 * mhz * 1e6 / 1e12


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
def oracle_rate(workload: str, seconds: float = 12.0):
    """Oracle float64 remainder apply on a bounded sample; returns (Gpairs/s, description)."""
    import numpy as np
    from oracle.operator import Discretization, NearField
    from workloads import make_workload
    wl = make_workload(workload)
    d = Discretization.from_workload(wl)
    N = d.N
    rng = np.random.default_rng(0)
    sigma = rng.standard_normal(N)
    near_rows = [int(i) for i in rng.integers(0, N, 8)]
    nf = NearField(d, rows=near_rows)            # one-time corrections, not timed
    rows_done, t_smooth = 0, 0.0
    chunk = 256
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        r0 = (rows_done * 7919) % max(1, N - chunk)
        rows = np.arange(r0, min(N, r0 + chunk))
        ts = time.perf_counter()
        d.smooth_apply("R", sigma, rows)
        t_smooth += time.perf_counter() - ts
        rows_done += len(rows)
    ts = time.perf_counter()
    nf.apply("R", sigma, near_rows)
    t_near = (time.perf_counter() - ts) / len(near_rows)
    t_row = t_smooth / rows_done + t_near
    rate = N / t_row / 1e9                      # pairs per second per row-time
    desc = (f"{rows_done} target rows of {workload} (smooth sum over all {N} sources) "
            f"+ near-field correction of {len(near_rows)} rows, float64 numpy, 1 thread")
    return rate, desc


def reference_line(args, vals, desc):
    """The reference arm's JSON line: the oracle's rate (mean over the timed steps)."""
    v = statistics.mean(vals[args.warmup:]) if len(vals) > args.warmup else vals[-1]
    return {
        "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "impl": "reference",
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_oracle_subprocess(workload: str, seconds: float):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-leg",
                        "--workload", workload, "--oracle-seconds", str(seconds)],
                       capture_output=True, text=True, env=env, timeout=600)
    for ln in r.stdout.splitlines()[::-1]:
        if ln.startswith("{"):
            return json.loads(ln)
    raise RuntimeError("oracle leg failed: " + r.stdout[-2000:] + r.stderr[-2000:])


# ----------------------------------------------------------------------------- GPU arm
PHASES = ["prep", "direct_R32", "direct_K32", "near", "vec", "direct_ff_or_64"]


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


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_2401_12501_gb300 as pm
    from paper_2401_12501_gb300 import _lib
    from workloads import make_workload

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = make_workload(args.workload)
    N = wl.N
    pairs = float(N) * N
    ctx = pm.Context(local_rank)
    t0 = time.perf_counter()
    surf = pm.Surface.from_fixture(ctx, wl.surface)
    t_build = time.perf_counter() - t0
    surf.set_coeff(wl.coeff.a, wl.coeff.grad_a)
    nblk = surf.info()[1]
    # launch shape of the float32 sums picked by the autotuner (untimed, before warm-up)
    tune = surf.autotune(nrhs=1, prec="fp32", reps=5) if not args.no_autotune else _builtin(surf)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    f_h = torch.from_numpy(wl.f.copy()).pin_memory()
    u_h = torch.empty(N, dtype=torch.float64).pin_memory()
    f_d = f_h.to(dev)
    tol = args.tol

    def step():
        return surf.solve(f_d, tol=tol, prec="fp32")

    # the accuracy the timed solves reach: u against a plain float64 solve (float64
    # operator applies and Krylov basis) of the same system to 1e-12
    u_ref, _ = surf.solve(wl.f, tol=1e-12, prec="fp64")
    u_chk, _ = surf.solve(wl.f, tol=tol, prec="fp32")
    wq = wl.surface.weights
    err_vs_fp64 = float(np.sqrt(np.dot(wq, (u_chk - u_ref) ** 2) / np.dot(wq, u_ref ** 2)))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist = None
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

    # phase split: the same steps again with per-phase events (event records
    # cannot sit inside the graph-driven GMRES cycle, so this pass issues its
    # launches from the host; the kernels are the same)
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
    # operator applies per solve: one float32 R apply per Arnoldi step, one accurate R
    # apply per refinement, one accurate K apply for u
    it = statistics.mean(i.iterations for i in infos)
    rf = statistics.mean(i.refinements for i in infos)
    applies = it + rf + 1
    value = job_throughput(world, applies * pairs, ms_per_step)
    solves_per_s = world * 1e3 / ms_per_step

    # end-to-end through the C ABI with host (pinned) buffers: f in, u out
    for _ in range(2):
        surf.solve(f_h.numpy(), tol=tol, prec="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u, _ = surf.solve(f_h.numpy(), tol=tol, prec="fp32")
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_value = job_throughput(world, applies * pairs, e2e_s * 1e3)

    # isolated float32 remainder apply (inputs resident, L2 flushed)
    sig = torch.from_numpy(np.random.default_rng(1).standard_normal(N)).to(dev)
    out = torch.empty_like(sig)
    for _ in range(3):
        surf.apply_R(sig, "fp32", out=out)
    surf.profile(True)
    surf.profile_read(0, reset=True)
    aev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        aev[k][0].record(stream)
        surf.apply_R(sig, "fp32", out=out)
        aev[k][1].record(stream)
    torch.cuda.synchronize()
    surf.profile(False)
    aph = _phase_totals(surf)
    apply_ms = sum(a.elapsed_time(b) for a, b in aev) / args.steps

    # roofline of the dominant kernel of the solve step (by device time)
    fp32_ms, fp32_n = ph["direct_R32"]
    ff_ms, ff_n = ph["direct_ff_or_64"]
    peak = fp32_peak_tflops()
    # per-launch time of the float32 sum inside the solve step (profiled pass)
    fp32_k = fp32_ms / max(1, fp32_n)
    r32 = {"bound": "alu", "kernel": "k_direct_R32 (float32 remainder sum)",
           "achieved": round(FLOPS_PER_PAIR_R * pairs / (fp32_k * 1e-3) / 1e12, 3),
           "peak": round(peak, 2), "unit": "TFLOP/s",
           "frac": round(FLOPS_PER_PAIR_R * pairs / (fp32_k * 1e-3) / 1e12 / peak, 4),
           "traffic": TRAFFIC_BYTES.get(("k_direct_R32", args.workload)),
           "kernel_ms": round(fp32_k, 5),
           "flops_per_pair": FLOPS_PER_PAIR_R,
           "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (unit counts)",
           "step_time_share": round(fp32_ms / prof_total_ms, 4)}
    ff_k = ff_ms / ff_n if ff_n else 0.0
    nt = -(-N // 128)
    sym = N >= 256 and nt * N * 8 <= SYM_PARTIAL_CAP
    ff_name = "k_sym_ff" if sym else "k_direct_ff"
    rff = {"bound": "alu",
           "kernel": ff_name + (" (symmetric tile-pair float-float remainder/parametrix sums)" if sym
                                else " (float-float remainder/parametrix sums)"),
           "achieved": round(FLOPS_PER_PAIR_R * pairs / (ff_k * 1e-3) / 1e12, 3) if ff_k else None,
           "peak": round(peak, 2), "unit": "TFLOP/s",
           "frac": round(FLOPS_PER_PAIR_R * pairs / (ff_k * 1e-3) / 1e12 / peak, 4) if ff_k else None,
           "traffic": TRAFFIC_BYTES.get((ff_name + "_R", args.workload)),
           "kernel_ms_per_apply": round(ff_k, 5),
           "note": "algorithmic flops of the float64-class sum (26 per ordered pair) over the "
                   "average of the step's float-float launches; float-float arithmetic costs "
                   "~10 float32 instructions per algorithmic flop (274 per unordered pair for "
                   "the remainder, 130 for the parametrix, each unordered pair evaluated once)",
           "step_time_share": round(ff_ms / prof_total_ms, 4)}
    dominant, other = (rff, r32) if ff_ms > fp32_ms else (r32, rff)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32",
        "dtype_detail": "f32 operator applies (compensated sums) + float-float residuals/"
                        "representation + f64 Krylov basis and near field",
        "data": "synthetic", "impl": "gb300",
        "config": {"workload": args.workload, "N": N,
                   "step": "one solve of div(a grad u) = f to relative residual "
                           f"{tol:g}: device GMRES (float32 applies) + float-float "
                           "refinement + u = K sigma + mean projection",
                   "value_definition": "smooth-sum pairs evaluated per second over the solve "
                                       "step = (Arnoldi steps + refinements + 1) * N^2 / time",
                   "near_blocks": nblk, "near_build_s": round(t_build, 3),
                   "autotune": {"knobs": tune["knobs"], "apply_ms": _r(tune["best_ms"], 4),
                                "builtin_apply_ms": _r(tune["default_ms"], 4),
                                "candidates": tune["candidates"]},
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "solves_per_s": round(solves_per_s, 2),
        "solve": {"iterations": it, "refinements": rf, "applies_per_solve": applies,
                  "residual_max": max(i.residual for i in infos),
                  "rel_err_vs_fp64_solve": err_vs_fp64,
                  "profiled_ms_per_step": round(prof_total_ms / args.steps, 4),
                  "phase_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in ph.items()
                                        if k != "launches_all"}},
        "apply_R_fp32": {"gpairs_per_s": round(pairs / (apply_ms * 1e-3) / 1e9, 2),
                         "ms": round(apply_ms, 5),
                         "phase_ms": {k: round(v[0] / args.steps, 5) for k, v in aph.items()
                                      if k != "launches_all"}},
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": 8 * N,
                "d2h_bytes_per_step": 8 * N, "solves_per_s": round(world / e2e_s, 2)},
        "gpu_launches": None,
        "roofline": dominant,
        "roofline_other": other,
        "clocks": clk.summary(),
    }
    line["gpu_launches"] = int(launches_timed)
    return line


# ----------------------------------------------------------------------------- other configs
def _builtin(s):
    """The autotuner's report for the built-in launch shapes (used with --no-autotune)."""
    return {"knobs": s.knobs(), "best_ms": None, "default_ms": None,
            "candidates": 0, "cached": False, "key": "built-in"}


def _r(v, nd):
    return None if v is None else round(v, nd)


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


def _snap_surface(family, n_target, rng):
    """Snap a drawn size to a factor-of-2 ladder of surfaces of the family (p = 8).

    Sizes stay log-uniform in the drawn range, but operators recur, so a served
    surface keeps its geometry and near field resident across requests."""
    from workloads import cubed_sphere, star_surface, torus
    p = 8
    ladder = 1536 * 2.0 ** np.arange(0, 12)
    n_b = float(ladder[np.argmin(np.abs(np.log(ladder / n_target)))])
    if family == "torus":
        nph = max(3, int(round(np.sqrt(n_b / (p * p) * 3 / 8))))
        nth = max(3, int(round(nph * 8 / 3)))
        return ("torus", p, nth, nph), lambda: torus(nth, nph, p)
    m = max(1, int(round(np.sqrt(n_b / (6 * p * p)))))
    if family == "sphere":
        return ("sphere", p, m), lambda: cubed_sphere(m, p)
    if family == "ellipsoid":
        return ("ellipsoid", p, m), lambda: cubed_sphere(m, p, axes=(1.0, 1.5, 2.0))
    return ("star", p, m), lambda: star_surface(m, p)


import numpy as np  # noqa: E402  (used by the serving helpers)


def run_served(args, dev):
    """Poisson arrivals of solve requests over a pool of operators; batched server
    vs a one-request-at-a-time server on the same arrival trace."""
    import threading as th
    import paper_2401_12501_gb300 as pm
    from workloads import random_harmonic_rhs, smooth_random_coefficient
    rng = np.random.default_rng(0)
    n_req, rate = args.serve_requests, args.serve_rate
    fams = ["sphere", "ellipsoid", "torus", "star"]
    lo, hi = np.log(1500.0), np.log(float(args.serve_nmax))
    keys, draws = {}, []
    for _ in range(n_req):
        fam = fams[int(rng.integers(0, 4))]
        key, mk = _snap_surface(fam, float(np.exp(rng.uniform(lo, hi))), rng)
        cseed = int(rng.integers(0, 2))
        keys.setdefault((key, cseed), mk)
        draws.append(((key, cseed), int(rng.integers(0, 1 << 30))))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    ctx = pm.Context(dev.index or 0)
    ops, builds, rhs = {}, [], {}
    geo = {}            # one near-field build per geometry; other coefficient seeds clone it
    for k, mk in sorted(keys.items(), key=lambda kv: (str(kv[0][0]), kv[0][1])):
        t0 = time.perf_counter()
        if k[0] in geo:
            surf, base = geo[k[0]]
            op = base.clone()
        else:
            surf = mk()
            op = pm.Surface.from_fixture(ctx, surf)
            geo[k[0]] = (surf, op)
        co = smooth_random_coefficient(surf, k[1])
        op.set_coeff(co.a, co.grad_a)
        builds.append(time.perf_counter() - t0)
        ops[k] = (surf, op)
    for i, (k, fseed) in enumerate(draws):
        surf = ops[k][0]
        rhs[i] = random_harmonic_rhs(surf, fseed % 1000, n_terms=20, lmax=12)

    def serve(max_batch, n_workers, arrivals=arrivals):
        sv = pm.Server(ctx, hbm_budget_bytes=int(args.serve_budget_gb * 2 ** 30),
                       max_batch=max_batch, n_workers=n_workers)
        tickets = [None] * n_req
        t_start = time.perf_counter()

        def client():
            for i in range(n_req):
                dt = arrivals[i] - (time.perf_counter() - t_start)
                if dt > 0:
                    time.sleep(dt)
                op = ops[draws[i][0]][1]
                prec = "fmm" if op.N >= args.serve_fmm_min else "fp32"
                tickets[i] = sv.submit(op, rhs[i], tol=args.serve_tol, prec=prec)

        c = th.Thread(target=client)
        c.start()
        lat, res = [], []
        for i in range(n_req):
            while tickets[i] is None:
                time.sleep(0.0005)
            u, info, l = sv.wait(tickets[i])
            lat.append(l)
            res.append(info.residual)
        c.join()
        wall = time.perf_counter() - t_start
        st = sv.stats()
        sv.close()
        lat = np.array(lat)
        return {"p50_latency_ms": round(float(np.percentile(lat, 50)) * 1e3, 2),
                "p99_latency_ms": round(float(np.percentile(lat, 99)) * 1e3, 2),
                "solves_per_s": round(n_req / wall, 2), "wall_s": round(wall, 3),
                "batches": st["batches"], "max_batch": st["max_batch"],
                "max_residual": float(max(res))}

    served = serve(max_batch=64, n_workers=4)
    plain = serve(max_batch=1, n_workers=1)
    # the same requests all submitted at t = 0: throughput with a full queue
    zero = np.zeros(n_req)
    sat_served = serve(max_batch=64, n_workers=4, arrivals=zero)
    sat_plain = serve(max_batch=1, n_workers=1, arrivals=zero)
    for _, op in ops.values():
        op.close()
    sizes = sorted(s.N for s, _ in ops.values())
    return {"requests": n_req, "arrival_rate_per_s": rate, "seed": 0,
            "operators": len(ops), "geometries": len(geo), "node_range": [sizes[0], sizes[-1]],
            "n_max_drawn": args.serve_nmax, "tol": args.serve_tol,
            "fmm_applies_from_n": args.serve_fmm_min,
            "near_build_s_total": round(sum(builds), 3),
            "near_build_s_max": round(max(builds), 3),
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
    ap.add_argument("--workload", default="ellipsoid_9600")
    ap.add_argument("--oracle-leg", action="store_true")
    ap.add_argument("--oracle-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in launch shapes (for profiler runs, whose timings "
                         "would mislead the autotuner)")
    ap.add_argument("--extras", default="batched,fmm,served,paper",
                    help="comma-separated extra measurements to run (batched, fmm, served, paper)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched, FMM and served measurements")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-nmax", type=int, default=30000)
    ap.add_argument("--serve-tol", type=float, default=1e-8)
    ap.add_argument("--serve-budget-gb", type=float, default=32.0)
    ap.add_argument("--serve-fmm-min", type=int, default=40000,
                    help="served operators with at least this many nodes use FMM applies")
    ap.add_argument("--micro", choices=["tc_gemm"], default=None,
                    help="time one kernel alone instead of the solve step (profiling aid)")
    args = ap.parse_args()

    if args.micro == "tc_gemm":
        run_micro_tc_gemm(args)
        return
    if args.oracle_leg:
        rate, desc = oracle_rate(args.workload, args.oracle_seconds)
        print(json.dumps({"value": rate, "sample": desc}))
        return

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))

    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        desc = ""
        for _ in range(args.warmup + args.steps):
            r = run_oracle_subprocess(args.workload, max(2.0, 60.0 / (args.steps + args.warmup)))
            vals.append(r["value"])
            desc = r["sample"]
        print(json.dumps(reference_line(args, vals, desc)))
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
        for name, key, fn in (("batched", "batched_star_24576", run_batched),
                              ("fmm", "fmm_torus_98304", run_fmm), ("served", "served", run_served),
                              ("paper", "paper_problems", run_paper)):
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
                line["cpu_baseline"] = {"value": r["value"], "unit": UNIT, "cores": 1,
                                        "kind": "oracle", "sample": r["sample"]}
            except Exception as e:  # report, do not hide
                line["cpu_baseline"] = {"value": None, "error": str(e)[:300]}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
