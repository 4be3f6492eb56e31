"""Build the CUDA library libparametrix.so in-tree for sm_103a (nvcc, no cmake).

Each translation unit compiles in parallel; the shared library links against
the shared CUDA runtime so that it shares the process's runtime with PyTorch.
"""

from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libparametrix.so")
CHECKED_LIB = os.path.join(HERE, "libparametrix_checked.so")
SOURCES = ["pm_api.cu", "pm_batch.cu", "pm_bvp.cu", "pm_check.cu", "pm_direct.cu", "pm_ffmat.cu", "pm_ffsum.cu", "pm_fmm.cu", "pm_green.cu", "pm_helm.cu", "pm_nearfield.cu", "pm_server.cu", "pm_solve.cu", "pm_symsum.cu", "pm_tcgemm.cu", "pm_tri.cu", "pm_tune.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, extra_flags=(), checked: bool = False) -> str:
    """Compile and link the library; checked=True builds libparametrix_checked.so with
    -DPM_BOUNDS_CHECK (pm_surface_check before and a finite scan after every apply)
    in its own object folder."""
    if checked:
        return _build(BUILD + "_checked", CHECKED_LIB, verbose, force,
                      ("-DPM_BOUNDS_CHECK", *extra_flags))
    return _build(BUILD, LIB, verbose, force, tuple(extra_flags))


def _build(build_dir, lib_path, verbose, force, extra_flags) -> str:
    BUILD, LIB = build_dir, lib_path
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers.append(os.path.join(HERE, "..", "include", "parametrix.h"))
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _newer(o, [s] + headers):
            jobs.append([nvcc(), *ARCH, *FLAGS, *extra_flags, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        list(ex.map(run, jobs))
    if jobs or force or _newer(LIB, objs):
        run([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", LIB, *objs])
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
