"""Build the CUDA library ``libfcm_gb300.so`` in-tree for sm_103a.

Every translation unit is compiled by its own ``nvcc -c`` process, in
parallel, then linked with ``nvcc -shared``. The single-image pass source is
and the recompute-run source are compiled eight times each, once per cluster
count (``-DFCM_INST_C=1..8``), and the
two batched kernels twice each, once per block size (``-DFCM_BATCH_NT`` and
``-DFCM_ROUNDS_NT`` = 256, 512).
Nothing is rebuilt when the library is newer than every source.

With FCM_DEBUG_BOUNDS=1 in the environment the bounds-guarded variant is
built instead, into ``_build_bounds/`` (``-DFCM_DEBUG_BOUNDS``: the kernels
that issue TMA copies or index lookup tables check their indices, skip an
out-of-range access and report FCM_FLAG_BOUNDS); the loader picks the same
variant from the same variable.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
DEBUG_BOUNDS = os.environ.get("FCM_DEBUG_BOUNDS", "0") not in ("", "0")
BUILD = os.path.join(PKG, "_build_bounds" if DEBUG_BOUNDS else "_build")
LIB = os.path.join(BUILD, "libfcm_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-I" + INCLUDE, "-I" + CSRC, "--expt-relaxed-constexpr"] + (["-DFCM_DEBUG_BOUNDS=1"] if DEBUG_BOUNDS else [])


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build")
    return exe


def _units():
    units = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        base = os.path.splitext(os.path.basename(src))[0]
        if base in ("fcm_single_inst", "fcm_recompute_inst"):
            for c in range(1, 9):
                units.append((src, os.path.join(BUILD, f"{base}_c{c}.o"), [f"-DFCM_INST_C={c}"]))
        elif base == "fcm_batched_inst":
            for nt in (256, 512):
                units.append((src, os.path.join(BUILD, f"{base}_nt{nt}.o"), [f"-DFCM_BATCH_NT={nt}"]))
        elif base == "fcm_multi_inst":
            for d in (1, 2, 3, 4):
                units.append((src, os.path.join(BUILD, f"{base}_d{d}.o"), [f"-DFCM_MULTI_D={d}"]))
        elif base == "fcm_rounds_inst":
            for nt in (256, 512):
                units.append((src, os.path.join(BUILD, f"{base}_nt{nt}.o"), [f"-DFCM_ROUNDS_NT={nt}"]))
        else:
            units.append((src, os.path.join(BUILD, base + ".o"), []))
    return units


def _deps():
    return (glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h"))
            + [os.path.abspath(__file__)])


def build(verbose: bool = False, jobs: int | None = None, extra_flags=()) -> str:
    """Compile and link the library; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _deps())
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= newest and not extra_flags:
        return LIB
    exe = nvcc()
    units = _units()

    def compile_one(u):
        src, obj, defs = u
        cmd = [exe, *ARCH, *FLAGS, *extra_flags, *defs, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)} {defs}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    jobs = jobs or max(1, min(len(units), os.cpu_count() or 4))
    with ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
