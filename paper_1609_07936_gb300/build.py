"""Builds libsail.so in this directory with nvcc for sm_103a.

Each translation unit compiles in its own nvcc process (in parallel), then one
nvcc -shared links them.  exact64.cu is compiled with -fmad=false: its FP64
kernels round every product and sum on their own.  Host code is compiled
with -ffp-contract=off for the same reason.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsail.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
          "-I", INCLUDE, "-I", CSRC]
UNITS = {
    "api.cu": [],
    "exact64.cu": ["-fmad=false"],
    "sweep_fp32.cu": [],
    "sweep_walk.cu": [],
    "sweep_hastings.cu": [],
    "sweep_guard.cu": [],
    "sweep_shared.cu": [],
    "sweep_shared8.cu": [],
    "sweep_shared4.cu": [],
    "sweep_shared2.cu": [],
    "sweep_batch8.cu": [],
    "sweep_batch16.cu": [],
    "resync_fp32.cu": [],
    "resync_tc.cu": [],
    "resync_tma.cu": [],
    "noalloc.cu": ["-fmad=false"],
}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    out = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".cu", ".cuh"))]
    out.append(os.path.join(INCLUDE, "sail.h"))
    out.append(os.path.abspath(__file__))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    procs = []
    objs = []
    for unit, extra in UNITS.items():
        obj = os.path.join(bdir, unit.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *COMMON, *extra, "-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    errors = []
    for unit, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            errors.append(f"{unit}:\n{out.decode(errors='replace')}")
        elif verbose and out:
            print(out.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed\n" + "\n".join(errors))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
