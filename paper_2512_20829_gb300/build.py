"""Build libfla.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into one shared
library with the CUDA runtime linked statically (nvcc device-links the
relocatable objects of the persistent window kernel).  ``records.cu`` is compiled
without FMA contraction (its double-precision values decide the kernel's
truncation test and are formed one rounding per operation).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libfla.so")

SOURCES = ["api.cu", "carrier.cu", "advance.cu", "binning.cu", "records.cu", "deposit.cu", "gather2d.cu", "noalloc.cu",
           "mlp.cu", "learn.cu", "batch.cu", "ns.cu"]
NO_FMA = {"records.cu"}
# The persistent window kernel (window.cu) calls phase functions that these
# files define under FLA_WINDOW_PHASES: each is compiled a second time into
# relocatable device code with the namespace renamed, so the phases keep their
# file's flags and the kernels of the launch-per-phase path are unchanged.
WINDOW_PHASES = ["carrier.cu", "advance.cu", "binning.cu", "records.cu", "deposit.cu"]
WINDOW_FLAGS = ["-rdc=true", "-Dfla=fla_w", "-DFLA_WINDOW_PHASES", "-Xcompiler", "-fvisibility=hidden", "-maxrregcount=128"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfla")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "fla.h"), __file__]
    return max(os.path.getmtime(f) for f in files if os.path.isfile(f))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    # host code: no FMA contraction either (host-side double values such as the
    # evaporation deadline must round as the expressions are written)
    common = ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "-I", INCLUDE, "--expt-relaxed-constexpr"]
    procs = []
    objs = []
    units = [(src, src.replace(".cu", ".o"), []) for src in SOURCES]
    units += [(src, src.replace(".cu", ".w.o"), WINDOW_FLAGS) for src in WINDOW_PHASES]
    units.append(("window.cu", "window.o", WINDOW_FLAGS))
    for src, oname, extra in units:
        obj = os.path.join(OUT_DIR, oname)
        cmd = [cc, *common, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if src in NO_FMA:
            cmd.insert(1, "-fmad=false")
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((src, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for src, cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([cc, "-shared", *ARCH, "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
