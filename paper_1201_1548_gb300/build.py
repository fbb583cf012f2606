"""Build libbsres.so (the CUDA library behind the C ABI in include/bsres.h) in-tree.

Every translation unit is compiled for sm_103a only, in parallel, and linked with nvcc.
Usage: ``python -m paper_1201_1548_gb300.build [--verbose-ptxas] [--debug]``; the binding
loads the debug library when the environment sets BSRES_DEBUG=1.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbsres.so")
# the debug build: every stage kernel bounds-checks its global accesses (BS_DEBUG_CHECKS)
# and reports a failed check through the call's status instead of faulting
DEBUG_OUT_DIR = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(HERE, "libbsres_debug.so")

SOURCES = ["resultant_kernels.cu", "tables.cu", "launch.cu", "api.cu", "gcd.cu", "modgcd.cu", "probe.cu", "noalloc.cu", "serve.cu", "bigcrt.cu", "yun.cu", "psc.cu", "fiber.cu", "content.cu", "mult.cu", "bigcd.cu"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xcompiler", "-Wall", "-diag-suppress", "177"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src, ptxas_verbose=False, debug=False):
    obj = os.path.join(DEBUG_OUT_DIR if debug else OUT_DIR, os.path.splitext(src)[0] + ".o")
    srcp = os.path.join(CSRC, src)
    cmd = [_nvcc(), *ARCH, *FLAGS, *(["-DBS_DEBUG_CHECKS"] if debug else []), "-c", srcp, "-o", obj]
    if ptxas_verbose:
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return obj, res.stderr


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "bsres.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, ptxas_verbose=False, quiet=True, debug=False):
    """Compile and link libbsres.so (debug=True: libbsres_debug.so with the kernels' bounds
    checks compiled in); returns its path."""
    lib = DEBUG_LIB if debug else LIB
    os.makedirs(DEBUG_OUT_DIR if debug else OUT_DIR, exist_ok=True)
    if not force and not ptxas_verbose and not _stale(lib):
        return lib
    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, ptxas_verbose, debug), SOURCES))
    if ptxas_verbose:
        for (_, log), src in zip(results, SOURCES):
            print(f"== {src}\n{log}")
    objs = [o for o, _ in results]
    tmp = lib + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    if not quiet:
        print(f"built {lib}")
    return lib


if __name__ == "__main__":
    build(force=True, ptxas_verbose="--verbose-ptxas" in sys.argv, quiet=False,
          debug="--debug" in sys.argv)
