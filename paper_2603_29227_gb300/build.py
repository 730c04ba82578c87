"""Build libksdf.so (the CUDA library behind include/ksdf.h) in-tree for sm_103a, and beside it
libksdf_peaks.so (include/ksdf_peaks.h: the throughput probes that give the benchmark its roofline
denominators; the product library does not link it).

Each translation unit is compiled by nvcc in parallel, then linked into one shared library with the
static CUDA runtime.  The results land next to this file; nothing is installed elsewhere.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libksdf.so")
PEAKS_OUT = os.path.join(HERE, "libksdf_peaks.so")
PEAKS_SRC = os.path.join(CSRC, "peaks", "ksdf_peaks.cu")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["ksdf_abi.cu", "ksdf_sort.cu", "ksdf_fit.cu", "ksdf_query.cu", "ksdf_backward.cu", "ksdf_noalloc.cu",
           "ksdf_bhm.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-Xptxas",
         "-warn-spills"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libksdf.so")
    return p


def _stale() -> bool:
    if not os.path.exists(OUT) or not os.path.exists(PEAKS_OUT):
        return True
    t = min(os.path.getmtime(OUT), os.path.getmtime(PEAKS_OUT))
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [PEAKS_SRC, __file__]
    deps += [os.path.join(HERE, "..", "include", h) for h in ("ksdf.h", "ksdf_bhm.h", "ksdf_peaks.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and not _stale():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    extra = list(extra or [])

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr.strip():
            sys.stderr.write(r.stderr)
        return obj

    def build_peaks():
        tmp = PEAKS_OUT + ".tmp%d" % os.getpid()
        cmd = [cc, *ARCH, *FLAGS, *extra, "-shared", PEAKS_SRC, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for ksdf_peaks.cu:\n%s\n%s" % (" ".join(cmd), r.stderr))
        os.replace(tmp, PEAKS_OUT)

    with ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        peaks = ex.submit(build_peaks)
        objs = list(ex.map(compile_one, SOURCES))
        peaks.result()
    tmp = OUT + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "-v" in sys.argv else None))
