"""In-tree build of libmsp.so for sm_103a (nvcc, no CMake).

The translation units compile in parallel; the shared library lands in
`paper_2205_03902_gb300/lib/`, object files in `_build/` at the repository root.
"""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(ROOT, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libmsp.so")
SOURCES = ["msp_position.cu", "msp_position_cluster.cu", "msp_api.cu", "msp_noalloc.cu", "msp_smd.cu", "msp_dft.cu",
           "msp_precise.cu", "msp_tcdft.cu", "msp_learn.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmsp")
    return exe


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)] + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libmsp.so if any source is newer than it; returns the library path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    flags = ["-std=c++17", "-O3", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
             "-diag-suppress", "128"]
    if verbose:
        flags += ["-Xptxas", "-v"]
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(OBJDIR, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [cc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            print(out)
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + out)
    tmp = LIB + ".tmp"
    cmd = [cc, "-shared", ARCH, *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


PEAKS_SRC = os.path.join(CSRC, "msp_peaks.cu")
PEAKS_EXE = os.path.join(OBJDIR, "msp_peaks")


def build_peaks() -> str:
    """Compile the stand-alone pipe micro-benchmarks (csrc/msp_peaks.cu, not part of libmsp)
    if stale; returns the executable's path."""
    deps = [PEAKS_SRC, os.path.join(CSRC, "msp_tc.cuh"), __file__]
    if os.path.exists(PEAKS_EXE) and all(os.path.getmtime(d) <= os.path.getmtime(PEAKS_EXE) for d in deps):
        return PEAKS_EXE
    os.makedirs(OBJDIR, exist_ok=True)
    cmd = [nvcc(), "-std=c++17", "-O3", ARCH, "-lineinfo", PEAKS_SRC, "-o", PEAKS_EXE]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return PEAKS_EXE


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
