"""Build librsim.so (the C ABI over the sm_103a kernels) in-tree with nvcc.

Each translation unit is compiled in parallel for ``sm_103a`` only, then linked
into ``paper_2408_11472_gb300/librsim.so`` (static CUDA runtime), and once more with
``-DRSIM_CHECK`` into ``librsim_check.so`` (kernel bounds checks; a debug build).  The pipe
microbenchmarks the benchmark's roofline divides by are built beside it as
``libalupeaks.so``.  Rebuilds only when a source or header is newer than the
library.

    python paper_2408_11472_gb300/build.py [--force] [--verbose-ptxas]
"""
from __future__ import annotations

import argparse
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(ROOT, "_build", "rsim")
LIB = os.path.join(PKG, "librsim.so")
# the same sources compiled with -DRSIM_CHECK: kernel bounds checks that make the entry points
# return RSIM_ERR_CHECK (a debug build for tests)
CHECK_BUILD_DIR = os.path.join(ROOT, "_build", "rsim_check")
CHECK_LIB = os.path.join(PKG, "librsim_check.so")
# measurement-only microbenchmarks of the arithmetic pipes (the roofline's denominators)
PEAKS_SRC = os.path.join(CSRC, "peaks", "alu_peaks.cu")
PEAKS_LIB = os.path.join(PKG, "libalupeaks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librsim")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not all(os.path.exists(p) for p in (LIB, CHECK_LIB, PEAKS_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(CHECK_LIB))
    return (all(os.path.getmtime(d) <= t for d in _deps())
            and os.path.getmtime(PEAKS_SRC) <= os.path.getmtime(PEAKS_LIB))


def build(force: bool = False, verbose_ptxas: bool = False, quiet: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                    "-I", CSRC, "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        flags += ["-Xptxas", "-v"]
    procs, objs, check_objs = [], [], []
    os.makedirs(CHECK_BUILD_DIR, exist_ok=True)
    peaks_tmp = PEAKS_LIB + ".tmp%d" % os.getpid()
    procs.append((PEAKS_SRC, subprocess.Popen(
        [nvcc] + ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", PEAKS_SRC,
                         "-o", peaks_tmp], stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for src in sources():
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        cobj = os.path.join(CHECK_BUILD_DIR, os.path.basename(src) + ".o")
        check_objs.append(cobj)
        cmd = [nvcc] + flags + ["-DRSIM_CHECK", "-c", src, "-o", cobj]
        procs.append((src + " (RSIM_CHECK)",
                      subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((src, text))
        elif text.strip() and (verbose_ptxas or not quiet):
            sys.stderr.write(text)
    if failed:
        msg = "\n".join("== %s ==\n%s" % (s, t) for s, t in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    os.replace(peaks_tmp, PEAKS_LIB)
    for lib, lib_objs in ((LIB, objs), (CHECK_LIB, check_objs)):
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + lib_objs, check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose-ptxas", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, verbose_ptxas=a.verbose_ptxas))
