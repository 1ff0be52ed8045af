"""Build the sm_103a library ``_build/libpf_gb300.so`` from ``csrc/*.cu`` with nvcc.

Each translation unit is compiled in parallel, then linked with -shared.  The build is
skipped when the library is newer than every source and header.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpf_gb300.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps():
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(ROOT, "include", "pf.h"), os.path.abspath(__file__)]


STUDY_THREADS = (128, 256, 512, 1024)   # threads per CTA of the step kernel's study builds


def lib_path(threads: int | None = None, checked: bool = False, naive: bool = False) -> str:
    """The library, the thread-block study build with `threads` threads per CTA, the
    checked build (index tests in the kernels, -DPF_CHECKED) or the naive-resampling study
    build (a reciprocal per element instead of saved constants, -DPF_NAIVE_RESAMPLE)."""
    if checked:
        return os.path.join(BUILD, "checked", "libpf_gb300.so")
    if naive:
        return os.path.join(BUILD, "naive", "libpf_gb300.so")
    if not threads or threads == 512:
        return LIB
    return os.path.join(BUILD, "t%d" % threads, "libpf_gb300.so")


def up_to_date(threads: int | None = None, checked: bool = False, naive: bool = False) -> bool:
    lib = lib_path(threads, checked, naive)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in deps())


def build(force: bool = False, verbose: bool = False, extra=(), threads: int | None = None,
          checked: bool = False, naive: bool = False) -> str:
    """Build the library (512 threads per CTA); with `threads` in STUDY_THREADS a separate
    study build under _build/t<threads>/ (-DPF_STEP_THREADS); with `checked` the checked
    build under _build/checked/ (-DPF_CHECKED: every kernel index that is in range by
    construction is tested, a miss fails the step with PF_ERR_STATE instead of faulting);
    with `naive` the study build under _build/naive/ (-DPF_NAIVE_RESAMPLE: divisions by S
    and N per element and an integer-to-half conversion per pixel, the form the paper's
    saved-constant optimisation removes)."""
    if threads and threads not in STUDY_THREADS:
        raise ValueError("threads per CTA must be one of %s" % (STUDY_THREADS,))
    if sum(bool(x) for x in (threads and threads != 512, checked, naive)) > 1:
        raise ValueError("one study or checked variant at a time")
    lib = lib_path(threads, checked, naive)
    if not force and up_to_date(threads, checked, naive):
        return lib
    bdir = os.path.dirname(lib)
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    flags = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
             "--expt-relaxed-constexpr", *extra]
    if checked:
        flags.append("-DPF_CHECKED")
    elif naive:
        flags.append("-DPF_NAIVE_RESAMPLE")
    elif lib != LIB:
        flags.append("-DPF_STEP_THREADS=%d" % threads)
    if verbose:
        flags += ["-Xptxas", "-v"]
    procs = []
    objs = []
    for src in sources():
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        procs.append((src, subprocess.Popen([cc, *flags, "-c", src, "-o", obj],
                                            stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if out and (verbose or p.returncode != 0):
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed on: " + ", ".join(os.path.basename(f) for f in failed))
    tmp = lib + ".tmp%d" % os.getpid()
    subprocess.run([cc, ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, lib)
    return lib


CORE_PEAKS_SRC = os.path.join(HERE, "microbench", "core_peaks.cu")
CORE_PEAKS_BIN = os.path.join(BUILD, "core_peaks")


def build_core_peaks(force: bool = False) -> str:
    """Build the CUDA-core throughput microbenchmark (a standalone program) under _build/."""
    if not force and os.path.exists(CORE_PEAKS_BIN) and os.path.getmtime(CORE_PEAKS_BIN) >= os.path.getmtime(
            CORE_PEAKS_SRC):
        return CORE_PEAKS_BIN
    os.makedirs(BUILD, exist_ok=True)
    tmp = CORE_PEAKS_BIN + ".tmp%d" % os.getpid()
    subprocess.run([nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-o", tmp, CORE_PEAKS_SRC], check=True)
    os.replace(tmp, CORE_PEAKS_BIN)
    return CORE_PEAKS_BIN


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
