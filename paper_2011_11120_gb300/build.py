"""Build the in-tree CUDA libraries for sm_103a with nvcc (no cmake, no torch extension).

    python -m paper_2011_11120_gb300.build

Produces ``paper_2011_11120_gb300/libmdc_gb300.so`` (the product library behind
``include/mdc.h``) and ``synth/libsynth_gen.so`` (the synthetic-workload
generator).  Translation units compile in parallel; each has one -gencode.

    python -m paper_2011_11120_gb300.build --debug

also builds ``libmdc_gb300_debug.so``: the same sources compiled with MDC_CHECK_BOUNDS, whose
kernels check their global indices against the buffer extents (a miss is recorded in the handle's
error flag and the access skipped; ``mdc_device_status`` reports MDC_ERR_BOUNDS).  Setting
MDC_LIB_DEBUG=1 makes the Python binding load it instead of the release library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libmdc_gb300.so")
DEBUG_LIB = os.path.join(PKG, "libmdc_gb300_debug.so")
SYNTH_LIB = os.path.join(ROOT, "synth", "libsynth_gen.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
           "-Xptxas", "-v"] + ARCH

SOURCES = ["api.cu", "fft.cu", "product.cu", "lsqr.cu", "static_scratch.cu", "mdd.cu", "tc_gemm.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str, obj: str, log: str, extra=()) -> None:
    cmd = [nvcc(), "-c", src, "-o", obj] + NVFLAGS + list(extra)
    with open(log, "w") as fh:
        res = subprocess.run(cmd, stdout=fh, stderr=subprocess.STDOUT)
    if res.returncode != 0:
        sys.stderr.write(open(log).read())
        raise RuntimeError(f"nvcc failed for {src}")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "mdc.h"))
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append((src, obj, obj + ".log"))
    synth_src = os.path.join(ROOT, "synth", "csrc", "synth_gen.cu")
    synth_obj = os.path.join(BUILD, "synth_gen.o")
    if force or _stale(synth_obj, [synth_src]):
        jobs.append((synth_src, synth_obj, synth_obj + ".log"))
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(lambda j: _compile(*j), jobs))
    if force or _stale(LIB, objs):
        subprocess.run([nvcc(), "-shared", "-o", LIB] + objs + ARCH, check=True)
    if force or _stale(SYNTH_LIB, [synth_obj]):
        subprocess.run([nvcc(), "-shared", "-o", SYNTH_LIB, synth_obj] + ARCH, check=True)
    if verbose:
        for s in SOURCES:
            print(open(os.path.join(BUILD, s.replace(".cu", ".o")) + ".log").read())
    return LIB


def build_debug(force: bool = False) -> str:
    """The bounds-checked library (MDC_CHECK_BOUNDS), beside the release one."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "mdc.h"))
    jobs, objs = [], []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s.replace(".cu", ".debug.o"))
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append((src, obj, obj + ".log", ["-DMDC_CHECK_BOUNDS"]))
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs) or 1, os.cpu_count() or 4))) as ex:
        list(ex.map(lambda j: _compile(*j), jobs))
    if force or _stale(DEBUG_LIB, objs):
        subprocess.run([nvcc(), "-shared", "-o", DEBUG_LIB] + objs + ARCH, check=True)
    return DEBUG_LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
    if "--debug" in sys.argv:
        print(build_debug(force="--force" in sys.argv))
