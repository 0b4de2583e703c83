"""Build the SQA / PT library for sm_103a: ``_build/libsqa_gb300.so``.

Plain nvcc, one object per translation unit compiled in parallel, then one
shared-library link.  Host code is compiled with ``-ffp-contract=off`` so the
acceptance tables are rounded operation by operation on any host.

``build(checked=True)`` makes the bounds-checked variant
``_build_checked/libsqa_gb300_checked.so`` (``-DSQA_BOUNDS_CHECK``: every
kernel index is tested before its access, violations are recorded in a device
status word and read with ``sqa_check_status``).  The package loads it instead
of the normal library when ``SQA_GB300_CHECKED=1`` is set.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsqa_gb300.so")
OUT_DIR_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(OUT_DIR_CHECKED, "libsqa_gb300_checked.so")
SOURCES = ("kernels.cu", "capi.cu", "host_plan.cpp", "intpeak.cu", "noalloc.cu", "server.cu", "batch.cu")
HEADERS = ("philox.cuh", "sqa_internal.h", "layout.cuh", "handle.h", "check.cuh")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _flags(verbose_ptxas: bool, checked: bool = False) -> list[str]:
    f = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math",
         "-I", os.path.join(ROOT, "include")]
    if checked:
        f += ["-DSQA_BOUNDS_CHECK"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "sqa.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, checked: bool = False) -> str:
    out_dir, lib = (OUT_DIR_CHECKED, LIB_CHECKED) if checked else (OUT_DIR, LIB)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    flags = _flags(verbose_ptxas, checked)

    def compile_one(src: str) -> str:
        obj = os.path.join(out_dir, src + ".o")
        cmd = [cc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose_ptxas and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([cc, ARCH, "-shared", "-Xcompiler", "-pthread", "-o", tmp, *objs, "-lcudart"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, checked="--checked" in sys.argv))
