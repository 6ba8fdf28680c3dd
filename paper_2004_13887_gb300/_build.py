"""Build the CUDA library libsph.so in-tree for sm_103a (nvcc, no torch linkage)."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libsph.so")
LIB_CHECKED = os.path.join(HERE, "libsph_checked.so")   # bounds-checked debug build (SPH_CHECKED)
SOURCES = ["sph.cu", "sph_batch.cu", "sph_noalloc.cu", "sph_schur.cu"]
HEADERS = ["sph_device.cuh", "sph_kernels.cuh", "sph_host.cuh", "sph_lines.cuh", "sph_adjoint.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "sph.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile csrc/*.cu into libsph.so (skipped when up to date): one nvcc per
    translation unit, run side by side, then one link.  checked: the
    bounds-checked debug build libsph_checked.so instead (-DSPH_CHECKED)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    tag = f".tmp{os.getpid()}{'c' if checked else ''}"
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(HERE, os.path.splitext(src)[0] + tag + ".o")
        cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I",
               os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, src), "-o", obj]
        if checked:
            cmd.insert(2, "-DSPH_CHECKED")
        if verbose:
            cmd.insert(2, "-Xptxas=-v")
        procs.append(subprocess.Popen(cmd))
        objs.append(obj)
    try:
        for p, src in zip(procs, SOURCES):
            if p.wait() != 0:
                raise subprocess.CalledProcessError(p.returncode, f"nvcc {src}")
        tmp = lib + tag
        subprocess.run([nvcc(), ARCH, "-shared", "-o", tmp] + objs, check=True)
        os.replace(tmp, lib)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return lib
