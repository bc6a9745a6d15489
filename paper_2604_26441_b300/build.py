"""Builds the in-tree CUDA library ``libgmg_b300.so`` for sm_103a with nvcc.

Usage: ``python -m paper_2604_26441_b300.build`` (or ``build_library()``).
The shared object is written next to this file; it links the CUDA runtime
dynamically so that it shares one runtime with PyTorch in the same process.
"""

from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libgmg_b300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd: list[str]) -> subprocess.CompletedProcess:
    return subprocess.run(cmd, capture_output=True, text=True)


def build_library(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
                  out: str | None = None) -> str:
    """Compiles every csrc/*.cu to an object in parallel (one nvcc per file; no
    relocatable device code crosses files), then links the shared library.
    `extra` flags go to every compile (e.g. -DGMG_CHECKED); `out` names another
    library file (default: libgmg_b300.so, rebuilt only when a source is newer)."""
    from concurrent.futures import ThreadPoolExecutor

    lib = out or LIB
    if not force and out is None and not needs_build():
        return lib
    objdir = os.path.join(HERE, "_build", os.path.splitext(os.path.basename(lib))[0])
    os.makedirs(objdir, exist_ok=True)
    base = [nvcc_path(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I",
            os.path.join(ROOT, "include"), *(extra or [])]
    jobs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.splitext(os.path.basename(src))[0] + ".o")
        jobs.append((src, obj, base + ["-c", src, "-o", obj]))
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda j: _run(j[2]), jobs))
    for (src, _, cmd), res in zip(jobs, results):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n" + res.stdout + res.stderr)
        if verbose and res.stderr:
            print(res.stderr, file=sys.stderr)
    link = [nvcc_path(), *ARCH, "-shared", "-cudart", "shared", "-o", lib + ".tmp", *[j[1] for j in jobs]]
    res = _run(link)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + res.stdout + res.stderr)
    os.replace(lib + ".tmp", lib)
    return lib


CHECKED_LIB = os.path.join(HERE, "libgmg_b300_checked.so")


def build_checked_library(force: bool = False) -> str:
    """The bounds-checked build (-DGMG_CHECKED): every checked global access of
    the hot-path kernels records an out-of-range index in a sticky device word
    instead of touching memory outside its buffer.  Rebuilt when a source is
    newer than it."""
    if not force and os.path.exists(CHECKED_LIB):
        t = os.path.getmtime(CHECKED_LIB)
        deps = sources() + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
        if all(os.path.getmtime(d) <= t for d in deps):
            return CHECKED_LIB
    return build_library(force=True, extra=["-DGMG_CHECKED"], out=CHECKED_LIB)


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True,
                        extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
