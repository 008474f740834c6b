"""Build libhweno.so (the CUDA kernels + C ABI) in-tree for sm_103a.

Every .cu under csrc/ is compiled separately (in parallel) with
``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3`` and linked into
``paper_2607_24325_b300/libhweno.so``.  ``-Xptxas -v`` output (registers,
spills, shared memory) is kept in ``_build/ptxas.log`` for inspection.
``build(checked=True)`` makes ``libhweno_checked.so`` from the same sources
with ``-DHWENO_CHECKED`` (index checks in the stage kernels; see
include/hweno_checked.h), in ``_build/checked``; ``build(noscreen=True)``
makes ``libhweno_noscreen.so`` with ``-DHWENO_SCREEN_OFF`` (the mixed
precision's FP32 screen off: every lane takes the FP64 indicator), in
``_build/noscreen``, for the test that the screen changes no output bit.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libhweno.so")
LIB_CHECKED = os.path.join(PKG, "libhweno_checked.so")
LIB_NOSCREEN = os.path.join(PKG, "libhweno_noscreen.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _fingerprint(flags: list[str]) -> str:
    """Hash of every source and header and of the compiler flags: a library
    is rebuilt whenever it was built from different contents (file times
    alone miss an edit made while a build was running)."""
    h = hashlib.sha256(" ".join(flags).encode())
    deps = sorted([os.path.join(CSRC, f) for f in os.listdir(CSRC)] +
                  [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)])
    for d in deps:
        if os.path.isfile(d):
            h.update(os.path.basename(d).encode())
            with open(d, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


def _stale(lib: str, fingerprint: str) -> bool:
    if not os.path.exists(lib):
        return True
    try:
        with open(lib + ".stamp") as fh:
            return fh.read().strip() != fingerprint
    except OSError:
        return True


def build(force: bool = False, verbose: bool = False, checked: bool = False, noscreen: bool = False) -> str:
    lib = LIB_CHECKED if checked else (LIB_NOSCREEN if noscreen else LIB)
    bdir = os.path.join(BUILD, "checked") if checked else (os.path.join(BUILD, "noscreen") if noscreen else BUILD)
    common = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
              "-Xptxas", "-v"] + (["-DHWENO_CHECKED"] if checked else []) + (["-DHWENO_SCREEN_OFF"] if noscreen else [])
    fp = _fingerprint(common)  # taken before compiling: an edit during the build makes the next call rebuild
    if not force and not _stale(lib, fp):
        return lib
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [nvcc, *common, "-c", src, "-o", obj]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{p.stderr}")
        return obj, p.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(compile_one, sources()))
    with open(os.path.join(bdir, "ptxas.log"), "w") as fh:
        for obj, log in results:
            fh.write(f"== {os.path.basename(obj)}\n{log}\n")
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stderr}")
    os.replace(tmp, lib)
    with open(lib + ".stamp", "w") as fh:
        fh.write(fp + "\n")
    if verbose:
        print(f"built {lib}", file=sys.stderr)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv,
          noscreen="--noscreen" in sys.argv)
