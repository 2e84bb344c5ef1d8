"""Build ``libdv.so`` (the C-ABI CUDA library) in-tree with nvcc for sm_103a.

    python -m paper_2407_11272_b300.build [--force] [--verbose]

Every ``csrc/*.cu`` file is compiled to an object in ``_build/`` and linked
into ``paper_2407_11272_b300/libdv.so`` against the shared CUDA runtime.
``-Xptxas -v`` output (registers, spills, shared memory per kernel) is kept
in ``_build/ptxas.log``.

    python -m paper_2407_11272_b300.build --debug

builds the bounds-checked debug library ``libdv_debug.so`` from the same
sources with ``-DDV_DEBUG`` (objects in ``_build/debug/``): every indexed global
access of the hot kernels is checked against its buffer's length, and an index
outside it is recorded and skipped (``dv_debug_report``). The binding loads it
instead of ``libdv.so`` when the environment variable ``DV_DEBUG`` is ``1``.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
INCLUDE = PKG.parent / "include"
BUILD = PKG.parent / "_build"
LIB = PKG / "libdv.so"
LIB_DEBUG = PKG / "libdv_debug.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
              "-Xptxas", "-v", f"-I{INCLUDE}", f"-I{CSRC}"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdv.so")


def _sources():
    return sorted(CSRC.glob("*.cu"))


def _deps():
    return _sources() + sorted(CSRC.glob("*.cuh")) + sorted(CSRC.glob("*.h")) + sorted(INCLUDE.glob("*.h")) + \
        [Path(__file__)]


def _target(debug: bool):
    return (BUILD / "debug", LIB_DEBUG) if debug else (BUILD, LIB)


def needs_build(debug: bool = False) -> bool:
    lib = _target(debug)[1]
    if not lib.exists():
        return True
    t = lib.stat().st_mtime
    return any(p.stat().st_mtime > t for p in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> Path:
    bdir, lib = _target(debug)
    if not force and not needs_build(debug):
        return lib
    nvcc = _nvcc()
    bdir.mkdir(parents=True, exist_ok=True)
    flags = NVCC_FLAGS + (["-DDV_DEBUG"] if debug else [])
    logs = {}

    def compile_one(src: Path):
        obj = bdir / (src.stem + ".o")
        cmd = [nvcc, *ARCH, *flags, "-c", str(src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        logs[src.name] = r.stdout + r.stderr
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src.name}:\n{r.stdout}\n{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    (bdir / "ptxas.log").write_text("\n".join(f"== {k}\n{v}" for k, v in sorted(logs.items())))
    tmp = lib.with_suffix(f".so.tmp{os.getpid()}")
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64",
           *map(str, objs), "-o", str(tmp)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print((bdir / "ptxas.log").read_text())
    return lib


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--debug", action="store_true", help="build the bounds-checked libdv_debug.so")
    a = ap.parse_args(argv)
    print(build(force=a.force, verbose=a.verbose, debug=a.debug))


if __name__ == "__main__":
    main(sys.argv[1:])
