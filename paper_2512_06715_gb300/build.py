"""In-tree build of the two native libraries.

* ``lib/libucgen.so``  -- host-only C++ instance generator (``include/uc_lp.h``).
* ``lib/libucpdhg.so`` -- CUDA solver for sm_103a behind the C ABI of
  ``include/pdhg.h``.

Translation units compile in parallel; one ``-gencode`` (sm_103a) only.  The
build runs identically on x86_64 (cross compile, no GPU needed) and on aarch64.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
LIBDIR = PKG / "lib"
OBJDIR = PKG / "_build"
INCLUDE = ROOT / "include"

ARCH = "-gencode=arch=compute_103a,code=sm_103a"
CUDA_SOURCES = [
    "pdhg_api.cu",
    "pdhg_layout.cu",
    "pdhg_kernels.cu",
    "pdhg_kkt.cu",
    "pdhg_batched.cu",
    "pdhg_adjoint.cu",
    "pdhg_noalloc.cu",
    "pdhg_staged.cu",
    "pdhg_rowstaged.cu",
    "pdhg_ring.cu",
]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libucpdhg.so")


def _run(cmd: list[str]) -> None:
    proc = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if proc.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + proc.stdout)
    if os.environ.get("UCPDHG_BUILD_VERBOSE") and proc.stdout.strip():
        sys.stderr.write(proc.stdout)


def _stale(target: Path, deps: list[Path]) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps)


def build_ucgen(force: bool = False) -> Path:
    LIBDIR.mkdir(exist_ok=True)
    out = LIBDIR / "libucgen.so"
    src = CSRC / "ucgen.cpp"
    if force or _stale(out, [src, INCLUDE / "uc_lp.h"]):
        cxx = os.environ.get("CXX", "g++")
        _run([cxx, "-O2", "-std=c++17", "-fPIC", "-shared", "-I", str(INCLUDE), str(src), "-o", str(out)])
    return out


def build_pdhg(force: bool = False, extra_flags: list[str] | None = None) -> Path:
    LIBDIR.mkdir(exist_ok=True)
    OBJDIR.mkdir(exist_ok=True)
    nvcc = _nvcc()
    out = LIBDIR / "libucpdhg.so"
    headers = sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))
    flags = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", str(INCLUDE),
             "--expt-relaxed-constexpr"] + list(extra_flags or [])
    srcs = [CSRC / s for s in CUDA_SOURCES if (CSRC / s).exists()]
    objs = [OBJDIR / (s.stem + ".o") for s in srcs]

    def compile_one(pair):
        src, obj = pair
        if force or _stale(obj, [src] + headers):
            _run([nvcc] + flags + ["-c", str(src), "-o", str(obj)])

    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        list(ex.map(compile_one, zip(srcs, objs)))
    if force or _stale(out, objs):
        _run([nvcc, ARCH, "-shared", "-o", str(out)] + [str(o) for o in objs])
    return out


def build(force: bool = False) -> None:
    build_ucgen(force)
    build_pdhg(force)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print("built", LIBDIR)
