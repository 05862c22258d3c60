"""Builds the CUDA library ``_lib/libbn_gb300.so`` for sm_103a with nvcc, and
its debug variant ``_lib/libbn_gb300_debug.so`` (compiled with BN_DEBUG: the
kernels' spill, carry and index checks, read through bn_debug_word).

Each ``csrc/*.cu`` translation unit compiles in parallel (both variants in
one pool); the objects are linked into one shared library per variant,
exporting the C ABI of ``include/bn.h``.  A stamp records the host
architecture and a hash of the sources and flags, so a copy of the tree
moved to another machine rebuilds itself.
"""
from __future__ import annotations

import hashlib
import os
import platform
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
LIB_DIR = PKG / "_lib"
OBJ_DIR = ROOT / "_build" / "bn"
LIB_NAME = "libbn_gb300.so"
DEBUG_LIB_NAME = "libbn_gb300_debug.so"
DEBUG_FLAGS = ["-DBN_DEBUG"]
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found (set NVCC or put the CUDA toolkit on PATH)")


def cuda_lib_dir(nvcc: str) -> Path:
    return Path(nvcc).resolve().parent.parent / "lib64"


def sources():
    return sorted(CSRC.glob("*.cu"))


def _stamp(debug: bool = False) -> str:
    h = hashlib.sha256()
    h.update(platform.machine().encode())
    h.update(" ".join(ARCH_FLAGS + NVCC_FLAGS + (DEBUG_FLAGS if debug else [])).encode())
    for f in sorted(list(CSRC.glob("*")) + [ROOT / "include" / "bn.h"]):
        if f.is_file():
            h.update(f.name.encode())
            h.update(f.read_bytes())
    return h.hexdigest()


def library_path(debug: bool = False) -> Path:
    return LIB_DIR / (DEBUG_LIB_NAME if debug else LIB_NAME)


def _stamp_path(debug: bool) -> Path:
    return LIB_DIR / ("stamp_debug.txt" if debug else "stamp.txt")


def is_current(debug: bool = False) -> bool:
    stamp = _stamp_path(debug)
    return library_path(debug).exists() and stamp.exists() and stamp.read_text() == _stamp(debug)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> Path:
    """Compile and link the library (or its debug variant) if it is missing or
    stale; return its path."""
    return build_variants((debug,), force, verbose)[0]


def build_variants(variants=(False, True), force: bool = False, verbose: bool = False):
    """Compile the stale variants' translation units in one parallel pool,
    link each; return the libraries' paths in the order asked."""
    todo = [d for d in variants if force or not is_current(d)]
    if todo:
        nvcc = nvcc_path()
        LIB_DIR.mkdir(parents=True, exist_ok=True)

        def compile_one(job):
            src, debug = job
            odir = OBJ_DIR.with_name(OBJ_DIR.name + ("_debug" if debug else ""))
            odir.mkdir(parents=True, exist_ok=True)
            obj = odir / (src.stem + ".o")
            cmd = [nvcc, *ARCH_FLAGS, *NVCC_FLAGS, *(DEBUG_FLAGS if debug else []), "-c", str(src),
                   "-o", str(obj)]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src.name}{' (debug)' if debug else ''}:\n{r.stderr}")
            if verbose and r.stderr:
                print(r.stderr)
            return debug, obj

        jobs = [(src, d) for d in todo for src in sources()]
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            objs = list(ex.map(compile_one, jobs))
        libdir = cuda_lib_dir(nvcc)
        for d in todo:
            out = library_path(d)
            tmp = out.with_name(out.name + f".tmp{os.getpid()}")
            cmd = [nvcc, *ARCH_FLAGS, "-shared", "-cudart", "shared", *[str(o) for dd, o in objs if dd == d],
                   "-o", str(tmp), "-Xlinker", f"-rpath,{libdir}"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed:\n{r.stderr}")
            os.replace(tmp, out)
            _stamp_path(d).write_text(_stamp(d))
    return [library_path(d) for d in variants]


if __name__ == "__main__":
    print(build(force=True, verbose=True))
