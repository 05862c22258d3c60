"""Builds the CUDA library ``_lib/libbn_gb300.so`` for sm_103a with nvcc.

Each ``csrc/*.cu`` translation unit compiles in parallel; the objects are
linked into one shared library exporting the C ABI of ``include/bn.h``.
A stamp records the host architecture and a hash of the sources and flags,
so a copy of the tree moved to another machine rebuilds itself.
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


def _stamp() -> str:
    h = hashlib.sha256()
    h.update(platform.machine().encode())
    h.update(" ".join(ARCH_FLAGS + NVCC_FLAGS).encode())
    for f in sorted(list(CSRC.glob("*")) + [ROOT / "include" / "bn.h"]):
        if f.is_file():
            h.update(f.name.encode())
            h.update(f.read_bytes())
    return h.hexdigest()


def library_path() -> Path:
    return LIB_DIR / LIB_NAME


def is_current() -> bool:
    stamp = LIB_DIR / "stamp.txt"
    return library_path().exists() and stamp.exists() and stamp.read_text() == _stamp()


def build(force: bool = False, verbose: bool = False) -> Path:
    """Compile and link the library if it is missing or stale; return its path."""
    if not force and is_current():
        return library_path()
    nvcc = nvcc_path()
    OBJ_DIR.mkdir(parents=True, exist_ok=True)
    LIB_DIR.mkdir(parents=True, exist_ok=True)

    def compile_one(src: Path) -> Path:
        obj = OBJ_DIR / (src.stem + ".o")
        cmd = [nvcc, *ARCH_FLAGS, *NVCC_FLAGS, "-c", str(src), "-o", str(obj)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src.name}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = sources()
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    out = library_path()
    tmp = out.with_name(out.name + f".tmp{os.getpid()}")
    libdir = cuda_lib_dir(nvcc)
    cmd = [nvcc, *ARCH_FLAGS, "-shared", "-cudart", "shared", *map(str, objs), "-o", str(tmp),
           "-Xlinker", f"-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, out)
    (LIB_DIR / "stamp.txt").write_text(_stamp())
    return out


if __name__ == "__main__":
    print(build(force=True, verbose=True))
