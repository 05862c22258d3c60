"""Host-side C++ logic of the library, compiled with the host compiler and run
on the CPU (no GPU): the serving loop's result-pool allocator and the cost
model that picks a multiplication kernel."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
CSRC = ROOT / "paper_2405_14642_gb300" / "csrc"
HOST = Path(__file__).resolve().parent / "host"


def _cuda_include():
    for cand in (Path("/usr/local/cuda/include"),):
        if (cand / "cuda_runtime.h").exists():
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = Path(nvcc).resolve().parent.parent / "include"
        if (inc / "cuda_runtime.h").exists():
            return inc
    return None


def _compile(tmp_path, name, sources, needs_cuda_headers=False):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    cmd = [cxx, "-std=c++17", "-O1", "-I", str(CSRC), "-I", str(ROOT / "include")]
    if needs_cuda_headers:
        inc = _cuda_include()
        if inc is None:
            pytest.skip("CUDA headers not found")
        cmd += ["-I", str(inc)]
    exe = tmp_path / name
    cmd += ["-x", "c++", *map(str, sources), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_pool_allocator_matches_first_fit_model(tmp_path):
    exe = _compile(tmp_path, "pool_check", [HOST / "pool_alloc_check.cpp"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_cost_model_choices(tmp_path):
    """The schoolbook product for small operands, the three-prime transform
    from 256 x 256 limbs (8K bits) up, estimates growing with the size."""
    exe = _compile(tmp_path, "cost_check",
                   [HOST / "cost_model_check.cpp", CSRC / "cost_model.cu"], needs_cuda_headers=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    rows = {}
    for line in r.stdout.split("\n"):
        if line.strip():
            na, nb, kind, est = line.split()
            rows[(int(na), int(nb))] = (int(kind), float(est))
    for n in (1, 32, 64, 128):
        assert rows[(n, n)][0] == 1, (n, rows[(n, n)])
    for n in (256, 512, 1024, 2048, 4096, 8192):
        assert rows[(n, n)][0] == 4, (n, rows[(n, n)])
    assert rows[(8192, 1)][0] == 1          # lopsided: 8192 word products
    square = [rows[(n, n)][1] for n in (32, 64, 128, 256, 512, 1024, 2048, 4096, 8192)]
    assert all(x < y for x, y in zip(square, square[1:]))


@pytest.mark.parametrize("orig,bad", [
    ("if (next != free_.end() && next->first == off + bytes) {",
     "if (false && next != free_.end() && next->first == off + bytes) {"),
    ("if (it->second < bytes) continue;", "if (it->second <= bytes) continue;"),
], ids=["no_forward_merge", "strict_fit"])
def test_pool_check_catches_planted_mistakes(tmp_path, orig, bad):
    text = (CSRC / "pool_alloc.h").read_text()
    assert text.count(orig) == 1
    mutant = tmp_path / "inc"
    mutant.mkdir()
    (mutant / "pool_alloc.h").write_text(text.replace(orig, bad))
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "mutant"
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", str(mutant), "-x", "c++",
                        str(HOST / "pool_alloc_check.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode != 0
