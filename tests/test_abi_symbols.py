"""The C-ABI library loads and exports every function include/*.h declares
(no GPU needed: nothing is called that touches a device)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
DECL = re.compile(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\**\s*(bn_[a-z_0-9]+)\s*\(", re.M)


def declared_functions():
    names = set()
    for h in sorted((ROOT / "include").glob("*.h")):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names.update(DECL.findall(text))
    return sorted(names)


def test_headers_declare_the_entry_points():
    names = declared_functions()
    for required in ["bn_add", "bn_mul_quad", "bn_mul_ntt", "bn_plan_create", "bn_plan_execute",
                     "bn_plan_execute_host", "bn_plan_destroy"]:
        assert required in names


def test_library_exports_all_declared_symbols():
    from paper_2405_14642_gb300 import _build
    try:
        path = _build.build()
    except RuntimeError as e:  # pragma: no cover - no toolkit on this machine
        pytest.skip(f"cannot build the CUDA library here: {e}")
    lib = ctypes.CDLL(str(path))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.bn_status_str.restype = ctypes.c_char_p
    assert lib.bn_status_str(4) == b"unsupported size"
    lib.bn_version.restype = ctypes.c_int
    assert lib.bn_version() >= 100


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2405_14642_gb300 import _binding, _build
    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_build, "library_path", lambda: tmp_path / "missing.so")
    with pytest.raises(RuntimeError, match="not built"):
        _binding.load()
