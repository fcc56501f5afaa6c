"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/dwf.h declares (no CUDA call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "dwf.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dwf_[a-zA-Z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ["dwf_create", "dwf_destroy", "dwf_load_gauge", "dwf_apply_Dbb",
                 "dwf_apply_Dbb_dag", "dwf_cgne_solve", "dwf_force"]:
        assert want in names


def test_library_builds_loads_and_exports():
    from paper_1501_04950_gb300.build import build
    path = build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_1501_04950_gb300 import dwf
    assert set(dwf.EXPORTS) == set(_declared())


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1501_04950_gb300 import dwf
    with pytest.raises(RuntimeError):
        dwf.load_library(str(tmp_path / "missing.so"))
