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


def test_multi_solve_rejects_bad_arguments_before_any_cuda_call():
    """dwf_cgne_solve_multi checks its job list on the host first: an empty list or
    a job without a handle is refused with DWF_ERR_INVALID_ARG and a message for
    the calling thread (no GPU is touched, so this runs on any machine)."""
    from paper_1501_04950_gb300 import dwf
    lib = dwf.lib()
    assert lib.dwf_cgne_solve_multi(None, 0, None) == 1
    assert lib.dwf_last_error(None) == b"bad argument"
    jobs = (dwf.SolveJobC * 2)()
    assert lib.dwf_cgne_solve_multi(jobs, 2, None) == 1
    assert lib.dwf_last_error(None) == b"job without a handle"


def test_header_is_c99_and_matches_the_binding(tmp_path):
    """include/dwf.h compiles as strict C99 (C callers are part of the boundary),
    and the option, stats and job structs have the sizes and field offsets that
    the ctypes binding uses."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1501_04950_gb300 import dwf
    structs = [("dwf_options", dwf.Options), ("dwf_stats", dwf.Stats),
               ("dwf_solve_job", dwf.SolveJobC)]
    lines = ['#include "dwf.h"', "#include <stddef.h>", "#include <stdio.h>", "int main(void) {"]
    for cname, cls in structs:
        lines.append('  printf("%%zu\\n", sizeof(%s));' % cname)
        for fname, _ in cls._fields_:
            lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "hdr.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "hdr"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    want = []
    for _, cls in structs:
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, fname).offset for fname, _ in cls._fields_]
    assert got == want
