"""Build libdwf.so in-tree with nvcc for sm_103a (GB300).

Every .cu file under csrc/ is compiled in parallel to an object in _build/,
then linked into paper_1501_04950_gb300/libdwf.so.  No CMake, no torch
extension machinery: the library is a plain C-ABI shared object.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdwf.so")
PROBE_SRC = os.path.join(HERE, "probe", "peaks.cu")
PROBE_LIB = os.path.join(HERE, "libdwf_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdwf")
    return path


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def build_probe(force: bool = False) -> str:
    """Compile the arithmetic-throughput probes (probe/peaks.cu) into libdwf_probe.so."""
    if (not force and os.path.exists(PROBE_LIB)
            and os.path.getmtime(PROBE_LIB) > os.path.getmtime(PROBE_SRC)):
        return PROBE_LIB
    cmd = [nvcc()] + ARCH + FLAGS + ["-shared", PROBE_SRC, "-o", PROBE_LIB]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (PROBE_SRC, " ".join(cmd), r.stderr))
    return PROBE_LIB


def build(verbose: bool = False, force: bool = False, extra_flags=None) -> str:
    """Compile csrc/*.cu and link libdwf.so (and the probe library); returns the
    library path."""
    os.makedirs(BUILD, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(
        os.path.join(HERE, "..", "include", "*.h"))
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in sources]
    flags = FLAGS + list(extra_flags or [])
    hdr_time = _newest(headers) if headers else 0.0

    def compile_one(src, obj):
        if (not force and os.path.exists(obj) and os.path.getmtime(obj) > os.path.getmtime(src)
                and os.path.getmtime(obj) > hdr_time):
            return obj, ""
        cmd = [nvcc()] + ARCH + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(sources) + 1, os.cpu_count() or 4))) as ex:
        probe = ex.submit(build_probe, force)
        for obj, log in ex.map(lambda so: compile_one(*so), zip(sources, objs)):
            if verbose and log:
                print(log)
        probe.result()
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest(objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
