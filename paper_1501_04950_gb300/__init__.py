"""GB300 (sm_103a) alpha-Mobius domain-wall solver (arXiv:1501.04950).

The work runs in libdwf.so (CUDA kernels behind the C ABI of include/dwf.h);
the Python side only marshals arguments.  Import paper_1501_04950_gb300.dwf
for the binding; build the library with paper_1501_04950_gb300.build.build().
"""
from .build import build  # noqa: F401

__all__ = ["build"]
