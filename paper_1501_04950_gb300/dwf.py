"""Thin ctypes binding of libdwf (include/dwf.h).

Argument marshalling only: every step of the path runs in libdwf's CUDA
kernels.  PyTorch supplies device memory (tensor.data_ptr()) and the current
CUDA stream; complex128 tensors are passed as interleaved double pairs in
the canonical layouts of include/dwf.h.  There is no CPU fallback: if the
library is missing the import of this module fails.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdwf.so")

DWF_OK = 0
DWF_ERR_NOT_CONVERGED = 4
FP64, FP32, FP16, BF16 = 0, 1, 2, 3
SOLVER_RELIABLE, SOLVER_DEFECT, SOLVER_FP64 = 0, 1, 2
SCHUR_PRECOND, SCHUR_PLAIN, SCHUR_ROWSCALED = 0, 1, 2
ERRORS = {1: "DWF_ERR_INVALID_ARG", 2: "DWF_ERR_CUDA", 3: "DWF_ERR_OOM",
          4: "DWF_ERR_NOT_CONVERGED", 5: "DWF_ERR_BREAKDOWN", 6: "DWF_ERR_TIMEOUT",
          7: "DWF_ERR_STATE"}


class Options(ctypes.Structure):
    _fields_ = [("precision_inner", ctypes.c_int), ("rb_parity", ctypes.c_int),
                ("bc_t", ctypes.c_int), ("rel_tol", ctypes.c_double), ("maxiter", ctypes.c_int),
                ("reliable_delta", ctypes.c_double), ("solver", ctypes.c_int),
                ("check_every", ctypes.c_int), ("profile", ctypes.c_int),
                ("graph", ctypes.c_int), ("rhs_block", ctypes.c_int),
                ("schur_form", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("true_resid", ctypes.c_double), ("true_resid_5d", ctypes.c_double),
                ("seconds", ctypes.c_double), ("applies", ctypes.c_int),
                ("applies_dag", ctypes.c_int), ("applies_fp64", ctypes.c_int),
                ("kernel_launches", ctypes.c_int), ("apply_ms", ctypes.c_double),
                ("apply_dag_ms", ctypes.c_double), ("applies_fp32", ctypes.c_int),
                ("applies_timed", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveJobC(ctypes.Structure):
    _fields_ = [("handle", ctypes.c_void_p), ("src4d", ctypes.c_void_p),
                ("prop4d", ctypes.c_void_p), ("sol5d", ctypes.c_void_p), ("nrhs", ctypes.c_int),
                ("alphas", ctypes.POINTER(ctypes.c_double)), ("stats", ctypes.POINTER(Stats)),
                ("status", ctypes.c_int)]


EXPORTS = [
    "dwf_default_options", "dwf_create", "dwf_destroy", "dwf_last_error", "dwf_field_bytes",
    "dwf_load_gauge", "dwf_pack_half", "dwf_unpack_half", "dwf_apply_Dbb", "dwf_apply_Dbb_dag",
    "dwf_apply_dalpha", "dwf_cgne_solve", "dwf_solve_normal", "dwf_force",
    "dwf_apply_Dbb_noalloc", "dwf_apply_overlap", "dwf_action", "dwf_cgne_solve_multi",
]
NOALLOC_SCRATCH_BYTES = 32 << 20


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError("libdwf.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "dwf_default_options": (I, [ctypes.POINTER(Options)]),
        "dwf_create": (I, [ctypes.POINTER(P), ctypes.POINTER(I), I, D, D, D,
                           ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(Options)]),
        "dwf_destroy": (I, [P]),
        "dwf_last_error": (ctypes.c_char_p, [P]),
        "dwf_field_bytes": (I, [P, I, ctypes.POINTER(S)]),
        "dwf_load_gauge": (I, [P, P, I, P]),
        "dwf_pack_half": (I, [P, P, P, I, I, P]),
        "dwf_unpack_half": (I, [P, P, P, I, I, P]),
        "dwf_apply_Dbb": (I, [P, P, P, I, I, P]),
        "dwf_apply_Dbb_dag": (I, [P, P, P, I, I, P]),
        "dwf_apply_Dbb_noalloc": (I, [P, P, P, I, I, P]),
        "dwf_apply_dalpha": (I, [P, P, P, D, D, P]),
        "dwf_cgne_solve": (I, [P, P, P, P, I, ctypes.POINTER(D), ctypes.POINTER(Stats), P]),
        "dwf_apply_overlap": (I, [P, P, P, P, I, ctypes.POINTER(D), ctypes.POINTER(Stats), P]),
        "dwf_solve_normal": (I, [P, P, P, ctypes.POINTER(Stats), P]),
        "dwf_force": (I, [P, P, P, P, I, P]),
        "dwf_action": (I, [P, ctypes.POINTER(D), P, P, ctypes.POINTER(Stats), P]),
        "dwf_cgne_solve_multi": (I, [ctypes.POINTER(SolveJobC), I, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


class DWFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERRORS.get(code, code), msg))
        self.code = code


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class DWF:
    """One alpha-Mobius operator D_alpha(m) on a lattice (include/dwf.h, dwf_create)."""

    def __init__(self, lattice, Ls, M5, m, alpha, b, c, **options):
        self.lib = lib()
        opt = Options()
        self.lib.dwf_default_options(ctypes.byref(opt))
        for k, v in options.items():
            if not hasattr(opt, k):
                raise TypeError("unknown option %s" % k)
            setattr(opt, k, v)
        self.lattice = tuple(int(v) for v in lattice)
        self.Ls, self.M5, self.m, self.alpha = int(Ls), float(M5), float(m), float(alpha)
        self.options = opt
        L = (ctypes.c_int * 4)(*self.lattice)
        bb = (ctypes.c_double * Ls)(*[float(v) for v in b])
        cc = (ctypes.c_double * Ls)(*[float(v) for v in c])
        h = ctypes.c_void_p()
        rc = self.lib.dwf_create(ctypes.byref(h), L, self.Ls, self.M5, self.m, self.alpha, bb, cc,
                                 ctypes.byref(opt))
        if rc != DWF_OK:
            raise DWFError(rc, self.lib.dwf_last_error(None).decode())
        self.h = h
        self.V = self.lattice[0] * self.lattice[1] * self.lattice[2] * self.lattice[3]
        self.Vh = self.V // 2

    def _check(self, rc, allow=()):
        if rc != DWF_OK and rc not in allow:
            raise DWFError(rc, self.lib.dwf_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.dwf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- fields -------------------------------------------------------------
    def field_bytes(self, prec):
        n = ctypes.c_size_t()
        self._check(self.lib.dwf_field_bytes(self.h, prec, ctypes.byref(n)))
        return n.value

    def new_field(self, prec, nrhs=1, device="cuda"):
        """An internal half-field buffer (opaque bytes) for nrhs right-hand sides."""
        return torch.zeros(self.field_bytes(prec) * nrhs, dtype=torch.uint8, device=device)

    def load_gauge(self, U):
        self._check(self.lib.dwf_load_gauge(self.h, _ptr(U), int(U.is_cuda), _stream()))

    def pack_half(self, dst, src, prec, nrhs=1):
        self._check(self.lib.dwf_pack_half(self.h, _ptr(dst), _ptr(src), prec, nrhs, _stream()))

    def unpack_half(self, dst, src, prec, nrhs=1):
        self._check(self.lib.dwf_unpack_half(self.h, _ptr(dst), _ptr(src), prec, nrhs, _stream()))

    # --- operators ------------------------------------------------------------
    def apply_Dbb(self, out, inp, prec, nrhs=1):
        self._check(self.lib.dwf_apply_Dbb(self.h, _ptr(out), _ptr(inp), prec, nrhs, _stream()))

    def apply_Dbb_noalloc(self, out, inp, prec, nrhs=1):
        """D_bb through the entry point that allocates nothing (static scratch)."""
        self._check(self.lib.dwf_apply_Dbb_noalloc(self.h, _ptr(out), _ptr(inp), prec, nrhs,
                                                   _stream()))

    def apply_Dbb_dag(self, out, inp, prec, nrhs=1):
        self._check(self.lib.dwf_apply_Dbb_dag(self.h, _ptr(out), _ptr(inp), prec, nrhs, _stream()))

    def apply_dalpha(self, out_full, in_full, alpha=None, m=None):
        alpha = self.alpha if alpha is None else alpha
        m = self.m if m is None else m
        self._check(self.lib.dwf_apply_dalpha(self.h, _ptr(out_full), _ptr(in_full), float(alpha),
                                              float(m), _stream()))

    # --- solvers ----------------------------------------------------------------
    def cgne_solve(self, src4d, prop4d, sol5d=None, nrhs=1, alphas=None, allow_not_converged=False):
        st = (Stats * nrhs)()
        al = None
        if alphas is not None:
            al = (ctypes.c_double * nrhs)(*[float(a) for a in alphas])
        rc = self.lib.dwf_cgne_solve(self.h, _ptr(src4d), _ptr(prop4d), _ptr(sol5d), nrhs, al, st,
                                     _stream())
        self._check(rc, allow=(DWF_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return [s.as_dict() for s in st]

    def apply_overlap(self, src4d, out4d, sol5d=None, nrhs=1, alphas=None):
        """out4d = D_OV(m) src4d through the mass-exchanged 5D solve (dwf_apply_overlap)."""
        st = (Stats * nrhs)()
        al = None
        if alphas is not None:
            al = (ctypes.c_double * nrhs)(*[float(a) for a in alphas])
        self._check(self.lib.dwf_apply_overlap(self.h, _ptr(src4d), _ptr(out4d), _ptr(sol5d), nrhs,
                                               al, st, _stream()))
        return [s.as_dict() for s in st]

    def solve_normal(self, x_half, phi_half):
        st = Stats()
        self._check(self.lib.dwf_solve_normal(self.h, _ptr(x_half), _ptr(phi_half), ctypes.byref(st),
                                              _stream()))
        return st.as_dict()

    def action(self, phi_half, X_half=None):
        """S = Re phi^+ (D_bb^+ D_bb)^-1 phi (dwf_action); returns (S, stats)."""
        S = ctypes.c_double()
        st = Stats()
        self._check(self.lib.dwf_action(self.h, ctypes.byref(S), _ptr(phi_half), _ptr(X_half),
                                        ctypes.byref(st), _stream()))
        return S.value, st.as_dict()

    def force(self, dSdU, phi_half, X_half=None, projected=False):
        self._check(self.lib.dwf_force(self.h, _ptr(dSdU), _ptr(phi_half), _ptr(X_half),
                                       int(bool(projected)), _stream()))


def cgne_solve_multi(jobs, allow_not_converged=False):
    """Propagator solves of several lattices in one call (dwf_cgne_solve_multi).

    jobs: sequence of (op, src4d, prop4d[, nrhs[, alphas[, sol5d]]]) with a
    distinct DWF handle per job (arguments as in DWF.cgne_solve).  Returns one list of stats dicts per job;
    raises DWFError with the first failed job's status and message."""
    n = len(jobs)
    arr = (SolveJobC * n)()
    keep = []
    for i, job in enumerate(jobs):
        op, src, prop = job[:3]
        nrhs = int(job[3]) if len(job) > 3 else 1
        alphas = job[4] if len(job) > 4 else None
        sol = job[5] if len(job) > 5 else None
        st = (Stats * nrhs)()
        al = None
        if alphas is not None:
            al = (ctypes.c_double * nrhs)(*[float(a) for a in alphas])
        keep.append((st, al))
        arr[i].handle = op.h
        arr[i].src4d = src.data_ptr()
        arr[i].prop4d = prop.data_ptr()
        arr[i].sol5d = sol.data_ptr() if sol is not None else None
        arr[i].nrhs = nrhs
        arr[i].alphas = al
        arr[i].stats = st
        arr[i].status = -1
    L = lib()
    rc = L.dwf_cgne_solve_multi(arr, n, _stream())
    if rc != DWF_OK and not (allow_not_converged and rc == DWF_ERR_NOT_CONVERGED):
        raise DWFError(rc, L.dwf_last_error(None).decode())
    return [[s.as_dict() for s in keep[i][0]] for i in range(n)]
