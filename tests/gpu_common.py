"""Helpers shared by the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np

import oracle as O
from synthetic import gauge_field


def site_norm_error(got, ref):
    """max_x |got(x) - ref(x)|_2 / RMS_x |ref(x)|_2 over 5D half-sites [Ls][Vh][4][3]."""
    d = np.sqrt((np.abs(got - ref) ** 2).sum(axis=(-1, -2)))
    r = np.sqrt((np.abs(ref) ** 2).sum(axis=(-1, -2)))
    return float(d.max() / np.sqrt((r ** 2).mean()))


def make_case(L, Ls, coeff="mobius", alpha=1.3, m=0.05, M5=-1.8, eps=0.5, seed=0, bc_t=1,
              black=0):
    if coeff == "shamir":
        b, c = np.ones(Ls), np.zeros(Ls)
    elif coeff == "mobius":
        b, c = np.full(Ls, 1.5), np.full(Ls, 0.5)
    else:
        rng = np.random.default_rng(99)
        b = 1.0 + rng.uniform(0.0, 1.0, Ls)
        c = rng.uniform(-0.5, 0.8, Ls)
    U = gauge_field(L, eps, seed=seed)
    sysm = O.DWFSystem(L, Ls, M5, m, alpha, b, c, U, bc_t=float(bc_t), black_parity=black)
    return sysm
