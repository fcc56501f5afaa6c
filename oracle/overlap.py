"""Oracle: dense 4D overlap operator of App. A/B, for small-lattice checks.

TEST INFRASTRUCTURE ONLY (see oracle/lattice.py).

App. A reduces the domain-wall system to the 4D operator
    D_OV(m) = 1/2 [ (1 + m) + (1 - m) gamma5 eps ],
with eps = (S - 1)(S + 1)^-1 written in the polar (tanh) form of Eq. polar,
    eps = [prod_i (1 + a_i X_i) - prod_i (1 - a_i X_i)]
          [prod_i (1 + a_i X_i) + prod_i (1 - a_i X_i)]^-1 ,
and Eq. argument,
    a_i X_i = (b_i + c_i) gamma5 D_w (2 + (b_i - c_i) D_w)^-1
(the printed equation's "D" in the denominator is read as D_w).  App. B
shows that the 4D propagator y_1 of Eq. tosolve solves D_OV(m) y_1 = b_1.

Everything here is dense (dimension 12 V) and meant for 2^4 lattices.  The
products are taken i = 1..Ls from left to right; the X_i commute whenever
b_i - c_i is the same for all i, which holds for every coefficient set the
paper uses.
"""
from __future__ import annotations

import numpy as np

from .lattice import GAMMA5, volume
from .wilson import dw


def dense_operator(apply, n, shape):
    """Dense matrix of a linear map on complex vectors of the given shape."""
    mat = np.zeros((n, n), dtype=np.complex128)
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1.0
        mat[:, k] = apply(e.reshape(shape)).reshape(n)
    return mat


def dense_dw(U, lattice, M5, bc_t=1.0):
    from .lattice import shape4
    shp = shape4(lattice) + (4, 3)
    n = volume(lattice) * 12
    return dense_operator(lambda v: dw(v, U, M5, False, bc_t), n, shp)


def dense_gamma5(lattice):
    return np.kron(np.eye(volume(lattice)), np.kron(GAMMA5, np.eye(3)))


def sign_tanh_form(dwm, g5, b, c):
    """eps of Eq. polar with a_i X_i from Eq. argument (dense)."""
    n = dwm.shape[0]
    one = np.eye(n, dtype=np.complex128)
    nplus = one.copy()
    nminus = one.copy()
    for bi, ci in zip(b, c):
        ax = (bi + ci) * g5 @ dwm @ np.linalg.inv(2.0 * one + (bi - ci) * dwm)
        nplus = nplus @ (one + ax)
        nminus = nminus @ (one - ax)
    return (nplus - nminus) @ np.linalg.inv(nplus + nminus)


def overlap_operator(dwm, g5, b, c, m):
    """D_OV(m) = 1/2 [(1 + m) + (1 - m) gamma5 eps]."""
    n = dwm.shape[0]
    eps = sign_tanh_form(dwm, g5, b, c)
    return 0.5 * ((1.0 + m) * np.eye(n) + (1.0 - m) * g5 @ eps)
