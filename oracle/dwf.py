"""Oracle: the alpha domain-wall operator D_alpha(m) of Sec. 2, Eq. mobius1.

TEST INFRASTRUCTURE ONLY (see oracle/lattice.py).

D_alpha(m) is an Ls x Ls block matrix in the 5th dimension whose blocks are
D_{i+} = b_i D_w + 1 or D_{i-} = c_i D_w - 1 (Eq. coeff), each multiplied
from the right by a spin matrix built from P_+-, alpha and m.  Written out
row by row (1-based rows/columns as in the paper):

  row 1   : (1,1) D_{1+}(P_- + alpha P_+), (1,2) alpha D_{1-} P_-,
            (1,Ls) -m D_{1-} P_+
  row i   : (i,i-1) alpha D_{i-} P_+, (i,i) alpha D_{i+}, (i,i+1) alpha D_{i-} P_-
  row Ls  : (Ls,1) -m D_{Ls-} P_-, (Ls,Ls-1) alpha D_{Ls-} P_+,
            (Ls,Ls) D_{Ls+}(P_+ + alpha P_-)

Row i uses the row's own coefficients b_i, c_i, including the two corner
blocks.  Blocks that land on the same column (Ls = 2) are added.

The 4D operator inside D_{i+-} is passed in as a function, so the same
literal block sum gives D_alpha (with D_w), its site-local part I (D_w
replaced by (4 + M5) times the identity, Sec. 3 Eq. redblack) and its
hopping part (D_w - (4 + M5)).

P (App. A, Eq. eqP): (P v)_s = P_- v_s + P_+ v_{s+1 mod Ls};
A = diag(1, alpha, ..., alpha) (Sec. 2).
"""
from __future__ import annotations

import numpy as np

from .lattice import ID4, P_MINUS, P_PLUS, spin_mul
from .wilson import dw


def blocks(Ls, alpha, m):
    """Non-zero blocks of Eq. mobius1 as (row i, column j, '+' or '-', spin matrix M).

    Block (i, j) equals D_{i,kind} M with D_{i+} = b_i D_w + 1, D_{i-} = c_i D_w - 1.
    Indices are 0-based (paper's row 1 is i = 0).
    """
    if Ls < 2:
        raise ValueError("Ls >= 2 required")
    out = []
    last = Ls - 1
    out.append((0, 0, "+", P_MINUS + alpha * P_PLUS))
    out.append((0, 1, "-", alpha * P_MINUS))
    out.append((0, last, "-", -m * P_PLUS))
    for i in range(1, last):
        out.append((i, i - 1, "-", alpha * P_PLUS))
        out.append((i, i, "+", alpha * ID4))
        out.append((i, i + 1, "-", alpha * P_MINUS))
    out.append((last, 0, "-", -m * P_MINUS))
    out.append((last, last - 1, "-", alpha * P_PLUS))
    out.append((last, last, "+", P_PLUS + alpha * P_MINUS))
    return out


def dalpha_generic(psi, op4, b, c, alpha, m):
    """sum over the blocks of Eq. mobius1 with D_w -> op4 (a linear 4D operator).

    psi: [Ls][t][z][y][x][4][3].  For row i the projected inputs of the
    D_{i+} blocks are summed into v_plus_i, those of the D_{i-} blocks into
    v_minus_i, and out_i = (b_i op4 + 1) v_plus_i + (c_i op4 - 1) v_minus_i.
    """
    Ls = psi.shape[0]
    vp = np.zeros_like(psi)
    vm = np.zeros_like(psi)
    for i, j, kind, M in blocks(Ls, alpha, m):
        term = spin_mul(M, psi[j])
        if kind == "+":
            vp[i] += term
        else:
            vm[i] += term
    wp = op4(vp)
    wm = op4(vm)
    bb = np.asarray(b, dtype=np.float64).reshape((Ls,) + (1,) * (psi.ndim - 1))
    cc = np.asarray(c, dtype=np.float64).reshape((Ls,) + (1,) * (psi.ndim - 1))
    return bb * wp + vp + cc * wm - vm


def dalpha_generic_adjoint(phi, op4_dag, b, c, alpha, m):
    """Conjugate transpose of dalpha_generic, block by block.

    Block (i, j) = D_{i,kind} M has adjoint M^dagger D_{i,kind}^dagger, with
    D_{i+}^dagger = b_i op4^dagger + 1 and D_{i-}^dagger = c_i op4^dagger - 1
    (b_i, c_i real); it maps row i of phi into column j of the result.
    """
    Ls = phi.shape[0]
    w = op4_dag(phi)
    out = np.zeros_like(phi)
    for i, j, kind, M in blocks(Ls, alpha, m):
        if kind == "+":
            d = b[i] * w[i] + phi[i]
        else:
            d = c[i] * w[i] - phi[i]
        out[j] += spin_mul(np.conj(M.T), d)
    return out


def dalpha(psi, U, M5, b, c, alpha, m, bc_t=1.0):
    """D_alpha(m) psi, Eq. mobius1 with D_w(M5) of Eq. wilson."""
    return dalpha_generic(psi, lambda v: dw(v, U, M5, False, bc_t), b, c, alpha, m)


def dalpha_dag(phi, U, M5, b, c, alpha, m, bc_t=1.0):
    """D_alpha(m)^dagger phi by the literal conjugate transpose of every block."""
    return dalpha_generic_adjoint(phi, lambda v: dw(v, U, M5, True, bc_t), b, c, alpha, m)


def mobius_standard(psi, U, M5, b, c, m, bc_t=1.0):
    """The conventional Mobius domain-wall operator (the alpha = 1 case, Sec. 2).

    (D psi)_s = (b_s D_w + 1) psi_s + (c_s D_w - 1)(P_- psi_{s+1} + P_+ psi_{s-1})
    with the mass boundary psi_{Ls+1} -> -m psi_1 and psi_0 -> -m psi_Ls.
    Written independently of the block list above, for the alpha = 1 check.
    """
    Ls = psi.shape[0]
    out = np.zeros_like(psi)
    for s in range(Ls):
        up = psi[s + 1] if s + 1 < Ls else -m * psi[0]
        dn = psi[s - 1] if s - 1 >= 0 else -m * psi[Ls - 1]
        nb = spin_mul(P_MINUS, up) + spin_mul(P_PLUS, dn)
        out[s] = (b[s] * dw(psi[s], U, M5, False, bc_t) + psi[s]
                  + c[s] * dw(nb, U, M5, False, bc_t) - nb)
    return out


def p_apply(v):
    """(P v)_s = P_- v_s + P_+ v_{s+1 mod Ls} (App. A, Eq. eqP)."""
    return spin_mul(P_MINUS, v) + spin_mul(P_PLUS, np.roll(v, -1, axis=0))


def p_inverse(w):
    """(P^-1 w)_s = P_- w_s + P_+ w_{s-1 mod Ls}; P P^-1 = 1 since P_+- are projectors."""
    return spin_mul(P_MINUS, w) + spin_mul(P_PLUS, np.roll(w, 1, axis=0))


def a_apply(v, alpha):
    """A v with A = diag(1, alpha, ..., alpha) (Sec. 2)."""
    out = v.copy()
    out[1:] *= alpha
    return out
