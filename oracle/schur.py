"""Oracle: red-black preconditioned operator D_bb of Sec. 3, Eq. redblack.

TEST INFRASTRUCTURE ONLY (see oracle/lattice.py).

With the 4D checkerboard split into black (b) and red (r) sites, D_alpha
has the block form [[I_bb, D_br], [D_rb, I_rr]] where I is the site-local
part of D_alpha (D_w replaced by (4 + M5) times the identity) and D_br, D_rb
are the parity blocks of the hopping part D_alpha - I.  Eq. redblack:

    D_bb = 1_bb - I_bb^-1 D_br I_rr^-1 D_rb .

I^-1 is formed by Gaussian elimination with partial pivoting (LAPACK getrf
through numpy) of the 4 Ls x 4 Ls matrix that I applies to (s, spin) at
every site; colour is untouched by I.

The Schur right-hand side follows from eliminating the red sites:
    r'_b = I^-1 (rhs_b - D_br I^-1 rhs_r)
and the red half of the solution is psi_r = I^-1 (rhs_r - D_rb psi_b).

D_bb^dagger is the conjugate transpose of each factor in reverse order:
    D_bb^dagger = 1 - D_rb^dagger (I^-1)^dagger D_br^dagger (I^-1)^dagger,
with the parity blocks of (D_alpha - I)^dagger built from the literal
adjoint of Eq. mobius1.

The black parity is the even sites unless black_parity = 1 is given.

Sec. 3 contrasts Eq. redblack with the older form of Eq. redblack1,
    D_bb^(1) = I_bb - D_br I_rr^-1 D_rb ,
and with that form's rows scaled from the left: every row s whose
coefficient b_s + c_s (= 1/omega_s for Zolotarev coefficients) exceeds one is
multiplied by 1 / (b_s + c_s).  schur_form 1 and 2 give these operators
(2: S D_bb^(1) with S the diagonal of the row factors); the right-hand side
of form k is the same left factor applied to I r'_b, so the solution psi_b
is the same for all three forms.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .dwf import dalpha_generic, dalpha_generic_adjoint
from .lattice import full_to_half, half_to_full, shape4
from .wilson import dw


@dataclass
class DWFSystem:
    """Parameters of one alpha-Mobius system (Sec. 2) plus the gauge field."""

    lattice: tuple
    Ls: int
    M5: float
    m: float
    alpha: float
    b: np.ndarray
    c: np.ndarray
    U: np.ndarray
    bc_t: float = 1.0
    black_parity: int = 0
    _iinv: np.ndarray = field(default=None, repr=False)

    def __post_init__(self):
        self.b = np.asarray(self.b, dtype=np.float64)
        self.c = np.asarray(self.c, dtype=np.float64)
        if self.b.shape != (self.Ls,) or self.c.shape != (self.Ls,):
            raise ValueError("b and c must have Ls entries")

    # --- parities ---------------------------------------------------------
    @property
    def red_parity(self):
        return 1 - self.black_parity

    # --- operators on full 5D fields ------------------------------------
    def local_op(self, psi):
        """I psi: Eq. mobius1 with D_w -> (4 + M5) 1."""
        k = 4.0 + self.M5
        return dalpha_generic(psi, lambda v: k * v, self.b, self.c, self.alpha, self.m)

    def hop_op(self, psi):
        """(D_alpha - I) psi: Eq. mobius1 with D_w -> D_w - (4 + M5)."""
        k = 4.0 + self.M5
        return dalpha_generic(
            psi, lambda v: dw(v, self.U, self.M5, False, self.bc_t) - k * v,
            self.b, self.c, self.alpha, self.m)

    def hop_op_dag(self, phi):
        """(D_alpha - I)^dagger phi, block by block."""
        k = 4.0 + self.M5
        return dalpha_generic_adjoint(
            phi, lambda v: dw(v, self.U, self.M5, True, self.bc_t) - k * v,
            self.b, self.c, self.alpha, self.m)

    # --- the site-local inverse ------------------------------------------
    def local_matrix(self):
        """The 4Ls x 4Ls matrix of I on (s, spin), index s * 4 + spin."""
        Ls = self.Ls
        n = 4 * Ls
        mat = np.zeros((n, n), dtype=np.complex128)
        for s in range(Ls):
            for sp in range(4):
                e = np.zeros((Ls, 1, 1, 1, 1, 4, 1), dtype=np.complex128)
                e[s, 0, 0, 0, 0, sp, 0] = 1.0
                col = self.local_op(e).reshape(Ls, 4)
                mat[:, s * 4 + sp] = col.reshape(n)
        return mat

    def local_inverse(self):
        if self._iinv is None:
            self._iinv = np.linalg.inv(self.local_matrix())
        return self._iinv

    def apply_local_matrix(self, mat, h):
        """Apply a 4Ls x 4Ls (s, spin) matrix to a half-field h[Ls][Vh][4][3]."""
        Ls = self.Ls
        m4 = mat.reshape(Ls, 4, Ls, 4)
        return np.einsum("aibj,bnjc->anic", m4, h)

    def iinv(self, h):
        return self.apply_local_matrix(self.local_inverse(), h)

    def iinv_dag(self, h):
        return self.apply_local_matrix(np.conj(self.local_inverse().T), h)

    # --- parity blocks ----------------------------------------------------
    def _block(self, op, h, p_in, p_out):
        return full_to_half(op(half_to_full(h, self.lattice, p_in)), self.lattice, p_out)

    def d_rb(self, hb):
        return self._block(self.hop_op, hb, self.black_parity, self.red_parity)

    def d_br(self, hr):
        return self._block(self.hop_op, hr, self.red_parity, self.black_parity)

    def d_rb_dag(self, hr):
        """(D_rb)^dagger: red -> black, from the adjoint of the hopping part."""
        return self._block(self.hop_op_dag, hr, self.red_parity, self.black_parity)

    def d_br_dag(self, hb):
        """(D_br)^dagger: black -> red."""
        return self._block(self.hop_op_dag, hb, self.black_parity, self.red_parity)

    # --- Eq. redblack -------------------------------------------------------
    def dbb(self, hb):
        """D_bb psi_b = psi_b - I^-1 D_br I^-1 D_rb psi_b (Eq. redblack)."""
        return hb - self.iinv(self.d_br(self.iinv(self.d_rb(hb))))

    def dbb_dag(self, hb):
        """D_bb^dagger phi_b = phi_b - D_rb^+ (I^-1)^+ D_br^+ (I^-1)^+ phi_b."""
        return hb - self.d_rb_dag(self.iinv_dag(self.d_br_dag(self.iinv_dag(hb))))

    # --- Eq. redblack1 and its row-scaled form (Sec. 3) --------------------
    def row_scale(self):
        """S_s = 1 / (b_s + c_s) where b_s + c_s > 1, else 1."""
        a = self.b + self.c
        return np.where(a > 1.0, 1.0 / a, 1.0)

    def _scale_rows(self, h):
        return self.row_scale().reshape(self.Ls, 1, 1, 1) * h

    def dbb_plain(self, hb):
        """I_bb psi_b - D_br I^-1 D_rb psi_b (Eq. redblack1)."""
        return self.apply_local_matrix(self.local_matrix(), hb) - self.d_br(self.iinv(self.d_rb(hb)))

    def dbb_plain_dag(self, hb):
        """(Eq. redblack1)^dagger = I^+ - D_rb^+ (I^-1)^+ D_br^+."""
        return (self.apply_local_matrix(np.conj(self.local_matrix().T), hb)
                - self.d_rb_dag(self.iinv_dag(self.d_br_dag(hb))))

    def schur_operator(self, form):
        """(apply, apply_dagger, left factor of the right-hand side) of form 0, 1 or 2."""
        if form == 0:
            return self.dbb, self.dbb_dag, lambda r: r
        if form == 1:
            return (self.dbb_plain, self.dbb_plain_dag,
                    lambda r: self.apply_local_matrix(self.local_matrix(), r))
        if form == 2:
            return (lambda h: self._scale_rows(self.dbb_plain(h)),
                    lambda h: self.dbb_plain_dag(self._scale_rows(h)),
                    lambda r: self._scale_rows(self.apply_local_matrix(self.local_matrix(), r)))
        raise ValueError("schur form must be 0, 1 or 2")

    def schur_rhs(self, rhs_full):
        """r'_b = I^-1 (rhs_b - D_br I^-1 rhs_r) from a full 5D right-hand side."""
        rb = full_to_half(rhs_full, self.lattice, self.black_parity)
        rr = full_to_half(rhs_full, self.lattice, self.red_parity)
        return self.iinv(rb - self.d_br(self.iinv(rr)))

    def reconstruct(self, hb, rhs_full):
        """Full 5D psi from psi_b: psi_r = I^-1 (rhs_r - D_rb psi_b)."""
        rr = full_to_half(rhs_full, self.lattice, self.red_parity)
        hr = self.iinv(rr - self.d_rb(hb))
        return (half_to_full(hb, self.lattice, self.black_parity)
                + half_to_full(hr, self.lattice, self.red_parity))

    def vh(self):
        Lt, Lz, Ly, Lx = shape4(self.lattice)
        return Lt * Lz * Ly * Lx // 2
