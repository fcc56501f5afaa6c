"""Oracle: D_bb psi at single black sites, for checks on full-size lattices.

TEST INFRASTRUCTURE ONLY (see oracle/lattice.py).

The whole-lattice oracle (oracle/schur.py) is too slow for 16^3 x 32 x 16
fields inside a test, so this module evaluates Eq. redblack one output site
at a time, literally:

    (D_bb psi)(x) = psi(x) - I^-1 (D_br u)(x),    u(y) = I^-1 (D_rb psi)(y),

where (D_rb psi)(y) and (D_br u)(x) are the hopping part of Eq. mobius1 at one
site: row i is b_i (D_w - (4 + M5)) v_plus_i + c_i (D_w - (4 + M5)) v_minus_i
with v_plus_i / v_minus_i the block sums of Eq. mobius1 at the neighbour
sites, and (D_w - (4 + M5)) v(y) = -1/2 sum_mu [(1 - gamma_mu) U_mu(y)
v(y + mu) + (1 + gamma_mu) U_mu(y - mu)^+ v(y - mu)] (Eq. wilson).

PointwiseDalpha evaluates the full 5D equation of Sec. 2 at one 4D site,
(D_alpha psi)(x) = I psi(x) + ((D_alpha - I) psi)(x), and the propagator
right-hand side rhs = D_1(1) P b of Eq. tosolve with b = (b_1, 0, ..., 0),
(P b)_s = P_- b_s + P_+ b_{s+1} (App. A, Eq. eqP), so that a solution psi of
any size can be checked at sampled sites.
"""
from __future__ import annotations

import numpy as np

from .dwf import blocks
from .lattice import GAMMA, ID4, P_MINUS, P_PLUS
from .schur import DWFSystem


class _SiteOps:
    """Single-site pieces of Eq. mobius1 / Eq. wilson shared by the evaluators."""

    def __init__(self, sys):
        self.sys = sys
        self.Lx, self.Ly, self.Lz, self.Lt = sys.lattice
        self.blk = blocks(sys.Ls, sys.alpha, sys.m)

    def _lex(self, c):
        x, y, z, t = c
        return x + self.Lx * (y + self.Ly * (z + self.Lz * t))

    def _parity(self, c):
        return sum(c) % 2

    def _shift(self, c, mu, d):
        L = (self.Lx, self.Ly, self.Lz, self.Lt)
        cc = list(c)
        cc[mu] += d
        sign = 1.0
        if cc[mu] < 0 or cc[mu] >= L[mu]:
            cc[mu] %= L[mu]
            if mu == 3:
                sign = self.sys.bc_t
        return tuple(cc), sign

    def _link(self, c, mu):
        x, y, z, t = c
        return self.sys.U[t, z, y, x, mu]

    def _block_sums(self, f):
        """v_plus, v_minus [Ls][4][3] of Eq. mobius1 from f [Ls][4][3] at one site."""
        Ls = self.sys.Ls
        vp = np.zeros((Ls, 4, 3), dtype=np.complex128)
        vm = np.zeros((Ls, 4, 3), dtype=np.complex128)
        for i, j, kind, M in self.blk:
            (vp if kind == "+" else vm)[i] += M @ f[j]
        return vp, vm

    def _hop_part(self, c, field_at):
        """(D_alpha - I) applied at site c; field_at(site) -> [Ls][4][3] (zero if wrong parity)."""
        sys = self.sys
        Ls = sys.Ls
        wp = np.zeros((Ls, 4, 3), dtype=np.complex128)
        wm = np.zeros((Ls, 4, 3), dtype=np.complex128)
        for mu in range(4):
            cf, sf = self._shift(c, mu, +1)
            vp, vm = self._block_sums(field_at(cf))
            u = self._link(c, mu)
            proj = ID4 - GAMMA[mu]
            wp += -0.5 * sf * np.einsum("ij,sja->sia", proj, vp @ u.T)
            wm += -0.5 * sf * np.einsum("ij,sja->sia", proj, vm @ u.T)
            cb, sb = self._shift(c, mu, -1)
            vp, vm = self._block_sums(field_at(cb))
            ub = np.conj(self._link(cb, mu).T)
            proj = ID4 + GAMMA[mu]
            wp += -0.5 * sb * np.einsum("ij,sja->sia", proj, vp @ ub.T)
            wm += -0.5 * sb * np.einsum("ij,sja->sia", proj, vm @ ub.T)
        b = sys.b.reshape(Ls, 1, 1)
        c_ = sys.c.reshape(Ls, 1, 1)
        return b * wp + c_ * wm

class PointwiseDbb(_SiteOps):
    def __init__(self, sys):
        super().__init__(sys)
        self.iinv = sys.local_inverse().reshape(sys.Ls, 4, sys.Ls, 4)

    def _iinv(self, f):
        return np.einsum("aibj,bjc->aic", self.iinv, f)

    def dbb_at(self, psi_half, site):
        """(D_bb psi)(site) [Ls][4][3] for a black site = (x, y, z, t)."""
        sys = self.sys
        black = sys.black_parity
        assert self._parity(site) == black

        def psi_at(c):
            if self._parity(c) != black:
                return np.zeros((sys.Ls, 4, 3), dtype=np.complex128)
            return psi_half[:, self._lex(c) // 2]

        cache = {}

        def u_at(c):
            if self._parity(c) == black:
                return np.zeros((sys.Ls, 4, 3), dtype=np.complex128)
            if c not in cache:
                cache[c] = self._iinv(self._hop_part(c, psi_at))
            return cache[c]

        return psi_at(site) - self._iinv(self._hop_part(site, u_at))


class PointwiseDalpha(_SiteOps):
    """D_alpha(m) of Sec. 2 (Eq. mobius1) and rhs = D_1(1) P b at single 4D sites."""

    def __init__(self, sys):
        super().__init__(sys)
        self.imat = sys.local_matrix().reshape(sys.Ls, 4, sys.Ls, 4)
        one = DWFSystem(sys.lattice, sys.Ls, sys.M5, 1.0, 1.0, sys.b, sys.c, sys.U,
                        bc_t=sys.bc_t, black_parity=sys.black_parity)
        self._d11 = _SiteOps(one)
        self._d11_imat = one.local_matrix().reshape(sys.Ls, 4, sys.Ls, 4)

    def apply_at(self, field_at, site):
        """(D_alpha psi)(site) [Ls][4][3]; field_at(c) -> psi at 4D site c, [Ls][4][3]."""
        return (np.einsum("aibj,bjc->aic", self.imat, field_at(site))
                + self._hop_part(site, field_at))

    def rhs_at(self, src4d, site):
        """(D_1(1) P b)(site) for b = (b_1, 0, ..., 0), b_1 = src4d [t][z][y][x][4][3]."""
        Ls = self.sys.Ls

        def pb_at(c):
            x, y, z, t = c
            b1 = src4d[t, z, y, x]
            v = np.zeros((Ls, 4, 3), dtype=np.complex128)
            v[0] = P_MINUS @ b1
            v[Ls - 1] = P_PLUS @ b1
            return v

        return (np.einsum("aibj,bjc->aic", self._d11_imat, pb_at(site))
                + self._d11._hop_part(site, pb_at))
