"""Oracle: the fermion force dS/dU for S = phi^+ (D_bb^+ D_bb)^-1 phi.

TEST INFRASTRUCTURE ONLY (see oracle/lattice.py).

D_bb is the red-black operator of Sec. 3, Eq. redblack; only its hopping
blocks D_br, D_rb depend on the links (I is site-local and link-free).  With
X = (D^+ D)^-1 phi and Y = D X, first-order perturbation theory gives

    dS = -2 Re[Y^+ dD_bb X]
       = 2 Re[eta1^+ dD_br xi1] + 2 Re[eta2^+ dD_rb xi2],
    eta1 = (I^-1)^+ Y,  xi1 = I^-1 D_rb X,
    eta2 = (I^-1)^+ D_br^+ (I^-1)^+ Y,  xi2 = X.  Every hopping term of
Eq. wilson that a link U_mu(x) enters (the forward hop x <- x+mu with
(1 - gamma_mu) U_mu(x), the backward hop x+mu <- x with (1 + gamma_mu)
U_mu(x)^+) contributes an outer product in colour, traced over spin and
summed over the 5th dimension; inside D_alpha the link multiplies the
b_i / c_i weighted block sums of Eq. mobius1.

Gradient convention: G_ij = dS/dRe U_ij + i dS/dIm U_ij, so that
dS = Re tr(G^+ dU) with U^+ perturbed together with U.  The su(3)
projection is F_mu(x) = TA(U_mu(x) G_mu(x)^+),
TA(M) = (M - M^+)/2 - tr(M - M^+)/6.
"""
from __future__ import annotations

import numpy as np

from .dwf import blocks
from .lattice import GAMMA, ID4, half_to_full, spin_mul
from .schur import DWFSystem
from .wilson import _shift


def _weighted_block_sum(sys: DWFSystem, xi):
    """w_i = b_i v_plus_i + c_i v_minus_i: what D_w multiplies in row i of Eq. mobius1."""
    vp = np.zeros_like(xi)
    vm = np.zeros_like(xi)
    for i, j, kind, M in blocks(sys.Ls, sys.alpha, sys.m):
        t = spin_mul(M, xi[j])
        if kind == "+":
            vp[i] += t
        else:
            vm[i] += t
    shp = (sys.Ls,) + (1,) * (xi.ndim - 1)
    return sys.b.reshape(shp) * vp + sys.c.reshape(shp) * vm


def _outer(a, b):
    """sum over s and spin of a[s,...,spin,i] conj(b[s,...,spin,j]) -> [...,i,j]."""
    return np.einsum("s...ai,s...aj->...ij", a, np.conj(b))


def hop_gradient(sys: DWFSystem, eta, xi):
    """G of F = Re[eta^+ d(D_alpha - I) xi] for full 5D fields eta, xi."""
    w = _weighted_block_sum(sys, xi)
    g = np.zeros(sys.U.shape, dtype=np.complex128)
    lead = 1
    for mu in range(4):
        w_fwd = _shift(w, lead, mu, +1, sys.bc_t)
        chi = spin_mul(ID4 - GAMMA[mu], w_fwd)
        g[..., mu, :, :] += -0.5 * _outer(eta, chi)
        eta_fwd = _shift(eta, lead, mu, +1, sys.bc_t)
        zeta = spin_mul(ID4 + GAMMA[mu], eta_fwd)
        g[..., mu, :, :] += -0.5 * _outer(w, zeta)
    return g


def cg_normal(sys: DWFSystem, phi, tol=1e-14, maxiter=100000):
    """X = (D_bb^+ D_bb)^-1 phi by plain CG (Hestenes-Stiefel) on D^+ D."""
    def a_op(v):
        return sys.dbb_dag(sys.dbb(v))
    x = np.zeros_like(phi)
    r = phi.copy()
    p = r.copy()
    rr = np.real(np.vdot(r.ravel(), r.ravel()))
    bb = rr
    it = 0
    while it < maxiter and rr > tol * tol * bb:
        ap = a_op(p)
        a = rr / np.real(np.vdot(p.ravel(), ap.ravel()))
        x = x + a * p
        r = r - a * ap
        rr_new = np.real(np.vdot(r.ravel(), r.ravel()))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def action(sys: DWFSystem, phi, x=None):
    """S = phi^+ (D^+ D)^-1 phi."""
    if x is None:
        x, _ = cg_normal(sys, phi)
    return float(np.real(np.vdot(phi.ravel(), x.ravel())))


def force_gradient(sys: DWFSystem, phi, x=None):
    """Raw link gradient G[t][z][y][x][mu][3][3] of S (convention in the module doc)."""
    if x is None:
        x, _ = cg_normal(sys, phi)
    y = sys.dbb(x)
    eta1 = sys.iinv_dag(y)
    xi1 = sys.iinv(sys.d_rb(x))
    eta2 = sys.iinv_dag(sys.d_br_dag(eta1))
    xi2 = x
    L, pb, pr = sys.lattice, sys.black_parity, sys.red_parity
    g = hop_gradient(sys, half_to_full(eta1, L, pb), half_to_full(xi1, L, pr))
    g += hop_gradient(sys, half_to_full(eta2, L, pr), half_to_full(xi2, L, pb))
    return 2.0 * g


def traceless_antihermitian(m):
    """TA(M) = (M - M^+)/2 - tr(M - M^+)/6 * 1 on the last two axes."""
    a = 0.5 * (m - np.conj(np.swapaxes(m, -1, -2)))
    tr = np.trace(a, axis1=-2, axis2=-1)
    return a - (tr / 3.0)[..., None, None] * np.eye(3)


def su3_force(U, g):
    """F_mu(x) = TA(U_mu(x) G_mu(x)^+)."""
    return traceless_antihermitian(U @ np.conj(np.swapaxes(g, -1, -2)))
