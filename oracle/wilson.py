"""Oracle: the Wilson Dirac matrix D_w(M5) of Sec. 2, Eq. wilson.

TEST INFRASTRUCTURE ONLY (see oracle/lattice.py).

    (D_w psi)(x) = (4 + M5) psi(x)
                   - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                                + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu) ]

Boundary conditions are periodic; bc_t = -1 multiplies every hop that
crosses the t boundary by -1 (antiperiodic fermions), an option the paper
does not discuss.

D_w^dagger is written out as the conjugate transpose of the stencil, term by
term: the forward hop of the adjoint carries (1 + gamma_mu) U_mu(x) and the
backward hop (1 - gamma_mu) U_mu(x - mu)^dagger.
"""
from __future__ import annotations

import numpy as np

from .lattice import GAMMA, ID4, colour_mul, dagger, spin_mul


def _shift(psi, lead, mu, direction, bc_t):
    """psi(x + direction * mu) with the boundary sign of the t direction."""
    ax = lead + (3 - mu)
    out = np.roll(psi, -direction, axis=ax)
    if mu == 3 and bc_t != 1.0:
        out = out.copy()
        idx = [slice(None)] * out.ndim
        idx[ax] = -1 if direction > 0 else 0
        out[tuple(idx)] *= bc_t
    return out


def hop(psi, U, dagger_op=False, bc_t=1.0):
    """H psi = sum_mu [(1 -+ gamma_mu) U_mu(x) psi(x+mu) + (1 +- gamma_mu) U_mu(x-mu)^+ psi(x-mu)].

    psi has shape [..., t, z, y, x, 4, 3].  With dagger_op=True the signs of
    gamma_mu flip (the adjoint stencil).  D_w = (4 + M5) - H / 2.
    """
    lead = psi.ndim - 6
    sg = -1.0 if dagger_op else 1.0
    out = np.zeros_like(psi)
    for mu in range(4):
        umu = U[..., mu, :, :]
        fwd = _shift(psi, lead, mu, +1, bc_t)
        out += spin_mul(ID4 - sg * GAMMA[mu], colour_mul(umu, fwd))
        u_back = np.roll(umu, 1, axis=3 - mu)          # U_mu(x - mu)
        bwd = _shift(psi, lead, mu, -1, bc_t)
        out += spin_mul(ID4 + sg * GAMMA[mu], colour_mul(dagger(u_back), bwd))
    return out


def dw(psi, U, M5, dagger_op=False, bc_t=1.0):
    """D_w(M5) psi (or D_w^dagger psi), Eq. wilson."""
    return (4.0 + M5) * psi - 0.5 * hop(psi, U, dagger_op, bc_t)
