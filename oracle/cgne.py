"""Oracle: CG on the normal equations and the 4D propagator (Sec. 2-3, App. B).

TEST INFRASTRUCTURE ONLY (see oracle/lattice.py).

Sec. 3 solves Eq. tosolve1 with "the conjugate gradient method on the normal
equation" applied to the red-black operator D_bb.  The oracle runs CG on
D_bb^dagger D_bb x = D_bb^dagger r' (CGNR in Saad's naming, Iterative Methods
for Sparse Linear Systems, Alg. 8.4), from x = 0, tracking the system
residual r = r' - D_bb x:

    w = D p;  a = |z|^2 / |w|^2;  x += a p;  r -= a w;
    z = D^dagger r;  beta = |z_new|^2 / |z|^2;  p = z + beta p.

It stops once the true residual |r' - D_bb x| / |r'| (recomputed whenever the
recursive one reaches the tolerance, and every 10 iterations) is <= tol.

The 4D propagator (Sec. 2, Eq. tosolve1 and App. B, Eq. tosolve):
    D_alpha(m) P z = D_1(1) P b ,   b = (b_1, 0, ..., 0),   z_1 = y_1 .
With psi = P z the solve is D_alpha(m) psi = rhs, rhs = D_1(1) P b (D_alpha
at alpha = 1 and m = 1 with the same b_i, c_i), and
z_1 = (P^-1 psi)_1 = P_- psi_1 + P_+ psi_Ls.
"""
from __future__ import annotations

import numpy as np

from .dwf import dalpha, p_apply, p_inverse
from .lattice import full_to_half, norm2, shape4
from .schur import DWFSystem


def cgnr(apply_d, apply_ddag, rhs, tol=1e-10, maxiter=100000, check_every=10):
    """CG on D^+ D x = D^+ rhs; returns (x, iterations, true relative residual)."""
    bnorm = np.sqrt(norm2(rhs))
    x = np.zeros_like(rhs)
    if bnorm == 0.0:
        return x, 0, 0.0
    r = rhs.copy()
    z = apply_ddag(r)
    p = z.copy()
    zz = norm2(z)
    it = 0
    true_res = 1.0
    while it < maxiter:
        w = apply_d(p)
        ww = norm2(w)
        if ww == 0.0:
            break
        a = zz / ww
        x = x + a * p
        r = r - a * w
        it += 1
        rel = np.sqrt(norm2(r)) / bnorm
        if rel <= tol or it % check_every == 0:
            r_true = rhs - apply_d(x)
            true_res = np.sqrt(norm2(r_true)) / bnorm
            if true_res <= tol:
                break
            r = r_true
        z = apply_ddag(r)
        zz_new = norm2(z)
        p = z + (zz_new / zz) * p
        zz = zz_new
    return x, it, true_res


def source_5d(src4d, Ls):
    """b = (b_1, 0, ..., 0) as a full 5D field."""
    b5 = np.zeros((Ls,) + src4d.shape, dtype=np.complex128)
    b5[0] = src4d
    return b5


def propagator_rhs(sys: DWFSystem, src4d):
    """rhs = D_1(1) P b (Eq. tosolve; alpha = 1, m = 1, same b_i and c_i)."""
    b5 = source_5d(src4d, sys.Ls)
    return dalpha(p_apply(b5), sys.U, sys.M5, sys.b, sys.c, 1.0, 1.0, sys.bc_t)


def solve_propagator(sys: DWFSystem, src4d, tol=1e-10, maxiter=100000, form=0):
    """Red-black CGNR solve of D_alpha(m) P z = D_1(1) P b.

    form selects the red-black operator of Sec. 3 (0: Eq. redblack, 1: Eq.
    redblack1, 2: Eq. redblack1 with scaled rows); tol applies to that
    operator's own residual.

    Returns dict with z1 (4D propagator), psi (full 5D solution of
    D_alpha psi = rhs), z (= P^-1 psi), iterations, the Schur-system true
    residual and the full 5D residual |rhs - D_alpha psi| / |rhs|.
    """
    rhs = propagator_rhs(sys, src4d)
    rb = sys.schur_rhs(rhs)
    op, op_dag, left = sys.schur_operator(form)
    xb, it, res = cgnr(op, op_dag, left(rb), tol=tol, maxiter=maxiter)
    psi = sys.reconstruct(xb, rhs)
    r5 = rhs - dalpha(psi, sys.U, sys.M5, sys.b, sys.c, sys.alpha, sys.m, sys.bc_t)
    res5 = np.sqrt(norm2(r5) / norm2(rhs))
    z = p_inverse(psi)
    return {
        "z1": z[0],
        "z": z,
        "psi": psi,
        "psi_b": xb,
        "schur_rhs": rb,
        "rhs": rhs,
        "iterations": it,
        "true_resid": res,
        "true_resid_5d": res5,
    }


def overlap_apply(sys: DWFSystem, src4d, tol=1e-12, maxiter=100000):
    """D_OV(m) b_1 from the 5D system (App. A / App. B with the masses exchanged).

    Eq. tosolve gives z_1 = D_OV(m)^-1 D_OV(1) b_1 for D_alpha(m) P z = D_1(1) P b,
    and D_OV(1) = 1.  Solving instead D_alpha(1) P z = D_1(m) P b gives
    z_1 = D_OV(1)^-1 D_OV(m) b_1 = D_OV(m) b_1: the 4D overlap operator applied
    through one red-black solve at mass 1 (the Pauli-Villars system).
    Returns (z_1, iterations, Schur true residual)."""
    sys1 = DWFSystem(sys.lattice, sys.Ls, sys.M5, 1.0, sys.alpha, sys.b, sys.c, sys.U,
                     bc_t=sys.bc_t, black_parity=sys.black_parity)
    b5 = source_5d(src4d, sys.Ls)
    rhs = dalpha(p_apply(b5), sys.U, sys.M5, sys.b, sys.c, 1.0, sys.m, sys.bc_t)
    xb, it, res = cgnr(sys1.dbb, sys1.dbb_dag, sys1.schur_rhs(rhs), tol=tol, maxiter=maxiter)
    psi = sys1.reconstruct(xb, rhs)
    return p_inverse(psi)[0], it, res


def propagator_from_psi(psi):
    """z_1 = P_- psi_1 + P_+ psi_Ls from a full 5D solution psi = P z."""
    return p_inverse(psi)[0]


def half_fields_of(sys: DWFSystem, full):
    return (full_to_half(full, sys.lattice, sys.black_parity),
            full_to_half(full, sys.lattice, sys.red_parity))


def lattice_sites(lattice):
    Lt, Lz, Ly, Lx = shape4(lattice)
    return Lt * Lz * Ly * Lx
