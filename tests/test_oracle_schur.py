"""Pins of the oracle's red-black operator, CG solver and propagator.

* CGNR solves a random dense system to the tolerance (checked with LAPACK);
* the red-black Schur solve equals a brute-force dense LU solve of the full
  5D system D_alpha psi = rhs on a 2^4 lattice (Sec. 3, Eq. redblack);
* <u, D_bb v> = <D_bb^+ u, v> (the adjoint is the adjoint);
* z_1 is independent of alpha and z_s = y_s / alpha for s >= 2 (Sec. 2,
  Eq. tosolve1: A z = y);
* the 4D propagator equals D_OV(m)^-1 b_1 with eps in the tanh form of
  App. A (Eq. polar, Eq. argument) and App. B (Eq. tosolve), built densely.
"""
import numpy as np
import pytest

import oracle as O
from oracle.overlap import dense_dw, dense_gamma5, dense_operator, overlap_operator
from synthetic import gauge_field, gaussian_half5d, gaussian_source4d, zolotarev_mobius

L2 = (2, 2, 2, 2)


def _sys(b, c, alpha, m=0.05, L=L2, eps=0.5, M5=-1.8, bc_t=1.0, black=0):
    U = gauge_field(L, eps, seed=0)
    return O.DWFSystem(L, len(b), M5, m, alpha, np.asarray(b), np.asarray(c), U,
                       bc_t=bc_t, black_parity=black)


def test_cgnr_random_dense():
    rng = np.random.default_rng(0)
    n = 40
    a = np.eye(n) * 3 + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    rhs = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, res = O.cgnr(lambda v: a @ v, lambda v: np.conj(a.T) @ v, rhs, tol=1e-12)
    assert res <= 1e-12
    assert np.abs(x - np.linalg.solve(a, rhs)).max() < 1e-10


@pytest.mark.parametrize("black", [0, 1])
@pytest.mark.parametrize("bc_t", [1.0, -1.0])
def test_schur_equals_dense_solve(black, bc_t):
    b = np.array([1.2, 1.6, 0.9, 1.4])
    c = np.array([0.3, 0.5, -0.2, 0.6])
    sys = _sys(b, c, 1.3, bc_t=bc_t, black=black)
    src = gaussian_source4d(L2, seed=1)
    res = O.solve_propagator(sys, src, tol=1e-12)
    assert res["true_resid"] <= 1e-12
    n = 4 * 16 * 12
    D = dense_operator(lambda v: O.dalpha(v, sys.U, sys.M5, b, c, sys.alpha, sys.m, bc_t),
                       n, res["rhs"].shape)
    psi = np.linalg.solve(D, res["rhs"].reshape(n)).reshape(res["rhs"].shape)
    assert np.abs(psi - res["psi"]).max() / np.abs(psi).max() < 1e-10
    assert res["true_resid_5d"] < 1e-10


def test_dbb_adjoint_and_definition():
    b = np.array([1.5, 1.5, 1.5, 1.5, 1.5, 1.5])
    c = np.array([0.5, 0.5, 0.5, 0.5, 0.5, 0.5])
    sys = _sys(b, c, 0.75, L=(2, 2, 4, 2))
    u = gaussian_half5d(sys.lattice, 6, seed=3)
    v = gaussian_half5d(sys.lattice, 6, seed=4)
    lhs = O.vdot(u, sys.dbb(v))
    rhs = O.vdot(sys.dbb_dag(u), v)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    # Eq. redblack is the Schur complement of the full operator: D_alpha [psi_b, psi_r]
    # with psi_r = -I^-1 D_rb psi_b has black part I D_bb psi_b.
    hb = v
    hr = -sys.iinv(sys.d_rb(hb))
    full = O.half_to_full(hb, sys.lattice, 0) + O.half_to_full(hr, sys.lattice, 1)
    d = O.dalpha(full, sys.U, sys.M5, b, c, sys.alpha, sys.m)
    blk = O.full_to_half(d, sys.lattice, 0)
    Imat = sys.local_matrix()
    assert np.abs(blk - sys.apply_local_matrix(Imat, sys.dbb(hb))).max() < 1e-12
    assert np.abs(O.full_to_half(d, sys.lattice, 1)).max() < 1e-12


@pytest.mark.parametrize("coeff", ["shamir", "mobius"])
def test_z1_independent_of_alpha(coeff):
    Ls = 4
    if coeff == "shamir":
        b, c = np.ones(Ls), np.zeros(Ls)
    else:
        b, c = 1.5 * np.ones(Ls), 0.5 * np.ones(Ls)
    src = gaussian_source4d(L2, seed=1, even_only=True)
    ref = O.solve_propagator(_sys(b, c, 1.0), src, tol=1e-12)
    for alpha in [0.55, 1.5]:
        res = O.solve_propagator(_sys(b, c, alpha), src, tol=1e-12)
        assert np.abs(res["z1"] - ref["z1"]).max() / np.abs(ref["z1"]).max() < 1e-9
        # A z = y: z_s = y_s / alpha for s >= 2
        assert np.abs(res["z"][1:] - ref["z"][1:] / alpha).max() / np.abs(ref["z"]).max() < 1e-9


OVERLAP_SETS = {
    "shamir": (np.ones(4), np.zeros(4)),
    "mobius": (1.5 * np.ones(4), 0.5 * np.ones(4)),
    "borici": (np.ones(4), np.ones(4)),
    "varying_b_minus_c_1": (np.array([1.2, 2.0, 1.5, 1.1]), np.array([0.2, 1.0, 0.5, 0.1])),
}


@pytest.mark.parametrize("name", list(OVERLAP_SETS))
@pytest.mark.parametrize("alpha", [1.0, 0.6])
def test_propagator_equals_overlap_inverse(name, alpha):
    b, c = OVERLAP_SETS[name]
    m = 0.05
    sys = _sys(b, c, alpha, m=m)
    src = gaussian_source4d(L2, seed=1)
    res = O.solve_propagator(sys, src, tol=1e-13)
    dwm = dense_dw(sys.U, L2, sys.M5)
    dov = overlap_operator(dwm, dense_gamma5(L2), b, c, m)
    y1 = np.linalg.solve(dov, src.reshape(-1)).reshape(src.shape)
    assert np.abs(y1 - res["z1"]).max() / np.abs(y1).max() < 1e-11


def test_zolotarev_propagator_is_order_independent():
    """The X_i commute for b_i - c_i = 1, so z_1 does not depend on the slice order."""
    b, c, a, _ = zolotarev_mobius(4, 0.05, 6.0)
    src = gaussian_source4d(L2, seed=1)
    r1 = O.solve_propagator(_sys(b, c, 1.25, m=0.05), src, tol=1e-13)
    perm = np.array([2, 0, 3, 1])
    r2 = O.solve_propagator(_sys(b[perm], c[perm], 1.0, m=0.05), src, tol=1e-13)
    assert np.abs(r1["z1"] - r2["z1"]).max() / np.abs(r1["z1"]).max() < 1e-10


def test_row_scale_factors():
    """S of the row-scaled Eq. redblack1: 1/(b_s + c_s) where that exceeds one."""
    sys = _sys(np.array([1.5, 0.4, 1.0, 2.0]), np.array([0.5, 0.2, 0.0, -0.5]), 1.0)
    assert np.allclose(sys.row_scale(), [0.5, 1.0, 1.0, 1.0 / 1.5])


@pytest.mark.parametrize("form", [1, 2])
def test_redblack1_forms(form):
    """Eq. redblack1 equals I_bb times Eq. redblack (I_bb - D_br I^-1 D_rb =
    I_bb (1 - I^-1 D_br I^-1 D_rb)); the row-scaled form is S times it; each
    adjoint is the adjoint."""
    b, c, _, _ = zolotarev_mobius(6, 0.05, 6.0)
    sys = _sys(b, c, 0.8, L=(2, 2, 4, 2))
    op, op_dag, left = sys.schur_operator(form)
    u = gaussian_half5d(sys.lattice, 6, seed=3)
    v = gaussian_half5d(sys.lattice, 6, seed=4)
    want = sys.apply_local_matrix(sys.local_matrix(), sys.dbb(v))
    if form == 2:
        want = sys.row_scale().reshape(6, 1, 1, 1) * want
    assert np.abs(op(v) - want).max() / np.abs(want).max() < 1e-13
    lhs = np.vdot(u, op(v))
    rhs = np.vdot(op_dag(u), v)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


def test_forms_share_the_solution():
    """All three operators of Sec. 3 solve for the same psi (hence z_1), which the
    dense LU solve of the full 5D system pins for form 0."""
    b, c, _, _ = zolotarev_mobius(4, 0.05, 6.0)
    sys = _sys(b, c, 1.25, m=0.06)
    src = gaussian_source4d(L2, seed=1)
    ref = O.solve_propagator(sys, src, tol=1e-12)
    n = 4 * 16 * 12
    D = dense_operator(lambda v: O.dalpha(v, sys.U, sys.M5, b, c, sys.alpha, sys.m, sys.bc_t),
                       n, ref["rhs"].shape)
    psi = np.linalg.solve(D, ref["rhs"].reshape(n)).reshape(ref["rhs"].shape)
    for form in (1, 2):
        res = O.solve_propagator(sys, src, tol=1e-12, form=form)
        assert res["true_resid"] <= 1e-12
        assert np.abs(res["psi"] - psi).max() / np.abs(psi).max() < 1e-9


@pytest.mark.parametrize("name,alpha", [("mobius", 1.0), ("varying_b_minus_c_1", 1.4), ("shamir", 0.7)])
def test_overlap_apply_equals_dense_overlap(name, alpha):
    """D_OV(m) b_1 from the mass-exchanged 5D solve equals the dense tanh-form
    overlap operator of App. A applied to b_1 (2^4 lattice)."""
    b, c = OVERLAP_SETS[name]
    m = 0.05
    sys = _sys(b, c, alpha, m=m)
    src = gaussian_source4d(L2, seed=1)
    z1, it, res = O.overlap_apply(sys, src, tol=1e-13)
    dov = overlap_operator(dense_dw(sys.U, L2, sys.M5), dense_gamma5(L2), b, c, m)
    want = (dov @ src.reshape(-1)).reshape(src.shape)
    assert res <= 1e-13
    assert np.abs(z1 - want).max() / np.abs(want).max() < 1e-11
