"""Pins of the oracle's D_alpha(m), P and A (Sec. 2, Eq. mobius1, Eq. eqP).

* D_alpha at alpha = 1 equals the conventional Mobius operator, written
  independently with its mass boundary conditions (abstract, Sec. 2);
* D_alpha P = D_1 P A with A = diag(1, alpha, ..., alpha) (Sec. 2);
* the literal adjoint is the adjoint (<u, D v> = <D^+ u, v>);
* D_alpha = D_w B + C with B, C real, site-local and chirality-block-diagonal
  Ls x Ls matrices written from the block list by hand (the factorisation the
  CUDA kernels are designed on);
* P P^-1 = 1.
"""
import numpy as np
import pytest

import oracle as O
from oracle.lattice import spin_mul
from synthetic import gauge_field

L = (2, 2, 2, 4)


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


COEFFS = {
    "shamir": (np.ones(6), np.zeros(6)),
    "mobius": (1.5 * np.ones(6), 0.5 * np.ones(6)),
    "varying": (np.array([1.1, 1.7, 2.3, 0.9, 1.4, 1.2]), np.array([0.2, -0.3, 0.8, 0.1, 0.5, 1.3])),
}


@pytest.mark.parametrize("name", list(COEFFS))
def test_alpha1_is_standard_mobius(name):
    b, c = COEFFS[name]
    U = gauge_field(L, 0.5, seed=0)
    psi = _rand((6,) + O.shape4(L) + (4, 3), 1)
    d1 = O.dalpha(psi, U, -1.8, b, c, 1.0, 0.03)
    d2 = O.mobius_standard(psi, U, -1.8, b, c, 0.03)
    assert np.abs(d1 - d2).max() < 1e-13


@pytest.mark.parametrize("name", list(COEFFS))
@pytest.mark.parametrize("alpha", [0.5, 1.25, 2.0])
def test_dalpha_p_equals_d1_p_a(name, alpha):
    b, c = COEFFS[name]
    U = gauge_field(L, 0.5, seed=0)
    psi = _rand((6,) + O.shape4(L) + (4, 3), 2)
    lhs = O.dalpha(O.p_apply(psi), U, -1.8, b, c, alpha, 0.01)
    rhs = O.dalpha(O.p_apply(O.a_apply(psi, alpha)), U, -1.8, b, c, 1.0, 0.01)
    assert np.abs(lhs - rhs).max() < 1e-13


def test_p_inverse_and_ls2_blocks():
    psi = _rand((5,) + O.shape4(L) + (4, 3), 3)
    assert np.abs(O.p_apply(O.p_inverse(psi)) - psi).max() < 1e-15
    assert np.abs(O.p_inverse(O.p_apply(psi)) - psi).max() < 1e-15
    # Ls = 2: the (1,2) entry carries both alpha D_1- P_- and -m D_1- P_+
    U = gauge_field(L, 0.5, seed=0)
    b, c = np.array([1.3, 1.6]), np.array([0.4, 0.2])
    p2 = _rand((2,) + O.shape4(L) + (4, 3), 4)
    d1 = O.dalpha(p2, U, -1.8, b, c, 1.0, 0.2)
    d2 = O.mobius_standard(p2, U, -1.8, b, c, 0.2)
    assert np.abs(d1 - d2).max() < 1e-13


def test_dalpha_adjoint():
    b, c = COEFFS["varying"]
    U = gauge_field(L, 0.5, seed=0)
    u = _rand((6,) + O.shape4(L) + (4, 3), 5)
    v = _rand((6,) + O.shape4(L) + (4, 3), 6)
    lhs = O.vdot(u, O.dalpha(v, U, -1.8, b, c, 1.3, 0.07))
    rhs = O.vdot(O.dalpha_dag(u, U, -1.8, b, c, 1.3, 0.07), v)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _bc_matrices(b, c, alpha, m):
    """B_+-, C_+- written out row by row from Eq. mobius1 (real Ls x Ls)."""
    Ls = len(b)
    Bp, Bm = np.zeros((Ls, Ls)), np.zeros((Ls, Ls))
    Cp, Cm = np.zeros((Ls, Ls)), np.zeros((Ls, Ls))
    for X, Y, fb, fc in [(Bp, Bm, b, c), (Cp, Cm, np.ones(Ls), -np.ones(Ls))]:
        # plus chirality (P_+ component of the input)
        X[0, 0] += alpha * fb[0]
        X[0, Ls - 1] += -m * fc[0]
        for i in range(1, Ls - 1):
            X[i, i - 1] += alpha * fc[i]
            X[i, i] += alpha * fb[i]
        X[Ls - 1, Ls - 2] += alpha * fc[Ls - 1]
        X[Ls - 1, Ls - 1] += fb[Ls - 1]
        # minus chirality
        Y[0, 0] += fb[0]
        Y[0, 1] += alpha * fc[0]
        for i in range(1, Ls - 1):
            Y[i, i] += alpha * fb[i]
            Y[i, i + 1] += alpha * fc[i]
        Y[Ls - 1, 0] += -m * fc[Ls - 1]
        Y[Ls - 1, Ls - 1] += alpha * fb[Ls - 1]
    return Bp, Bm, Cp, Cm


@pytest.mark.parametrize("name", list(COEFFS))
def test_factorisation_dw_b_plus_c(name):
    b, c = COEFFS[name]
    alpha, m, M5 = 1.35, 0.04, -1.8
    U = gauge_field(L, 0.5, seed=0)
    psi = _rand((6,) + O.shape4(L) + (4, 3), 7)
    Bp, Bm, Cp, Cm = _bc_matrices(b, c, alpha, m)

    def chiral_apply(Mp, Mm, v):
        out = np.empty_like(v)
        out[..., :2, :] = np.einsum("st,t...->s...", Mp, v[..., :2, :])
        out[..., 2:, :] = np.einsum("st,t...->s...", Mm, v[..., 2:, :])
        return out

    bpsi = chiral_apply(Bp, Bm, psi)
    want = O.dw(bpsi, U, M5) + chiral_apply(Cp, Cm, psi)
    got = O.dalpha(psi, U, M5, b, c, alpha, m)
    assert np.abs(got - want).max() < 1e-13
    # I = (4 + M5) B + C is the site-local part
    sys = O.DWFSystem(L, 6, M5, m, alpha, b, c, U)
    Imat = sys.local_matrix().reshape(6, 4, 6, 4)
    Ip = (4 + M5) * Bp + Cp
    Im = (4 + M5) * Bm + Cm
    for sp in range(4):
        want_blk = Ip if sp < 2 else Im
        assert np.abs(Imat[:, sp, :, sp] - want_blk).max() < 1e-14
    # chirality is not mixed by I
    assert np.abs(Imat[:, :2, :, 2:]).max() == 0.0
    assert np.abs(Imat[:, 2:, :, :2]).max() == 0.0


def test_gamma5_commutes_with_local_part():
    b, c = COEFFS["varying"]
    U = gauge_field(L, 0.5, seed=0)
    sys = O.DWFSystem(L, 6, -1.8, 0.02, 0.8, b, c, U)
    I = sys.local_matrix()
    g5 = np.kron(np.eye(6), O.GAMMA5)
    assert np.abs(I @ g5 - g5 @ I).max() == 0.0
    assert np.abs(I @ sys.local_inverse() - np.eye(24)).max() < 1e-12
    assert np.abs(np.imag(I)).max() == 0.0
