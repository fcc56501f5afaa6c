"""Pins of the oracle's gamma matrices and Wilson matrix (Sec. 2, Eq. wilson).

None of these compare the oracle with itself: the Clifford algebra, the
free-field momentum-space closed form and gamma5-hermiticity are fixed by
the mathematics, independently of how D_w is coded.
"""
import numpy as np
import pytest

import oracle as O
from oracle.lattice import ID4, spin_mul
from synthetic import gauge_field, unit_gauge


def test_clifford_and_chiral_basis():
    g = O.GAMMA
    for mu in range(4):
        assert np.allclose(g[mu], np.conj(g[mu].T))
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * ID4)
        assert np.allclose(O.GAMMA5 @ g[mu] + g[mu] @ O.GAMMA5, 0)
    assert np.allclose(O.GAMMA5, np.diag([1, 1, -1, -1]))
    assert np.allclose(O.P_PLUS + O.P_MINUS, ID4)
    assert np.allclose(O.P_PLUS @ O.P_PLUS, O.P_PLUS)
    assert np.allclose(O.P_PLUS @ O.P_MINUS, 0)


@pytest.mark.parametrize("bc_t", [1.0, -1.0])
def test_free_field_closed_form(bc_t):
    """U = 1: D_w e^{ipx} u = [M5 + sum(1 - cos p) + i sum gamma_mu sin p_mu] e^{ipx} u."""
    L = (4, 4, 2, 6)
    Lx, Ly, Lz, Lt = L
    U = unit_gauge(L)
    M5 = -1.8
    rng = np.random.default_rng(11)
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                             indexing="ij")
    for n in [(0, 0, 0, 0), (1, 0, 1, 2), (3, 1, 0, 5), (2, 3, 1, 1)]:
        tshift = 0.5 if bc_t < 0 else 0.0
        p = np.array([2 * np.pi * n[0] / Lx, 2 * np.pi * n[1] / Ly,
                      2 * np.pi * n[2] / Lz, 2 * np.pi * (n[3] + tshift) / Lt])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = phase[..., None, None] * u
        k = (M5 + np.sum(1 - np.cos(p))) * ID4 + 1j * sum(O.GAMMA[m] * np.sin(p[m]) for m in range(4))
        want = phase[..., None, None] * (k @ u)
        got = O.dw(psi, U, M5, bc_t=bc_t)
        assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("bc_t", [1.0, -1.0])
def test_gamma5_hermiticity_and_adjoint(bc_t):
    """<u, D_w v> = <gamma5 D_w gamma5 u, v> and D_w^+ = gamma5 D_w gamma5."""
    L = (4, 2, 2, 4)
    U = gauge_field(L, 0.5, seed=3)
    rng = np.random.default_rng(4)
    shp = (3,) + O.shape4(L) + (4, 3)
    u = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    v = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    g5 = lambda w: spin_mul(O.GAMMA5, w)
    lhs = O.vdot(u, O.dw(v, U, -1.8, bc_t=bc_t))
    rhs = O.vdot(g5(O.dw(g5(u), U, -1.8, bc_t=bc_t)), v)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    d1 = O.dw(u, U, -1.8, dagger_op=True, bc_t=bc_t)
    d2 = g5(O.dw(g5(u), U, -1.8, bc_t=bc_t))
    assert np.abs(d1 - d2).max() < 1e-13


def test_dw_single_link_matrix_element():
    """One link, two sites: the (x, x+mu) block is -1/2 (1 - gamma_mu) U_mu(x) (Eq. wilson)."""
    L = (4, 4, 4, 4)
    U = gauge_field(L, 0.7, seed=9)
    shp = O.shape4(L) + (4, 3)
    for mu, dx in [(0, (1, 0, 0, 0)), (2, (0, 0, 1, 0)), (3, (0, 0, 0, 1))]:
        x0 = (1, 2, 0, 3)  # (x, y, z, t)
        xn = tuple((x0[k] + dx[k]) % L[k] for k in range(4))
        v = np.zeros(shp, dtype=np.complex128)
        v[xn[3], xn[2], xn[1], xn[0], 2, 1] = 1.0
        out = O.dw(v, U, 0.3)
        blk = out[x0[3], x0[2], x0[1], x0[0]]
        e = np.zeros((4, 3), dtype=np.complex128)
        e[2, 1] = 1.0
        want = -0.5 * (ID4 - O.GAMMA[mu]) @ (e @ U[x0[3], x0[2], x0[1], x0[0], mu].T)
        assert np.abs(blk - want).max() < 1e-15
