"""Pins of the oracle's fermion force for S = phi^+ (D_bb^+ D_bb)^-1 phi.

The adjoint-formula gradient is compared with central finite differences of
S itself (S from a dense solve, so the only error is the O(h^2) truncation
and rounding), on raw link entries (Re and Im) and along su(3) generators
exp(i h T_a) U (the projected force).
"""
import numpy as np

import oracle as O
from synthetic import gauge_field, gaussian_half5d

L2 = (2, 2, 2, 2)
LS = 4


def _system(U):
    b = np.array([1.5, 1.3, 1.8, 1.6])
    c = np.array([0.5, 0.2, 0.9, 0.4])
    return O.DWFSystem(L2, LS, -1.8, 0.1, 1.5, b, c, U)


def _action_dense(U, phi):
    sys = _system(U)
    n = phi.size
    D = O.overlap.dense_operator(sys.dbb, n, phi.shape)
    x = np.linalg.solve(np.conj(D.T) @ D, phi.reshape(n))
    return float(np.real(np.vdot(phi.reshape(n), x)))


def test_force_vs_finite_differences_raw_entries():
    U = gauge_field(L2, 0.5, seed=0)
    phi = gaussian_half5d(L2, LS, seed=2)
    sys = _system(U)
    x, _ = O.cg_normal(sys, phi, tol=1e-14)
    g = O.force_gradient(sys, phi, x)
    rng = np.random.default_rng(3)
    h = 1e-5
    for _ in range(4):
        t, z, y, xx = (int(v) for v in rng.integers(0, 2, size=4))
        mu = int(rng.integers(0, 4))
        i, j = int(rng.integers(0, 3)), int(rng.integers(0, 3))
        for part, unit in [("re", 1.0), ("im", 1j)]:
            up = U.copy()
            um = U.copy()
            up[t, z, y, xx, mu, i, j] += h * unit
            um[t, z, y, xx, mu, i, j] -= h * unit
            fd = (_action_dense(up, phi) - _action_dense(um, phi)) / (2 * h)
            want = g[t, z, y, xx, mu, i, j].real if part == "re" else g[t, z, y, xx, mu, i, j].imag
            assert abs(fd - want) <= 1e-6 * max(1.0, abs(want)), (part, fd, want)


def test_su3_force_vs_group_direction_fd():
    """dS/dh of S(exp(i h T_a) U) equals i tr(T_a F), F = TA(U G^+)."""
    U = gauge_field(L2, 0.5, seed=0)
    phi = gaussian_half5d(L2, LS, seed=2)
    sys = _system(U)
    g = O.force_gradient(sys, phi)
    f = O.su3_force(U, g)
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    T = lam / 2
    h = 1e-5
    rng = np.random.default_rng(5)
    for _ in range(2):
        t, z, y, xx = (int(v) for v in rng.integers(0, 2, size=4))
        mu = int(rng.integers(0, 4))
        for a in range(8):
            w, v = np.linalg.eigh(T[a])
            def rot(s):
                e = v @ np.diag(np.exp(1j * s * w)) @ np.conj(v.T)
                uu = U.copy()
                uu[t, z, y, xx, mu] = e @ U[t, z, y, xx, mu]
                return uu
            fd = (_action_dense(rot(h), phi) - _action_dense(rot(-h), phi)) / (2 * h)
            want = (1j * np.trace(T[a] @ f[t, z, y, xx, mu])).real
            assert abs(fd - want) <= 1e-6 * max(1.0, abs(want)), (a, fd, want)
    # F is traceless anti-Hermitian
    assert np.abs(f + np.conj(np.swapaxes(f, -1, -2))).max() < 1e-12
    assert np.abs(np.trace(f, axis1=-2, axis2=-1)).max() < 1e-12
