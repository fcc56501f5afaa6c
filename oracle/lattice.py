"""Oracle: gamma matrices, lattice geometry and the canonical half-field layout.

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow FP64 CPU statement of
the paper's method; only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import it.  It shares no code with the CUDA path.

Conventions (the paper leaves them open, Sec. 2 eq. coeff and eq. wilson):

* chiral Dirac basis, gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = 1, 2, 3),
  gamma_4 = [[0, 1], [1, 0]], gamma5 = gamma_1 gamma_2 gamma_3 gamma_4
  = diag(1, 1, -1, -1), so P_+ keeps spins 0, 1 and P_- spins 2, 3;
* mu = 0, 1, 2, 3 <-> x, y, z, t; 4D arrays are indexed [t][z][y][x];
* site parity (x + y + z + t) mod 2; the half-field index of a site is its
  lexicographic index (x fastest) divided by 2 (exact because Lx is even).
"""
from __future__ import annotations

import numpy as np

SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]


def _gammas():
    z2 = np.zeros((2, 2), dtype=np.complex128)
    i2 = np.eye(2, dtype=np.complex128)
    g = []
    for k in range(3):
        g.append(np.block([[z2, -1j * SIGMA[k]], [1j * SIGMA[k], z2]]))
    g.append(np.block([[z2, i2], [i2, z2]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


GAMMA, GAMMA5 = _gammas()
ID4 = np.eye(4, dtype=np.complex128)
P_PLUS = 0.5 * (ID4 + GAMMA5)    # Sec. 2, P_+ = (1 + gamma5)/2
P_MINUS = 0.5 * (ID4 - GAMMA5)   # Sec. 2, P_- = (1 - gamma5)/2


def shape4(lattice):
    """(Lt, Lz, Ly, Lx) from lattice = (Lx, Ly, Lz, Lt)."""
    Lx, Ly, Lz, Lt = (int(v) for v in lattice)
    return Lt, Lz, Ly, Lx


def volume(lattice):
    Lt, Lz, Ly, Lx = shape4(lattice)
    return Lt * Lz * Ly * Lx


def parity_grid(lattice):
    """Array [t][z][y][x] of (x + y + z + t) mod 2."""
    Lt, Lz, Ly, Lx = shape4(lattice)
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly),
                             np.arange(Lx), indexing="ij")
    return (x + y + z + t) % 2


def spin_mul(g, psi):
    """Apply a 4x4 spin matrix g to psi[..., spin, colour]."""
    return np.matmul(g, psi)


def colour_mul(u, psi):
    """sum_b u[..., a, b] psi[..., spin, b] for u[t,z,y,x,3,3], psi[..., t,z,y,x,4,3]."""
    return np.matmul(psi, np.swapaxes(u, -1, -2))


def dagger(u):
    return np.conj(np.swapaxes(u, -1, -2))


def full_to_half(f, lattice, parity):
    """[Ls][t][z][y][x][4][3] -> canonical half-field [Ls][V/2][4][3] of one parity."""
    Ls = f.shape[0]
    V = volume(lattice)
    flat = f.reshape(Ls, V, 4, 3)
    mask = parity_grid(lattice).reshape(V) == parity
    return np.ascontiguousarray(flat[:, mask])


def half_to_full(h, lattice, parity):
    """Canonical half-field of one parity -> full field, zero on the other parity."""
    Ls = h.shape[0]
    Lt, Lz, Ly, Lx = shape4(lattice)
    V = Lt * Lz * Ly * Lx
    mask = parity_grid(lattice).reshape(V) == parity
    flat = np.zeros((Ls, V, 4, 3), dtype=np.complex128)
    flat[:, mask] = h
    return flat.reshape(Ls, Lt, Lz, Ly, Lx, 4, 3)


def vdot(a, b):
    """<a, b> = sum conj(a) b."""
    return np.vdot(a.ravel(), b.ravel())


def norm2(a):
    return float(np.real(np.vdot(a.ravel(), a.ravel())))
