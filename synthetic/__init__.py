"""Seeded synthetic inputs for the alpha-Mobius domain-wall solver.

This module is the one piece shared by the CUDA path's tests/bench and the
CPU oracle.  It holds no arithmetic of the method itself (no Wilson matrix,
no domain-wall operator, no solver): only random gauge fields, sources and
the 5th-dimension coefficients b_i, c_i that both sides take as inputs.

Canonical layouts (all complex128, C order):

* gauge field   U[t][z][y][x][mu][3][3], mu = 0..3 <-> x, y, z, t
* 4D spinor     psi[t][z][y][x][spin 4][colour 3]
* 5D half-field psi[s][h][spin 4][colour 3], h = (lexicographic site index) // 2
  over the sites of one checkerboard parity (x fastest).

The gauge recipe follows the workload description of the paper's Sec. 3
(SU(3) fields of lattice-QCD shape): U = exp(i eps H) with H a random
traceless Hermitian 3x3 matrix, built per link from Gaussian entries.
"""
from __future__ import annotations

import numpy as np

from .zolotarev import zolotarev_sign_coefficients, concave_order, zolotarev_mobius

__all__ = [
    "gauge_field",
    "unit_gauge",
    "gaussian_source4d",
    "point_source4d",
    "gaussian_half5d",
    "plaquette",
    "zolotarev_sign_coefficients",
    "concave_order",
    "zolotarev_mobius",
]


def _shape4(lattice):
    Lx, Ly, Lz, Lt = (int(v) for v in lattice)
    return Lt, Lz, Ly, Lx


def gauge_field(lattice, eps: float, seed: int = 0) -> np.ndarray:
    """Random SU(3) links U_mu(x) = V diag(exp(i eps lambda_k)) V^dagger.

    For every link (draw order [t][z][y][x][mu]) a complex Gaussian matrix
    A = (N(0,1) + i N(0,1)) / sqrt(2) is drawn (all real parts of the field
    first, then all imaginary parts), H = (A + A^dagger)/2 with its trace
    removed, and U = exp(i eps H) is formed from the eigendecomposition of H.
    U is unitary to rounding and has det U = exp(i eps tr H) = 1.
    """
    shp = _shape4(lattice) + (4, 3, 3)
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shp)
    im = rng.standard_normal(shp)
    a = (re + 1j * im) / np.sqrt(2.0)
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1)
    h = h - (tr / 3.0)[..., None, None] * np.eye(3)
    lam, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * lam)
    u = np.einsum("...ik,...k,...jk->...ij", v, ph, np.conj(v))
    return np.ascontiguousarray(u)


def unit_gauge(lattice) -> np.ndarray:
    """The free field U_mu(x) = 1."""
    shp = _shape4(lattice) + (4, 3, 3)
    u = np.zeros(shp, dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def gaussian_source4d(lattice, seed: int = 1, even_only: bool = False) -> np.ndarray:
    """Unit-variance complex Gaussian 4D source [t][z][y][x][4][3].

    With even_only=True the odd sites ((x+y+z+t) odd) are set to zero (a
    source on the even 4D sites only).
    """
    shp = _shape4(lattice) + (4, 3)
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shp)
    im = rng.standard_normal(shp)
    src = (re + 1j * im) / np.sqrt(2.0)
    if even_only:
        Lt, Lz, Ly, Lx = _shape4(lattice)
        t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly),
                                 np.arange(Lx), indexing="ij")
        odd = ((x + y + z + t) % 2) == 1
        src[odd] = 0.0
    return np.ascontiguousarray(src)


def point_source4d(lattice, spin: int, colour: int, site=(0, 0, 0, 0)) -> np.ndarray:
    """Point source delta_{x,site} delta_{spin} delta_{colour}; site = (x, y, z, t)."""
    shp = _shape4(lattice) + (4, 3)
    src = np.zeros(shp, dtype=np.complex128)
    x, y, z, t = site
    src[t, z, y, x, spin, colour] = 1.0
    return src


def gaussian_half5d(lattice, Ls: int, seed: int = 2) -> np.ndarray:
    """Unit-variance complex Gaussian 5D half-field [Ls][V/2][4][3]."""
    Lt, Lz, Ly, Lx = _shape4(lattice)
    vh = Lt * Lz * Ly * Lx // 2
    rng = np.random.default_rng(seed)
    shp = (Ls, vh, 4, 3)
    re = rng.standard_normal(shp)
    im = rng.standard_normal(shp)
    return np.ascontiguousarray((re + 1j * im) / np.sqrt(2.0))


def plaquette(u: np.ndarray) -> float:
    """Average plaquette (1/3) Re tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+.

    A diagnostic of the synthetic field's roughness (1 for the free field).
    """
    axis = {0: 3, 1: 2, 2: 1, 3: 0}
    tot = 0.0
    n = 0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            umu = u[..., mu, :, :]
            unu = u[..., nu, :, :]
            unu_xmu = np.roll(unu, -1, axis=axis[mu])
            umu_xnu = np.roll(umu, -1, axis=axis[nu])
            p = umu @ unu_xmu @ np.conj(np.swapaxes(umu_xnu, -1, -2)) @ np.conj(np.swapaxes(unu, -1, -2))
            tot += np.real(np.trace(p, axis1=-2, axis2=-1)).mean() / 3.0
            n += 1
    return tot / n
