"""The single-site D_bb evaluation agrees with the whole-lattice oracle."""
import itertools

import numpy as np
import pytest

import oracle as O
from oracle.pointwise import PointwiseDbb
from synthetic import gauge_field, gaussian_half5d


@pytest.mark.parametrize("bc_t,black", [(1.0, 0), (-1.0, 1)])
def test_pointwise_matches_whole_lattice(bc_t, black):
    L = (4, 2, 2, 4)
    Ls = 6
    rng = np.random.default_rng(1)
    b = 1.0 + rng.uniform(0, 1, Ls)
    c = rng.uniform(-0.5, 0.5, Ls)
    sysm = O.DWFSystem(L, Ls, -1.8, 0.03, 1.3, b, c, gauge_field(L, 0.5, seed=0),
                       bc_t=bc_t, black_parity=black)
    psi = gaussian_half5d(L, Ls, seed=4)
    full = sysm.dbb(psi)
    pw = PointwiseDbb(sysm)
    n = 0
    for x, y, z, t in itertools.product(range(4), range(2), range(2), range(4)):
        if (x + y + z + t) % 2 != black:
            continue
        lex = x + 4 * (y + 2 * (z + 2 * t))
        got = pw.dbb_at(psi, (x, y, z, t))
        assert np.abs(got - full[:, lex // 2]).max() < 1e-13
        n += 1
    assert n == 32


@pytest.mark.parametrize("bc_t,alpha,m", [(1.0, 1.3, 0.03), (-1.0, 0.7, 0.2)])
def test_pointwise_dalpha_and_rhs_match_whole_lattice(bc_t, alpha, m):
    """D_alpha psi (Eq. mobius1) and rhs = D_1(1) P b (Eq. tosolve) at every site
    against the whole-lattice oracle on a 4x2x2x4, Ls = 5 lattice."""
    from oracle.pointwise import PointwiseDalpha
    from synthetic import gaussian_source4d
    L = (4, 2, 2, 4)
    Ls = 5
    rng = np.random.default_rng(7)
    b = 1.0 + rng.uniform(0, 1, Ls)
    c = rng.uniform(-0.5, 0.5, Ls)
    U = gauge_field(L, 0.5, seed=0)
    sysm = O.DWFSystem(L, Ls, -1.8, m, alpha, b, c, U, bc_t=bc_t)
    psi = (rng.standard_normal((Ls, 4, 2, 2, 4, 4, 3))
           + 1j * rng.standard_normal((Ls, 4, 2, 2, 4, 4, 3)))
    full = O.dalpha(psi, U, -1.8, b, c, alpha, m, bc_t)
    src = gaussian_source4d(L, seed=3)
    rhs = O.propagator_rhs(sysm, src)
    pw = PointwiseDalpha(sysm)
    for x, y, z, t in itertools.product(range(4), range(2), range(2), range(4)):
        got = pw.apply_at(lambda cc: psi[:, cc[3], cc[2], cc[1], cc[0]], (x, y, z, t))
        assert np.abs(got - full[:, t, z, y, x]).max() < 1e-13
        got = pw.rhs_at(src, (x, y, z, t))
        assert np.abs(got - rhs[:, t, z, y, x]).max() < 1e-13
