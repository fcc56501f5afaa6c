"""Checks of the seeded input generators (shared by the CUDA tests and the oracle)."""
import json
import os

import numpy as np
import pytest

import synthetic as S
from synthetic.zolotarev import _err


def test_gauge_is_special_unitary_and_seeded():
    u = S.gauge_field((4, 2, 2, 4), 0.5, seed=0)
    eye = np.eye(3)
    assert np.abs(u @ np.conj(np.swapaxes(u, -1, -2)) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1).max() < 1e-14
    assert np.array_equal(u, S.gauge_field((4, 2, 2, 4), 0.5, seed=0))
    assert not np.array_equal(u, S.gauge_field((4, 2, 2, 4), 0.5, seed=1))


def test_plaquette_limits():
    assert abs(S.plaquette(S.unit_gauge((2, 2, 2, 2))) - 1.0) < 1e-15
    p3 = S.plaquette(S.gauge_field((4, 4, 4, 4), 0.3, seed=0))
    p5 = S.plaquette(S.gauge_field((4, 4, 4, 4), 0.5, seed=0))
    assert 1.0 > p3 > p5 > 0.3


def test_sources():
    s = S.gaussian_source4d((4, 2, 2, 2), seed=1, even_only=True)
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (2, 2, 2, 4)], indexing="ij")
    odd = (x + y + z + t) % 2 == 1
    assert np.all(s[odd] == 0) and np.all(s[~odd] != 0)
    p = S.point_source4d((4, 2, 2, 2), 3, 2, site=(1, 0, 1, 0))
    assert p.sum() == 1 and p[0, 1, 0, 1, 3, 2] == 1


@pytest.mark.parametrize("Ls", [4, 8, 12])
def test_zolotarev_equal_ripple(Ls):
    """Chebyshev alternation: Ls + 1 extrema of R - 1 of equal size, alternating sign."""
    a, delta = S.zolotarev_sign_coefficients(Ls, 0.05, 6.0)
    x = np.exp(np.linspace(np.log(0.05), np.log(6.0), 400001))
    e = _err(x, 1.0 / a)
    assert abs(np.abs(e).max() - delta) <= 1e-9 * delta
    # the zeros of R - 1 sit at 1/a_i and split [xmin, xmax] into Ls + 1 pieces
    edges = np.concatenate([[0.05], np.sort(1.0 / a), [6.0]])
    signs = []
    for k in range(Ls + 1):
        sel = (x >= edges[k]) & (x <= edges[k + 1])
        ek = e[sel]
        j = np.argmax(np.abs(ek))
        assert abs(abs(ek[j]) - delta) <= 1e-6 * delta
        signs.append(np.sign(ek[j]))
    assert all(signs[k] == -signs[k + 1] for k in range(Ls))
    # more slices -> smaller ripple (Zolotarev: exponential convergence)
    if Ls > 4:
        assert delta < S.zolotarev_sign_coefficients(Ls - 2, 0.05, 6.0)[1]


def test_concave_order_and_mobius_form():
    b, c, a, _ = S.zolotarev_mobius(10)
    assert np.allclose(b - c, 1.0) and np.allclose(b + c, a)
    assert a[0] == a.min() or a[-1] == a.min()
    k = int(np.argmax(a))
    assert 3 <= k <= 6
    assert np.all(np.diff(a[: k + 1]) > 0) and np.all(np.diff(a[k:]) < 0)


def test_table1_fixture_is_the_papers():
    with open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")) as f:
        t = json.load(f)
    assert len(t["rows"]) == 8
    assert all(0.35 <= r[4] <= 0.65 for r in t["rows"])
