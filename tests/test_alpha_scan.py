"""The alpha-scan driver (Sec. 3, Table 1 rows): host-side row handling, and one
small GPU scan whose ratios are n(alpha)/n(1) of converged solves."""
import numpy as np
import pytest

from paper_1501_04950_gb300 import alpha_scan


def test_table1_rows_and_coefficients():
    assert len(alpha_scan.TABLE1_ROWS) == 8
    m, Ls, b, c = alpha_scan.row_coefficients(alpha_scan.TABLE1_ROWS[6])
    assert (m, Ls) == (0.06, 8) and np.all(b == 1.7) and np.all(c == 0.7)
    m, Ls, b, c = alpha_scan.row_coefficients(alpha_scan.TABLE1_ROWS[7])
    assert Ls == 10 and np.allclose(b - c, 1.0) and np.all(b + c > 0)


@pytest.mark.gpu
def test_small_scan():
    res = alpha_scan.scan(alpha_scan.TABLE1_ROWS[2], lattice=(4, 4, 4, 4), alphas=[0.55, 1.0],
                          fields=1, sources=3, eps=0.3)
    k = res["alphas"].index(1.0)
    assert res["ratio_mean"][k] == 1.0 and res["ratio_std"][k] == 0.0
    assert all(r > 0 for r in res["ratio_mean"])
    assert res["iterations_alpha1_mean"] > 0


def test_zolotarev_orderings():
    """Every ordering is a permutation of the same a_i; concave puts the smallest
    at both ends and the largest in the centre (Sec. 3); b - c = 1, b + c = a."""
    from synthetic import zolotarev_mobius
    m, Ls, b, c = alpha_scan.row_coefficients(alpha_scan.TABLE1_ROWS[7], "concave")
    bz, cz, _, _ = zolotarev_mobius(Ls, 0.05, 6.0)
    assert np.allclose(b, bz) and np.allclose(c, cz)
    a = b + c
    assert np.argmax(a) in (Ls // 2 - 1, Ls // 2) and min(a[0], a[-1]) == a.min()
    for order in alpha_scan.ORDERS:
        _, _, bo, co = alpha_scan.row_coefficients(alpha_scan.TABLE1_ROWS[7], order)
        assert np.allclose(np.sort(bo + co), np.sort(a)) and np.allclose(bo - co, 1.0)
    _, _, bo, co = alpha_scan.row_coefficients(alpha_scan.TABLE1_ROWS[7], "ascending")
    assert np.all(np.diff(bo + co) > 0)
