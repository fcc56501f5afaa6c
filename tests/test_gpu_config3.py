"""Zolotarev alpha-Mobius solves with 16-bit inner fields (Sec. 3, the Zolotarev
coefficients in concave order; FP16 and BF16 storage with a per-5D-site FP32
scale, FP32 arithmetic, FP64 defect correction).

* 4^4, Ls = 12: the propagator z_1 against the oracle's own 1e-12 solve.
* 24^3 x 48, Ls = 12 (m = 0.005, alpha = 1.25, eps = 0.5, Gaussian b_1): the
  full 5D solution psi returned by the solver is checked at 12 sampled 4D sites
  with the single-site oracle, |(D_alpha psi)(x) - rhs(x)| against the RMS of
  rhs(x) over the samples (rhs = D_1(1) P b, Eq. tosolve), and z_1 =
  P_- psi_1 + P_+ psi_Ls at the same sites.  A Schur residual of 1e-10 leaves a
  5D residual of order kappa(I) 1e-10; the per-site bound 1e-7 is two orders
  above the observed value and far below the O(1) of a wrong solution.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle.lattice import P_MINUS, P_PLUS
from oracle.pointwise import PointwiseDalpha
from synthetic import gauge_field, gaussian_source4d, zolotarev_mobius

pytestmark = pytest.mark.gpu

LS = 12


def _system(L, m, alpha, eps=0.5):
    b, c, _, _ = zolotarev_mobius(LS, 0.05, 6.0)
    return O.DWFSystem(L, LS, -1.8, m, alpha, b, c, gauge_field(L, eps, seed=0))


def _op(sysm, prec, **kw):
    from paper_1501_04950_gb300 import dwf
    op = dwf.DWF(sysm.lattice, LS, sysm.M5, sysm.m, sysm.alpha, sysm.b, sysm.c,
                 precision_inner=prec, solver=dwf.SOLVER_DEFECT, **kw)
    op.load_gauge(torch.from_numpy(sysm.U).cuda())
    return op


@pytest.mark.parametrize("prec", [2, 3])
def test_zolotarev_small_vs_oracle(prec):
    L = (4, 4, 4, 4)
    sysm = _system(L, 0.005, 1.25, eps=0.3)
    src = gaussian_source4d(L, seed=1)
    op = _op(sysm, prec, maxiter=40000)
    s = torch.from_numpy(src).cuda()
    prop = torch.empty_like(s)
    st = op.cgne_solve(s, prop)
    ref = O.solve_propagator(sysm, src, tol=1e-12)
    err = np.abs(prop.cpu().numpy() - ref["z1"]).max() / np.abs(ref["z1"]).max()
    print("prec %d: iters %d restarts %d resid %.2e z1 err %.2e"
          % (prec, st[0]["iterations"], st[0]["restarts"], st[0]["true_resid"], err))
    assert st[0]["true_resid"] <= 1e-10
    assert err < 1e-7


@pytest.mark.parametrize("prec", [2, 3])
def test_zolotarev_24c48_sampled(prec):
    L = (24, 24, 24, 48)
    sysm = _system(L, 0.005, 1.25)
    src = gaussian_source4d(L, seed=1)
    op = _op(sysm, prec, maxiter=60000)
    s = torch.from_numpy(src).cuda()
    prop = torch.empty_like(s)
    sol = torch.empty((LS,) + src.shape, dtype=torch.complex128, device="cuda")
    st = op.cgne_solve(s, prop, sol)
    torch.cuda.synchronize()
    print("prec %d: iters %d restarts %d resid %.2e resid5d %.2e"
          % (prec, st[0]["iterations"], st[0]["restarts"], st[0]["true_resid"],
             st[0]["true_resid_5d"]))
    assert st[0]["true_resid"] <= 1e-10
    pw = PointwiseDalpha(sysm)
    cache = {}

    def psi_at(c):
        if c not in cache:
            x, y, z, t = c
            cache[c] = sol[:, t, z, y, x].cpu().numpy()
        return cache[c]

    rng = np.random.default_rng(5)
    res, ref = [], []
    for _ in range(12):
        site = tuple(int(rng.integers(0, n)) for n in L)
        x, y, z, t = site
        rhs = pw.rhs_at(src, site)
        res.append(np.linalg.norm(pw.apply_at(psi_at, site) - rhs))
        ref.append(np.linalg.norm(rhs))
        ps = psi_at(site)
        z1 = np.einsum("ij,jc->ic", P_MINUS, ps[0]) + np.einsum("ij,jc->ic", P_PLUS, ps[LS - 1])
        assert np.abs(prop[t, z, y, x].cpu().numpy() - z1).max() <= 1e-14 * np.abs(z1).max()
    worst = max(res) / np.sqrt(np.mean(np.square(ref)))
    print("sampled 5D residual / RMS rhs: %.2e" % worst)
    assert worst < 1e-7
