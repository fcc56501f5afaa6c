"""GPU fermion force dS/dU, S = phi^+ (D_bb^+ D_bb)^-1 phi.

* against the oracle's adjoint-formula gradient (raw link gradient and the
  su(3) projection TA(U G^+)) on small lattices, tuned (Ls = 8) and generic
  (Ls = 6) kernels;
* on the 8^3x16, Ls = 8 adjoint workload (Mobius b = 1.5, c = 0.5, m = 0.02,
  alpha = 1.5, FP64): central finite differences (h = 1e-5) of the GPU action
  on 64 random links (one raw entry each, real and imaginary part) and along
  the 8 su(3) generators of 8 links;
* through torch.autograd (FermionAction).
FD tolerance: the truncation error O(h^2 S''') is ~1e-10, but at this volume
S = phi^+ X is ~1e5-1e6, so the FP64 rounding of S and the solver residual
(X^+ r at rel_tol 1e-13) divided by 2h = 2e-5 leave an FD noise floor of
~1e-5 on derivatives of order one: the bound is 1e-4 of max(1, |dS|).
"""
import numpy as np
import pytest
import torch

import oracle as O
from synthetic import gauge_field, gaussian_half5d

from gpu_common import make_case

pytestmark = pytest.mark.gpu


def _op(sysm, **kw):
    from paper_1501_04950_gb300 import dwf
    opts = dict(solver=dwf.SOLVER_FP64, rel_tol=1e-13)
    opts.update(kw)
    return dwf.DWF(sysm.lattice, sysm.Ls, sysm.M5, sysm.m, sysm.alpha, sysm.b, sysm.c,
                   bc_t=int(sysm.bc_t), rb_parity=sysm.black_parity, **opts)


@pytest.mark.parametrize("Ls,coeff,bc_t,black", [(8, "mobius", 1, 0), (6, "varying", -1, 1)])
def test_force_matches_oracle_gradient(Ls, coeff, bc_t, black):
    sysm = make_case((4, 4, 4, 4), Ls, coeff, alpha=1.5, m=0.05, bc_t=bc_t, black=black)
    op = _op(sysm)
    U = torch.from_numpy(sysm.U).cuda()
    op.load_gauge(U)
    phi = gaussian_half5d(sysm.lattice, Ls, seed=2)
    phit = torch.from_numpy(phi).cuda()
    G = torch.empty_like(U)
    op.force(G, phit, None, projected=False)
    F = torch.empty_like(U)
    op.force(F, phit, None, projected=True)
    x_ref, _ = O.cg_normal(sysm, phi, tol=1e-13)
    g_ref = O.force_gradient(sysm, phi, x_ref)
    f_ref = O.su3_force(sysm.U, g_ref)
    g = G.cpu().numpy()
    f = F.cpu().numpy()
    err_g = np.abs(g - g_ref).max() / np.abs(g_ref).max()
    err_f = np.abs(f - f_ref).max() / np.abs(f_ref).max()
    print("force vs oracle: raw %.2e projected %.2e" % (err_g, err_f))
    assert err_g < 1e-9 and err_f < 1e-9


def _config4():
    L = (8, 8, 8, 16)
    Ls = 8
    b, c = np.full(Ls, 1.5), np.full(Ls, 0.5)
    U = gauge_field(L, 0.5, seed=0)
    sysm = O.DWFSystem(L, Ls, -1.8, 0.02, 1.5, b, c, U)
    phi = gaussian_half5d(L, Ls, seed=2)
    return sysm, phi


def _action(op, U, phit):
    op.load_gauge(U)
    X = torch.empty_like(phit)
    op.solve_normal(X, phit)
    return float(torch.real(torch.vdot(phit.reshape(-1), X.reshape(-1))).item())


def test_config4_force_vs_finite_differences():
    from paper_1501_04950_gb300 import dwf
    sysm, phi = _config4()
    op = _op(sysm)
    op_fd = _op(sysm, solver=dwf.SOLVER_RELIABLE)
    U = torch.from_numpy(sysm.U).cuda()
    phit = torch.from_numpy(phi).cuda()
    op.load_gauge(U)
    G = torch.empty_like(U)
    op.force(G, phit, None, projected=False)
    F = torch.empty_like(U)
    op.force(F, phit, None, projected=True)
    G = G.cpu().numpy()
    F = F.cpu().numpy()
    rng = np.random.default_rng(3)
    h = 1e-5
    worst = 0.0
    for _ in range(64):
        t, z, y, x = (int(rng.integers(0, n)) for n in (16, 8, 8, 8))
        mu, i, j = int(rng.integers(0, 4)), int(rng.integers(0, 3)), int(rng.integers(0, 3))
        for part, unit in (("re", 1.0), ("im", 1j)):
            up = U.clone()
            um = U.clone()
            up[t, z, y, x, mu, i, j] += h * unit
            um[t, z, y, x, mu, i, j] -= h * unit
            fd = (_action(op_fd, up, phit) - _action(op_fd, um, phit)) / (2 * h)
            want = G[t, z, y, x, mu, i, j].real if part == "re" else G[t, z, y, x, mu, i, j].imag
            rel = abs(fd - want) / max(1.0, abs(want))
            worst = max(worst, rel)
            assert rel < 1e-4, (part, fd, want)
    # su(3) directions: dS/dh of S(exp(i h T_a) U) = i tr(T_a F)
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    for _ in range(8):
        t, z, y, x = (int(rng.integers(0, n)) for n in (16, 8, 8, 8))
        mu = int(rng.integers(0, 4))
        for a in range(8):
            w, v = np.linalg.eigh(lam[a] / 2)
            def rot(s):
                e = torch.from_numpy(v @ np.diag(np.exp(1j * s * w)) @ np.conj(v.T)).cuda()
                uu = U.clone()
                uu[t, z, y, x, mu] = e @ U[t, z, y, x, mu]
                return uu
            fd = (_action(op_fd, rot(h), phit) - _action(op_fd, rot(-h), phit)) / (2 * h)
            want = (1j * np.trace(lam[a] / 2 @ F[t, z, y, x, mu])).real
            rel = abs(fd - want) / max(1.0, abs(want))
            worst = max(worst, rel)
            assert rel < 1e-4, (a, fd, want)
    print("config 4 FD worst relative error %.2e" % worst)


def test_autograd_function():
    from paper_1501_04950_gb300.force import fermion_action
    sysm = make_case((4, 4, 2, 4), 8, "mobius", alpha=1.5, m=0.02)
    op = _op(sysm, rel_tol=1e-12)
    U = torch.from_numpy(sysm.U).cuda().requires_grad_(True)
    phit = torch.from_numpy(gaussian_half5d(sysm.lattice, 8, seed=5)).cuda()
    S = fermion_action(U, phit, op)
    (gU,) = torch.autograd.grad(S, U)
    x_ref, _ = O.cg_normal(sysm, phit.cpu().numpy(), tol=1e-13)
    assert abs(S.item() - O.action(sysm, phit.cpu().numpy(), x_ref)) < 1e-9 * abs(S.item())
    g_ref = O.force_gradient(sysm, phit.cpu().numpy(), x_ref)
    assert np.abs(gU.cpu().numpy() - g_ref).max() / np.abs(g_ref).max() < 1e-9
