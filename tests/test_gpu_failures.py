"""Failure statuses of the C ABI, produced without faulting the GPU.

Every failure is made on the host (a non-finite link or source, a too small
iteration budget) or through the bounded waits of the tensor-copy staged hop
kernel: its one-shot test hook (DWF_TEST_SKIP_HOP) leaves one hop's stage
unarmed, so the consumers' clock-bounded waits run out, the kernel sets the
device error flag and returns, and the solver reports DWF_ERR_TIMEOUT.  The
handle must stay usable after each failure.  The staged kernel also has to
agree bit for bit with the direct-load kernel.
"""
import numpy as np
import pytest
import torch

from synthetic import gaussian_half5d, gaussian_source4d

from gpu_common import make_case

pytestmark = pytest.mark.gpu

BREAKDOWN, NOT_CONVERGED, TIMEOUT = 5, 4, 6


def _op(sysm, **kw):
    from paper_1501_04950_gb300 import dwf
    return dwf.DWF(sysm.lattice, sysm.Ls, sysm.M5, sysm.m, sysm.alpha, sysm.b, sysm.c,
                   bc_t=int(sysm.bc_t), rb_parity=sysm.black_parity, **kw)


def _src(L):
    return torch.from_numpy(gaussian_source4d(L, seed=1)).cuda()


def _solve_code(op, src, prop):
    from paper_1501_04950_gb300 import dwf
    try:
        st = op.cgne_solve(src, prop)
    except dwf.DWFError as e:
        return e.code, None
    return 0, st


def test_nan_link_and_source_give_breakdown():
    L = (4, 4, 4, 4)
    sysm = make_case(L, 8, "mobius", alpha=1.2, m=0.05)
    op = _op(sysm)
    U = sysm.U.copy()
    U[1, 2, 3, 0, 2, 1, 1] = np.nan          # one link entry
    op.load_gauge(torch.from_numpy(U).cuda())
    src = _src(L)
    prop = torch.empty_like(src)
    code, _ = _solve_code(op, src, prop)
    assert code == BREAKDOWN
    # the handle stays usable: a finite field solves
    op.load_gauge(torch.from_numpy(sysm.U).cuda())
    code, st = _solve_code(op, src, prop)
    assert code == 0 and st[0]["true_resid"] <= 1e-10
    bad = src.clone()
    bad[0, 0, 0, 1, 2, 1] = float("inf")    # a non-finite source entry
    code, _ = _solve_code(op, bad, prop)
    assert code == BREAKDOWN
    code, st = _solve_code(op, src, prop)
    assert code == 0 and st[0]["true_resid"] <= 1e-10


def test_maxiter_gives_not_converged_with_outputs():
    L = (4, 4, 4, 4)
    sysm = make_case(L, 8, "mobius", alpha=1.2, m=0.05)
    op = _op(sysm, maxiter=5)
    op.load_gauge(torch.from_numpy(sysm.U).cuda())
    src = _src(L)
    prop = torch.zeros_like(src)
    code, _ = _solve_code(op, src, prop)
    assert code == NOT_CONVERGED
    prop.zero_()
    st = op.cgne_solve(src, prop, allow_not_converged=True)[0]
    # stats are filled with the last iterate's figures, prop4d with its z_1
    assert 0 < st["iterations"] <= 16 and st["restarts"] >= 1
    assert 1e-10 < st["true_resid"] < 1.0
    p = prop.cpu().numpy()
    assert np.isfinite(p).all() and np.abs(p).max() > 0


@pytest.mark.parametrize("hop", [0, 5])
def test_staged_wait_timeout(hop, monkeypatch):
    """The staged kernel's bounded waits run out (one unarmed hop) -> DWF_ERR_TIMEOUT;
    the next solve on the same handle converges."""
    L = (4, 4, 4, 4)
    sysm = make_case(L, 8, "mobius", alpha=1.2, m=0.05)
    monkeypatch.setenv("DWF_TMA", "1")
    monkeypatch.setenv("DWF_TEST_SKIP_HOP", str(hop))
    monkeypatch.setenv("DWF_WAIT_BUDGET", "4000000")   # ~2 ms per wait
    op = _op(sysm)
    monkeypatch.delenv("DWF_TEST_SKIP_HOP")
    monkeypatch.delenv("DWF_WAIT_BUDGET")
    op.load_gauge(torch.from_numpy(sysm.U).cuda())
    src = _src(L)
    prop = torch.empty_like(src)
    code, _ = _solve_code(op, src, prop)
    assert code == TIMEOUT
    code, st = _solve_code(op, src, prop)
    assert code == 0 and st[0]["true_resid"] <= 1e-10
    monkeypatch.delenv("DWF_TMA")
    ref = _op(sysm)
    ref.load_gauge(torch.from_numpy(sysm.U).cuda())
    prop_ref = torch.empty_like(src)
    ref.cgne_solve(src, prop_ref)
    torch.cuda.synchronize()
    assert torch.allclose(prop, prop_ref, rtol=0, atol=1e-8 * prop_ref.abs().max().item())


@pytest.mark.parametrize("Ls", [8, 12, 16])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_staged_matches_direct_loads(Ls, prec, monkeypatch):
    """Tensor-copy staged neighbours (DWF_TMA=1) against direct loads: bitwise equal
    D_bb and D_bb^+ (antiperiodic t, odd black parity, site-varying coefficients)."""
    sysm = make_case((4, 4, 2, 6), Ls, "varying", alpha=0.8, bc_t=-1, black=1)
    psi = torch.from_numpy(gaussian_half5d(sysm.lattice, Ls, seed=9)).cuda()
    outs = []
    for staged in (False, True):
        if staged:
            monkeypatch.setenv("DWF_TMA", "1")
        else:
            monkeypatch.delenv("DWF_TMA", raising=False)
        op = _op(sysm)
        op.load_gauge(torch.from_numpy(sysm.U).cuda())
        x = op.new_field(prec)
        op.pack_half(x, psi, prec)
        res = []
        for fn in (op.apply_Dbb, op.apply_Dbb_dag):
            y = op.new_field(prec)
            fn(y, x, prec)
            res.append(y.cpu())
        outs.append(res)
        op.close()
    monkeypatch.delenv("DWF_TMA", raising=False)
    for k in range(2):
        assert torch.equal(outs[0][k], outs[1][k])


@pytest.mark.parametrize("Ls", [8, 12, 16])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_small_tile_matches_default_tile(Ls, prec, monkeypatch):
    """The small CTA tile of the tuned hop kernels (DWF_HOP_TILE=small, 64 threads)
    against the default tile: bitwise equal D_bb and D_bb^+ (ragged last CTAs for
    Ls = 8 and 12)."""
    sysm = make_case((6, 4, 2, 6), Ls, "varying", alpha=0.8, bc_t=-1, black=1)
    psi = torch.from_numpy(gaussian_half5d(sysm.lattice, Ls, seed=11)).cuda()
    outs = []
    for tile in ("default", "small"):
        monkeypatch.setenv("DWF_HOP_TILE", tile)
        op = _op(sysm)
        op.load_gauge(torch.from_numpy(sysm.U).cuda())
        x = op.new_field(prec)
        op.pack_half(x, psi, prec)
        res = []
        for fn in (op.apply_Dbb, op.apply_Dbb_dag):
            y = op.new_field(prec)
            fn(y, x, prec)
            res.append(y.cpu())
        outs.append(res)
        op.close()
    monkeypatch.delenv("DWF_HOP_TILE", raising=False)
    for k in range(2):
        assert torch.equal(outs[0][k], outs[1][k])
