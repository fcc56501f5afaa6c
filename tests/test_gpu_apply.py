"""GPU parity of the D_bb / D_bb^+ / D_alpha applies against the FP64 oracle.

Tolerances (max_x |diff(x)| / RMS_x |ref(x)| over 5D half-sites):
  FP64  1e-12 (the required apply parity),
  FP32  5e-6  (FP32 rounding of inputs, links and ~3e3 accumulations per site),
  FP16  1e-2  (11-bit significands of inputs, links and the intermediate field),
  BF16  5e-2  (8-bit significands).
Lattices are chosen so that the last CTA is ragged (Vh not a multiple of the
sites per CTA) and so that Ls ranges over 4 .. 16.
"""
import numpy as np
import pytest
import torch

import oracle as O
from synthetic import gaussian_half5d

from gpu_common import make_case, site_norm_error

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 5e-6, 2: 1e-2, 3: 5e-2}
CASES = [
    ((4, 4, 4, 4), 8, "shamir"),
    ((6, 4, 2, 4), 12, "varying"),
    ((2, 2, 2, 6), 4, "mobius"),
    ((4, 2, 6, 2), 16, "mobius"),
]


def _op(sysm, **kw):
    from paper_1501_04950_gb300 import dwf
    op = dwf.DWF(sysm.lattice, sysm.Ls, sysm.M5, sysm.m, sysm.alpha, sysm.b, sysm.c,
                 bc_t=int(sysm.bc_t), rb_parity=sysm.black_parity, **kw)
    op.load_gauge(torch.from_numpy(sysm.U).cuda())
    return op


def _apply(op, psi, prec, dag=False, nrhs=1):
    x = op.new_field(prec, nrhs)
    y = op.new_field(prec, nrhs)
    op.pack_half(x, torch.from_numpy(np.ascontiguousarray(psi)).cuda(), prec, nrhs)
    (op.apply_Dbb_dag if dag else op.apply_Dbb)(y, x, prec, nrhs)
    out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    op.unpack_half(out, y, prec, nrhs)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("L,Ls,coeff", CASES)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_dbb_parity(L, Ls, coeff, prec):
    sysm = make_case(L, Ls, coeff)
    op = _op(sysm)
    psi = gaussian_half5d(L, Ls, seed=2)
    ref = sysm.dbb(psi)
    err = site_norm_error(_apply(op, psi, prec), ref)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("L,Ls,coeff", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_dbb_dag_parity(L, Ls, coeff, prec):
    sysm = make_case(L, Ls, coeff, alpha=0.75)
    op = _op(sysm)
    psi = gaussian_half5d(L, Ls, seed=3)
    ref = sysm.dbb_dag(psi)
    err = site_norm_error(_apply(op, psi, prec, dag=True), ref)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("bc_t,black", [(-1, 0), (1, 1), (-1, 1)])
def test_dbb_boundary_and_parity_options(bc_t, black):
    sysm = make_case((4, 4, 2, 4), 6, "varying", bc_t=bc_t, black=black)
    op = _op(sysm)
    psi = gaussian_half5d(sysm.lattice, 6, seed=4)
    assert site_norm_error(_apply(op, psi, 0), sysm.dbb(psi)) <= 1e-12
    assert site_norm_error(_apply(op, psi, 0, dag=True), sysm.dbb_dag(psi)) <= 1e-12


def test_multi_rhs_apply_equals_single():
    sysm = make_case((4, 4, 4, 2), 8, "mobius")
    op = _op(sysm)
    psis = np.stack([gaussian_half5d(sysm.lattice, 8, seed=10 + k) for k in range(3)])
    for prec in (0, 1):
        got = _apply(op, psis, prec, nrhs=3)
        for k in range(3):
            one = _apply(op, psis[k], prec)
            assert np.array_equal(got[k], one)
            assert site_norm_error(got[k], sysm.dbb(psis[k])) <= TOL[prec]


@pytest.mark.parametrize("alpha,m,bc_t", [(1.3, 0.07, 1), (1.0, 1.0, 1), (0.6, 0.02, -1)])
def test_dalpha_full_parity(alpha, m, bc_t):
    sysm = make_case((4, 2, 4, 4), 8, "varying", bc_t=bc_t)
    from paper_1501_04950_gb300 import dwf
    op = dwf.DWF(sysm.lattice, 8, sysm.M5, sysm.m, sysm.alpha, sysm.b, sysm.c, bc_t=bc_t)
    op.load_gauge(torch.from_numpy(sysm.U).cuda())
    rng = np.random.default_rng(5)
    shp = (8,) + O.shape4(sysm.lattice) + (4, 3)
    psi = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    out = torch.empty(shp, dtype=torch.complex128, device="cuda")
    op.apply_dalpha(out, torch.from_numpy(psi).cuda(), alpha, m)
    ref = O.dalpha(psi, sysm.U, sysm.M5, sysm.b, sysm.c, alpha, m, float(bc_t))
    got = out.cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-13


def test_dbb_adjoint_identity_fp64():
    """<u, D v> = <D^+ u, v> on the GPU path alone (a property at any size)."""
    sysm = make_case((4, 4, 4, 4), 8, "mobius")
    op = _op(sysm)
    u = gaussian_half5d(sysm.lattice, 8, seed=6)
    v = gaussian_half5d(sysm.lattice, 8, seed=7)
    dv = _apply(op, v, 0)
    du = _apply(op, u, 0, dag=True)
    lhs = np.vdot(u.ravel(), dv.ravel())
    rhs = np.vdot(du.ravel(), v.ravel())
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


@pytest.mark.parametrize("Ls", [8, 12, 16])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_tuned_matches_generic(Ls, prec, monkeypatch):
    """The tuned kernels (Ls in {8, 12, 16}) against the generic dense ones."""
    sysm = make_case((4, 2, 4, 6), Ls, "varying", alpha=1.4, bc_t=-1)
    psi = gaussian_half5d(sysm.lattice, Ls, seed=8)
    outs = []
    for generic in (False, True):
        if generic:
            monkeypatch.setenv("DWF_GENERIC_KERNELS", "1")
        else:
            monkeypatch.delenv("DWF_GENERIC_KERNELS", raising=False)
        op = _op(sysm)
        outs.append((_apply(op, psi, prec), _apply(op, psi, prec, dag=True)))
        op.close()
    monkeypatch.delenv("DWF_GENERIC_KERNELS", raising=False)
    tol = {0: 1e-13, 1: 2e-6, 2: 1e-2}[prec]
    for k in range(2):
        assert site_norm_error(outs[0][k], outs[1][k]) <= tol


@pytest.mark.parametrize("L,prec,tol", [((16, 16, 16, 32), 1, 5e-6), ((16, 16, 16, 32), 0, 1e-12),
                                         ((32, 32, 32, 64), 1, 5e-6)])
def test_full_size_sampled_parity(L, prec, tol):
    """16^3x32, Ls = 16 (the benchmark workload and its launch configuration) and
    32^3x64, Ls = 16 (16.8M 5D half-sites, the largest batched lattice): the GPU
    D_bb at 24 sampled black sites against the single-site oracle."""
    import oracle as O
    from oracle.pointwise import PointwiseDbb
    from synthetic import gauge_field
    Ls = 16
    sysm = O.DWFSystem(L, Ls, -1.8, 0.01, 1.0, np.full(Ls, 1.5), np.full(Ls, 0.5),
                       gauge_field(L, 0.5, seed=0))
    op = _op(sysm)
    psi = gaussian_half5d(L, Ls, seed=2)
    x = op.new_field(prec)
    y = op.new_field(prec)
    op.pack_half(x, torch.from_numpy(psi).cuda(), prec)
    op.apply_Dbb(y, x, prec)
    out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    op.unpack_half(out, y, prec)
    torch.cuda.synchronize()
    del x, y
    pw = PointwiseDbb(sysm)
    rng = np.random.default_rng(7)
    refs, gots = [], []
    while len(refs) < 24:
        c = tuple(int(rng.integers(0, n)) for n in L)
        if sum(c) % 2 != 0:
            continue
        lex = c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]))
        refs.append(pw.dbb_at(psi, c))
        gots.append(out[:, lex // 2].cpu().numpy())
    refs = np.stack(refs, axis=1)
    gots = np.stack(gots, axis=1)
    rms = np.sqrt((np.abs(refs) ** 2).sum(axis=(-1, -2)).mean())
    d = np.sqrt((np.abs(gots - refs) ** 2).sum(axis=(-1, -2)))
    assert d.max() / rms <= tol, d.max() / rms


@pytest.mark.parametrize("prec", [2, 3])
def test_16bit_store_subnormal_sites(prec):
    """A 5D site whose components are all below the smallest normal float (the far
    tail of a point-source solve) keeps scale 1 instead of overflowing its 1/max
    scale: it stores as zero in FP16 and as the (subnormal) value in BF16, whose
    exponent range is FP32's; normal sites keep their 16-bit accuracy, and D_bb of
    such a field stays finite."""
    L, Ls = (4, 4, 4, 4), 8
    sysm = make_case(L, Ls, "mobius")
    op = _op(sysm)
    psi = gaussian_half5d(L, Ls, seed=6)
    psi[3, 5] *= 1e-40          # subnormal in FP32
    psi[4, 7] *= 3e-36          # small but normal
    x = op.new_field(prec)
    op.pack_half(x, torch.from_numpy(psi).cuda(), prec)
    back = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    op.unpack_half(back, x, prec)
    b = back.cpu().numpy()
    assert np.isfinite(b).all()
    assert np.abs(b[3, 5]).max() <= (0.0 if prec == 2 else 1.2e-38)
    tol = 2e-3 if prec == 2 else 1e-2
    assert np.abs(b[4, 7] - psi[4, 7]).max() <= tol * np.abs(psi[4, 7]).max()
    mask = np.ones(psi.shape[:2], dtype=bool)
    mask[3, 5] = mask[4, 7] = False
    assert np.abs(b[mask] - psi[mask]).max() <= tol * np.abs(psi).max()
    y = op.new_field(prec)
    op.apply_Dbb(y, x, prec)
    out = torch.empty_like(back)
    op.unpack_half(out, y, prec)
    assert torch.isfinite(out).all()
