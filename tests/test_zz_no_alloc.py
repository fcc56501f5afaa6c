"""The D_bb entry point that allocates nothing (dwf_apply_Dbb_noalloc).

It exists for callers that cannot allocate device memory, e.g. frameworks whose
pool allocator owns the GPU, or loops that cannot afford cudaMalloc's implicit
synchronisation.  It must give the result of dwf_apply_Dbb (within the apply
tolerances of test_gpu_apply.py) on consecutive calls, using only the
library's static scratch array, and reject problems larger than that array.
This file is named to be collected last.
"""
import numpy as np
import pytest
import torch

from synthetic import gaussian_half5d

from gpu_common import make_case, site_norm_error

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 5e-6, 2: 1e-2, 3: 5e-2}


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_noalloc_matches_apply_twice(prec):
    """On a fresh handle the allocation-free call comes first and leaves the free
    device memory unchanged; two calls in a row match dwf_apply_Dbb of a second
    handle (the kernels are loaded by a warm-up apply on a third handle, so that
    lazy module loading does not count as an allocation of the call)."""
    from paper_1501_04950_gb300 import dwf
    sysm = make_case((8, 8, 8, 16), 8, "mobius", alpha=1.25, m=0.02)
    nrhs = 2
    psi = np.stack([gaussian_half5d(sysm.lattice, 8, seed=20 + k) for k in range(nrhs)])

    def make():
        op = dwf.DWF(sysm.lattice, 8, sysm.M5, sysm.m, sysm.alpha, sysm.b, sysm.c)
        op.load_gauge(torch.from_numpy(sysm.U).cuda())
        x = op.new_field(prec, nrhs)
        op.pack_half(x, torch.from_numpy(psi).cuda(), prec, nrhs)
        return op, x

    warm, xw = make()
    yw = warm.new_field(prec, nrhs)
    warm.apply_Dbb_noalloc(yw, xw, prec, nrhs)
    warm.apply_Dbb(yw, xw, prec, nrhs)
    op, x = make()
    ys = [op.new_field(prec, nrhs) for _ in range(2)]
    got = [torch.empty(psi.shape, dtype=torch.complex128, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    op.apply_Dbb_noalloc(ys[0], x, prec, nrhs)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    op.apply_Dbb_noalloc(ys[1], x, prec, nrhs)
    ref_op, xr = make()
    ref = ref_op.new_field(prec, nrhs)
    ref_op.apply_Dbb(ref, xr, prec, nrhs)
    ref_c = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    ref_op.unpack_half(ref_c, ref, prec, nrhs)
    for call in range(2):
        op.unpack_half(got[call], ys[call], prec, nrhs)
        torch.cuda.synchronize()
        for k in range(nrhs):
            err = site_norm_error(got[call][k].cpu().numpy(), ref_c[k].cpu().numpy())
            assert err <= TOL[prec], (call, k, err)
    for o in (warm, op, ref_op):
        o.close()


def test_noalloc_rejects_oversize():
    from paper_1501_04950_gb300 import dwf
    sysm = make_case((8, 8, 8, 16), 8, "mobius")
    op = dwf.DWF(sysm.lattice, 8, sysm.M5, sysm.m, sysm.alpha, sysm.b, sysm.c)
    op.load_gauge(torch.from_numpy(sysm.U).cuda())
    fb = op.field_bytes(dwf.FP64)
    nrhs = dwf.NOALLOC_SCRATCH_BYTES // fb + 1
    x = op.new_field(dwf.FP64, nrhs)
    y = op.new_field(dwf.FP64, nrhs)
    with pytest.raises(dwf.DWFError) as e:
        op.apply_Dbb_noalloc(y, x, dwf.FP64, nrhs)
    assert e.value.code == 1 and "static scratch" in str(e.value)
    op.close()
