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

TOL = {0: 1e-12, 1: 5e-6}


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_apply_twice(prec):
    from paper_1501_04950_gb300 import dwf
    sysm = make_case((8, 8, 8, 16), 8, "mobius", alpha=1.25, m=0.02)
    op = dwf.DWF(sysm.lattice, 8, sysm.M5, sysm.m, sysm.alpha, sysm.b, sysm.c)
    op.load_gauge(torch.from_numpy(sysm.U).cuda())
    nrhs = 2
    psi = np.stack([gaussian_half5d(sysm.lattice, 8, seed=20 + k) for k in range(nrhs)])
    x = op.new_field(prec, nrhs)
    op.pack_half(x, torch.from_numpy(psi).cuda(), prec, nrhs)
    ref = op.new_field(prec, nrhs)
    op.apply_Dbb(ref, x, prec, nrhs)
    ref_c = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    op.unpack_half(ref_c, ref, prec, nrhs)
    for call in range(2):
        y = op.new_field(prec, nrhs)
        op.apply_Dbb_noalloc(y, x, prec, nrhs)
        got = torch.empty_like(ref_c)
        op.unpack_half(got, y, prec, nrhs)
        torch.cuda.synchronize()
        for k in range(nrhs):
            err = site_norm_error(got[k].cpu().numpy(), ref_c[k].cpu().numpy())
            assert err <= TOL[prec], (call, k, err)
    op.close()


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
