"""kpm_moments_csr_noalloc against kpm_moments.

The no-allocation entry point serves callers that cannot allocate device
memory during a call; it must give the moments the ordinary FP64 entry point
gives for the same CSR matrix, seed and rescaling, call after call, although
all calls reuse one fixed device scratch array.  This file is collected last.
"""
import numpy as np
import pytest

from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the FP64 parity tolerance used by the other GPU tests


def _csr(K, complex_):
    if complex_:
        L = (6, 5, 4)
        N = 120
        kw = dict(dims=3, L=L, periodic=(True, False, True), onsite=I.onsite_disorder(8, N, 1.0),
                  hop=I.spin_hoppings(L, *I.spins(8, N)), bond_mask=I.dilution_mask(8, N, 3))
    else:
        kw = dict(dims=2, L=(32, 32), onsite=I.onsite_disorder(1, 1024, 1.0))
    return K.kpm_stencil_to_csr(complex_=complex_, **kw)


@pytest.mark.parametrize("complex_,M,R", [(False, 256, 8), (True, 130, 5)])
def test_noalloc_matches_kpm_moments_twice(gpu_lib, complex_, M, R):
    import torch

    from paper_1105_5481_gb300 import kpm as K

    rp, col, val = _csr(K, complex_)
    n, nnz = rp.size - 1, col.size
    a, b, seed = 6.2, 0.05, 17
    with K.kpm_create_csr(n, rp, col, val, complex_=complex_) as h:
        ref = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp64")
    d_rp = torch.from_numpy(rp).cuda()
    d_col = torch.from_numpy(col).cuda()
    d_val = torch.from_numpy(val.view(np.float64) if complex_ else val).cuda()
    out = torch.empty(M, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(np.nan)
        K.kpm_moments_csr_noalloc(n, nnz, d_rp, d_col, d_val, M, R, a, b, seed=seed,
                                  complex_=complex_, out=out)
        torch.cuda.synchronize()
        assert np.abs(out.cpu().numpy() - ref).max() <= TOL
        host = K.kpm_moments_csr_noalloc(n, nnz, d_rp, d_col, d_val, M, R, a, b, seed=seed,
                                         complex_=complex_)
        assert np.abs(host - ref).max() <= TOL


def test_noalloc_rejects_problems_beyond_its_scratch(gpu_lib):
    import torch

    from paper_1105_5481_gb300 import kpm as K

    rp, col, val = _csr(K, False)
    d_rp = torch.from_numpy(rp).cuda()
    d_col = torch.from_numpy(col).cuda()
    d_val = torch.from_numpy(val).cuda()
    with pytest.raises(K.KPMError) as e:
        K.kpm_moments_csr_noalloc(rp.size - 1, col.size, d_rp, d_col, d_val, 16384, 256, 6.2, 0.0)
    assert e.value.status == K.KPM_EINVAL and "KPM_NOALLOC_SCRATCH_BYTES" in str(e.value)
