"""kpm_moments_csr_noalloc against kpm_moments and the oracle.

The no-allocation entry point serves callers that cannot allocate device
memory during a call (a frozen or exhausted pool, all memory budgeted at
start-up, no tolerance for the synchronisation of cudaMalloc/cudaFree).  It
must give the moments the ordinary FP64 entry point and the FP64 oracle give
for the same CSR matrix, seed and rescaling, call after call, although all
calls reuse one fixed device scratch array; a call must leave the device's
free memory unchanged; and a malformed CSR structure, which the library can
only inspect on the device, must be refused without any out-of-bounds access.
This file is collected last.
"""
import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the FP64 parity tolerance used by the other GPU tests


def _case(complex_):
    if complex_:
        L = (6, 5, 4)
        N = 120
        kw = dict(dims=3, L=L, periodic=(True, False, True), onsite=I.onsite_disorder(8, N, 1.0),
                  hop=I.spin_hoppings(L, *I.spins(8, N)), bond_mask=I.dilution_mask(8, N, 3))
    else:
        kw = dict(dims=2, L=(32, 32), onsite=I.onsite_disorder(1, 1024, 1.0))
    return kw


def _csr(K, complex_):
    return K.kpm_stencil_to_csr(complex_=complex_, **_case(complex_))


def _device(rp, col, val, complex_):
    import torch

    return (torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(),
            torch.from_numpy(val.view(np.float64) if complex_ else val).cuda())


@pytest.mark.parametrize("complex_,M,R", [(False, 256, 8), (True, 130, 5)])
def test_noalloc_matches_kpm_moments_and_oracle_twice(gpu_lib, complex_, M, R):
    import torch

    from paper_1105_5481_gb300 import kpm as K

    rp, col, val = _csr(K, complex_)
    n, nnz = rp.size - 1, col.size
    a, b, seed = 6.2, 0.05, 17
    with K.kpm_create_csr(n, rp, col, val, complex_=complex_) as h:
        ref = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp64")
    kw = _case(complex_)
    H = O.lattice_hamiltonian(kw["L"], periodic=kw.get("periodic"), onsite=kw.get("onsite"),
                              hop=kw.get("hop"), mask=kw.get("bond_mask"))
    v0 = (I.phase_block if complex_ else I.rademacher_block)(seed, n, R)
    mu_o, _ = O.moments_doubling(H, a, b, v0, M)
    d_rp, d_col, d_val = _device(rp, col, val, complex_)
    out = torch.empty(M, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(np.nan)
        K.kpm_moments_csr_noalloc(n, nnz, d_rp, d_col, d_val, M, R, a, b, seed=seed,
                                  complex_=complex_, out=out)
        torch.cuda.synchronize()
        dev = out.cpu().numpy()
        assert np.abs(dev - ref).max() <= TOL
        assert np.abs(dev - mu_o).max() <= TOL
        host = K.kpm_moments_csr_noalloc(n, nnz, d_rp, d_col, d_val, M, R, a, b, seed=seed,
                                         complex_=complex_)
        assert np.abs(host - ref).max() <= TOL
        assert np.abs(host - mu_o).max() <= TOL


def test_noalloc_leaves_free_device_memory_unchanged(gpu_lib):
    import torch

    from paper_1105_5481_gb300 import kpm as K

    rp, col, val = _csr(K, False)
    d_rp, d_col, d_val = _device(rp, col, val, False)
    out = torch.empty(256, dtype=torch.float64, device="cuda")
    args = (rp.size - 1, col.size, d_rp, d_col, d_val, 256, 8, 6.2, 0.05)
    K.kpm_moments_csr_noalloc(*args, seed=3, out=out)      # first call: module and address set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for s in range(3):
        K.kpm_moments_csr_noalloc(*args, seed=4 + s, out=out)
        K.kpm_moments_csr_noalloc(*args, seed=4 + s)         # host output as well
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_refuses_a_malformed_structure(gpu_lib):
    import torch

    from paper_1105_5481_gb300 import kpm as K

    rp, col, val = _csr(K, False)
    n, nnz = rp.size - 1, col.size
    bad_end = rp.copy()
    bad_end[-1] = nnz + 5                                   # rowptr[n] != nnz
    bad_col = col.copy()
    bad_col[nnz // 2] = n + 100                              # a column outside [0, n)
    bad_order = rp.copy()
    bad_order[10] = bad_order[12] + 1                        # rowptr decreases
    good = K.kpm_moments_csr_noalloc(n, nnz, *_device(rp, col, val, False), 64, 8, 6.2, 0.05)
    for r, c in ((bad_end, col), (rp, bad_col), (bad_order, col)):
        d_rp, d_col, d_val = _device(r, c, val, False)
        with pytest.raises(K.KPMError) as e:
            K.kpm_moments_csr_noalloc(n, nnz, d_rp, d_col, d_val, 64, 8, 6.2, 0.05)
        assert e.value.status == K.KPM_EINVAL and "malformed CSR" in str(e.value)
        out = torch.zeros(64, dtype=torch.float64, device="cuda")
        K.kpm_moments_csr_noalloc(n, nnz, d_rp, d_col, d_val, 64, 8, 6.2, 0.05, out=out)
        assert torch.isnan(out).all()
    # the shared scratch is usable again after a refused call
    again = K.kpm_moments_csr_noalloc(n, nnz, *_device(rp, col, val, False), 64, 8, 6.2, 0.05)
    assert np.array_equal(again, good)


def test_noalloc_rejects_problems_beyond_its_scratch(gpu_lib):
    from paper_1105_5481_gb300 import kpm as K

    rp, col, val = _csr(K, False)
    d_rp, d_col, d_val = _device(rp, col, val, False)
    with pytest.raises(K.KPMError) as e:
        K.kpm_moments_csr_noalloc(rp.size - 1, col.size, d_rp, d_col, d_val, 16384, 256, 6.2, 0.0)
    assert e.value.status == K.KPM_EINVAL and "KPM_NOALLOC_SCRATCH_BYTES" in str(e.value)
