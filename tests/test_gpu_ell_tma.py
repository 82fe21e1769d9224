"""The TMA-fed padded-ELL step (bulk copies of the streamed rows, column
indices and values into a shared-memory ring, one producer warp, eight
consumer warps) against the plain ELL step and the FP64 oracle.

Each row's v_{n+1} is computed by the same operations in the same order in
both kernels, so the recursion's vectors are bitwise the same and the
moments differ only by the order of the moment sums (compensated FP32 per
thread, FP64 across threads): |d mu| <= 1e-12 between the two kernels, and
<= 1e-5 against the oracle (the FP32-vector tolerance).  The lattices give
ELL widths 2, 4, 6 and 8, vector blocks of 1, 2 and 8 chunks per row, and
last tiles that are only partly filled."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K(gpu_lib):
    from paper_1105_5481_gb300 import kpm

    return kpm


def _case(name):
    if name == "chain_W2":            # 1D periodic chain: 2 entries per row
        L = (1237,)
        return dict(dims=1, L=L, hop=None, onsite=None, bond_mask=None), False
    if name == "square_W6":           # 2D with disorder: 5 entries per row -> width 6
        L = (37, 29)
        return dict(dims=2, L=L, onsite=I.onsite_disorder(3, 37 * 29, 2.0)), False
    if name == "square_W4":
        L = (40, 25)
        return dict(dims=2, L=L), False
    if name == "cube_spin_dilute_W6":  # the large workload's structure, ragged size
        L = (13, 11, 7)
        N = 1001
        return dict(dims=3, L=L, hop=I.spin_hoppings(L, *I.spins(5, N)),
                    bond_mask=I.dilution_mask(5, N, 3)), True
    if name == "cube_onsite_W8":      # 7 entries per row -> width 8
        L = (9, 8, 7)
        N = 504
        return dict(dims=3, L=L, hop=I.spin_hoppings(L, *I.spins(6, N)),
                    onsite=I.onsite_disorder(6, N, 1.0)), True
    raise KeyError(name)


def _solve(K, kw, cplx, M, R, a, b, seed, tma):
    old = os.environ.get("KPM_ELL_TMA")
    os.environ["KPM_ELL_TMA"] = tma
    try:
        rp, col, val = K.kpm_stencil_to_csr(complex_=cplx, **kw)
        with K.kpm_create_csr(rp.size - 1, rp, col, val, complex_=cplx) as h:
            first = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp32", per_vec=True)
            again = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp32", per_vec=True)
            third = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp32", per_vec=True)
        assert np.array_equal(first[1], again[1]) and np.array_equal(first[1], third[1])
        return first
    finally:
        if old is None:
            del os.environ["KPM_ELL_TMA"]
        else:
            os.environ["KPM_ELL_TMA"] = old


@pytest.mark.parametrize("name", ["chain_W2", "square_W4", "square_W6", "cube_spin_dilute_W6",
                                  "cube_onsite_W8"])
@pytest.mark.parametrize("R", [4, 13, 32])
def test_tma_step_matches_plain_step_and_oracle(K, name, R):
    kw, cplx = _case(name)
    H = O.lattice_hamiltonian(kw["L"], onsite=kw.get("onsite"), hop=kw.get("hop"),
                              mask=kw.get("bond_mask"))
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    M, seed = 160, 29
    mu_p, pv_p = _solve(K, kw, cplx, M, R, a, b, seed, "0")
    v0 = I.random_block(seed, H.n, R, cplx)
    _, per_o = O.moments_doubling(H, a, b, v0, M)
    for tma in ("4,1,2", "2,2,2", "3,1,3", "8,1,2", "2,2,3", "2,2,2,1", "4,1,2,0"):
        mu_t, pv_t = _solve(K, kw, cplx, M, R, a, b, seed, tma)
        assert np.abs(pv_t - pv_p).max() <= 1e-12, tma
        assert np.abs(pv_t - per_o).max() <= 1e-5, tma
        assert np.abs(mu_t - mu_p).max() <= 1e-12, tma
