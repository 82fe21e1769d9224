"""The TMA-fed padded-ELL step (bulk copies of the streamed rows, column
indices and values into a shared-memory ring, one producer warp, eight
consumer warps) against the plain ELL step and the FP64 oracle.

The planner takes this form for FP32 vectors on padded-ELL operators when
the lattice fills the GPU with full 256-thread CTAs (rows x chunks per row
>= 256 x 152); the lattices here are sized for that, and every case checks
the form the plan chose.  Each row's v_{n+1} is computed by the same
operations in the same order in both kernels; the two assign rows to threads
differently, so the moment dots are summed in a different order.  Each
thread sums in compensated FP32 pairs (error up to about 2u = 2^-23 of the
sum of magnitudes), then in FP64, so the two kernels' moments differ by up
to about 4 x 2^-23 ~ 5e-7 (measured 6e-9): |d mu| <= 1e-6 between them, and
<= 1e-5 against the oracle (the FP32-vector tolerance).  The lattices give
ELL widths 2, 4, 6 and 8, vector blocks of 1 to 8 chunks per row, and last
tiles that are only partly filled."""
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
        return dict(dims=1, L=(40003,)), False
    if name == "square_W4":           # 2D clean: 4 entries per row
        return dict(dims=2, L=(201, 199)), False
    if name == "square_W6":           # 2D with disorder: 5 entries per row -> width 6
        L = (203, 197)
        return dict(dims=2, L=L, onsite=I.onsite_disorder(3, L[0] * L[1], 2.0)), False
    if name == "cube_spin_dilute_W6":  # the large workload's structure, ragged size
        L = (35, 34, 33)
        N = 35 * 34 * 33
        return dict(dims=3, L=L, hop=I.spin_hoppings(L, *I.spins(5, N)),
                    bond_mask=I.dilution_mask(5, N, 3)), True
    if name == "cube_onsite_W8":      # 7 entries per row -> width 8
        L = (35, 33, 34)
        N = 35 * 33 * 34
        return dict(dims=3, L=L, hop=I.spin_hoppings(L, *I.spins(6, N)),
                    onsite=I.onsite_disorder(6, N, 1.0)), True
    raise KeyError(name)


def _solve(K, rp, col, val, cplx, M, R, a, b, seed, tma):
    old = os.environ.get("KPM_ELL_TMA")
    os.environ["KPM_ELL_TMA"] = tma
    try:
        with K.kpm_create_csr(rp.size - 1, rp, col, val, complex_=cplx) as h:
            first = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp32", per_vec=True)
            form = K.kpm_testing_last_step_form(h)
            again = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp32", per_vec=True)
            third = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp32", per_vec=True)
        assert np.array_equal(first[1], again[1]) and np.array_equal(first[1], third[1])
        return first, form
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
    M, seed = 96, 29
    rp, col, val = K.kpm_stencil_to_csr(complex_=cplx, **kw)
    (mu_p, pv_p), form = _solve(K, rp, col, val, cplx, M, R, a, b, seed, "0")
    assert form == "fused step"
    v0 = I.random_block(seed, H.n, R, cplx)
    _, per_o = O.moments_doubling(H, a, b, v0, M)
    assert np.abs(pv_p - per_o).max() <= 1e-5
    # (stages, passes per tile, CTAs per SM[, prefetch distance]); 8 x 1 of the
    # widest rows does not fit in shared memory and falls back to the plain step
    for tma in ("2,2,2", "4,1,2", "3,1,3", "2,2,3", "2,2,2,1", "8,1,2"):
        (mu_t, pv_t), form = _solve(K, rp, col, val, cplx, M, R, a, b, seed, tma)
        if tma != "8,1,2":
            assert form == "TMA-fed ELL step", tma
        assert np.abs(pv_t - pv_p).max() <= 1e-6, tma
        assert np.abs(pv_t - per_o).max() <= 1e-5, tma
        assert np.abs(mu_t - mu_p).max() <= 1e-6, tma


def test_small_lattices_keep_the_plain_step(K):
    # too few rows to fill the GPU with 256-thread CTAs: a chain of steps
    # takes smaller CTAs of the plain step instead of the TMA-fed form (and by
    # default such a lattice runs as the column-resident solve, no chain at all)
    rp, col, val = K.kpm_stencil_to_csr(dims=2, L=(32, 32))
    old = os.environ.get("KPM_COLRES")
    os.environ["KPM_COLRES"] = "0"
    try:
        with K.kpm_create_csr(rp.size - 1, rp, col, val) as h:
            K.kpm_moments(h, 16, 8, 4.1, 0.0, precision="fp32")
            assert K.kpm_testing_last_step_form(h) == "fused step"
    finally:
        if old is None:
            os.environ.pop("KPM_COLRES", None)
        else:
            os.environ["KPM_COLRES"] = old
    with K.kpm_create_csr(rp.size - 1, rp, col, val) as h:
        K.kpm_moments(h, 16, 8, 4.1, 0.0, precision="fp32")
        assert K.kpm_testing_last_step_form(h) == "column-resident solve"
