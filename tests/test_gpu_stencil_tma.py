"""The TMA-fed stencil step (bulk copies of the rows of v_n and v_{n-1}, the
forward hoppings and the on-site terms of a tile into a shared-memory ring,
one producer warp, eight consumer warps) against the plain stencil step and
the FP64 oracle.

The planner takes this form only when KPM_STENCIL_TMA asks for it (it
measured slower than the plain step on the 3D spin lattice), for FP32
vectors on 2D and 3D stencils whose vector block reaches the size given in
its fourth field (0 here, so that the oracle stays quick) and that fill the
GPU with 256-thread CTAs; every case checks the form the plan chose.  Each
row's v_{n+1} is computed by the same operations in the same order in both
kernels; the two assign rows to threads differently, so the compensated FP32
moment dots are summed in a different order and the moments may differ by
up to about 4 x 2^-23 ~ 5e-7: |d mu| <= 1e-6 between the kernels, <= 1e-5
against the oracle (the FP32-vector tolerance).  The lattices cover complex
and real hoppings, on-site terms, open edges, padded columns, 1 to 16 chunks
per row and partly filled last tiles."""
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
    if name == "cube_spin":             # the 3D spin lattice's structure, ragged size
        L = (35, 34, 33)
        N = int(np.prod(L))
        return dict(dims=3, L=L, hop=I.spin_hoppings(L, *I.spins(5, N))), True
    if name == "cube_spin_onsite_open":  # on-site terms and an open direction
        L = (33, 31, 29)
        N = int(np.prod(L))
        return dict(dims=3, L=L, periodic=(True, False, True), hop=I.spin_hoppings(L, *I.spins(6, N)),
                    onsite=I.onsite_disorder(6, N, 1.0)), True
    if name == "square_onsite":         # 2D disorder realisation (the batch workload's operator)
        L = (203, 197)
        return dict(dims=2, L=L, onsite=I.onsite_disorder(3, L[0] * L[1], 2.0)), False
    if name == "square_clean_open":     # uniform operator, open in x
        return dict(dims=2, L=(211, 190), periodic=(False, True)), False
    if name == "square_spin":           # 2D complex hoppings
        L = (181, 173)
        N = L[0] * L[1]
        return dict(dims=2, L=L, hop=I.spin_hoppings(L, *I.spins(7, N))), True
    raise KeyError(name)


def _solve(K, kw, cplx, M, R, a, b, seed, tma):
    old = os.environ.get("KPM_STENCIL_TMA")
    os.environ["KPM_STENCIL_TMA"] = tma
    try:
        with K.kpm_create_stencil(complex_=cplx, **kw) as h:
            first = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp32", per_vec=True)
            form = K.kpm_testing_last_step_form(h)
            again = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp32", per_vec=True)
        assert np.array_equal(first[1], again[1])
        return first, form
    finally:
        if old is None:
            del os.environ["KPM_STENCIL_TMA"]
        else:
            os.environ["KPM_STENCIL_TMA"] = old


@pytest.mark.parametrize("name", ["cube_spin", "cube_spin_onsite_open", "square_onsite",
                                  "square_clean_open", "square_spin"])
@pytest.mark.parametrize("R", [8, 13, 64])
def test_stencil_tma_matches_plain_step_and_oracle(K, name, R):
    kw, cplx = _case(name)
    H = O.lattice_hamiltonian(kw["L"], periodic=kw.get("periodic"), onsite=kw.get("onsite"),
                              hop=kw.get("hop"))
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    M, seed = 64, 41
    (mu_p, pv_p), form = _solve(K, kw, cplx, M, R, a, b, seed, "0")
    assert form == "fused step"
    v0 = I.random_block(seed, H.n, R, cplx)
    _, per_o = O.moments_doubling(H, a, b, v0, M)
    assert np.abs(pv_p - per_o).max() <= 1e-5
    # (stages, passes per tile, CTAs per SM, minimum block MB)
    for tma in ("2,2,2,0", "4,1,2,0", "3,1,3,0", "2,4,2,0"):
        (mu_t, pv_t), form = _solve(K, kw, cplx, M, R, a, b, seed, tma)
        assert form == "TMA-fed stencil step", tma
        assert np.abs(pv_t - pv_p).max() <= 1e-6, tma
        assert np.abs(pv_t - per_o).max() <= 1e-5, tma
        assert np.abs(mu_t - mu_p).max() <= 1e-6, tma


def test_default_and_small_blocks_keep_the_plain_step(K):
    # without KPM_STENCIL_TMA, and below the size it gives, the plain step runs
    kw, cplx = _case("square_onsite")
    old = os.environ.pop("KPM_STENCIL_TMA", None)
    try:
        with K.kpm_create_stencil(complex_=cplx, **kw) as h:
            K.kpm_moments(h, 16, 16, 8.0, 0.0, precision="fp32")
            assert K.kpm_testing_last_step_form(h) == "fused step"
        os.environ["KPM_STENCIL_TMA"] = "2,2,2,16"     # a 2.5 MB block is below 16 MB
        with K.kpm_create_stencil(complex_=cplx, **kw) as h:
            K.kpm_moments(h, 16, 16, 8.0, 0.0, precision="fp32")
            assert K.kpm_testing_last_step_form(h) == "fused step"
    finally:
        os.environ.pop("KPM_STENCIL_TMA", None)
        if old is not None:
            os.environ["KPM_STENCIL_TMA"] = old


def test_stencil_tma_wait_runs_out_and_reports_a_timeout(K):
    # the producer issues no copy (a host-side testing aid): the consumers'
    # bounded waits run out, the call returns KPM_ETIMEOUT, the context stays usable
    kw, cplx = _case("cube_spin")
    H = O.lattice_hamiltonian(kw["L"], hop=kw["hop"])
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    old = os.environ.get("KPM_STENCIL_TMA")
    os.environ["KPM_STENCIL_TMA"] = "2,2,2,0"
    try:
        K.kpm_testing_stall_step_pipeline(True)
        try:
            with K.kpm_create_stencil(complex_=True, **kw) as h:
                with pytest.raises(K.KPMError) as e:
                    K.kpm_moments(h, 4, 32, a, b, seed=1, precision="fp32")
                assert e.value.status == K.KPM_ETIMEOUT
                assert K.kpm_testing_last_step_form(h) == "TMA-fed stencil step"
        finally:
            K.kpm_testing_stall_step_pipeline(False)
        with K.kpm_create_stencil(complex_=True, **kw) as h:
            mu = K.kpm_moments(h, 64, 32, a, b, seed=1, precision="fp32")
            assert K.kpm_testing_last_step_form(h) == "TMA-fed stencil step"
    finally:
        if old is None:
            del os.environ["KPM_STENCIL_TMA"]
        else:
            os.environ["KPM_STENCIL_TMA"] = old
    mu_o, _ = O.moments_doubling(H, a, b, I.random_block(1, H.n, 32, True), 64)
    assert np.abs(mu - mu_o).max() <= 1e-5
