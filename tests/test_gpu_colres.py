"""The column-resident solve through the C ABI: every product of a realisation
of a small stencil operator in one launch of independent thread-block
clusters, one per group of vector columns, with the two vector blocks in
shared memory.  Checked against the FP64 oracle (Eqs. (rn), (munr), doubling
form) on the same seeded inputs at the parity tolerances (|d mu| <= 1e-10
FP64, <= 1e-5 FP32 vectors), against the chain of step launches it replaces,
at every cluster shape (forced through KPM_COLRES="C,cpc"), with ragged row
splits, CTAs without rows, column groups with padding columns, several
realisations, a continued solve and a start block written on the device; and
the same for CSR operators held as a padded ELL (rows of at most 8 entries)."""
import contextlib
import os

import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "fp32": 1e-5}
FORM = "column-resident solve"


@pytest.fixture(scope="module")
def K(gpu_lib):
    from paper_1105_5481_gb300 import kpm

    return kpm


@contextlib.contextmanager
def colres_env(value):
    """KPM_COLRES for the plans made inside the block (None: unset)."""
    old = os.environ.get("KPM_COLRES")
    if value is None:
        os.environ.pop("KPM_COLRES", None)
    else:
        os.environ["KPM_COLRES"] = value
    try:
        yield
    finally:
        if old is None:
            os.environ.pop("KPM_COLRES", None)
        else:
            os.environ["KPM_COLRES"] = old


def _ragged():
    """3D complex spin hoppings, odd sizes, one open dimension, dilution, disorder."""
    L = (5, 3, 7)
    n = 105
    kw = dict(dims=3, L=L, periodic=(True, False, True), onsite=I.onsite_disorder(4, n, 2.0),
              hop=I.spin_hoppings(L, *I.spins(4, n)), bond_mask=I.dilution_mask(4, n, 3))
    return kw, True


def _oracle_H(kw):
    return O.lattice_hamiltonian(kw["L"], periodic=kw.get("periodic"), onsite=kw.get("onsite"),
                                 hop=kw.get("hop"), t=kw.get("t", 1.0), mask=kw.get("bond_mask"))


def test_small_solve_runs_as_one_launch_and_matches_oracle_and_chain(K):
    # the 2D L=32 FP64 workload (t=1, on-site U[-0.5, 0.5), R=8, M=256)
    w = I.workload("square_L32_fp64")
    kw = dict(dims=2, L=w["L"], onsite=w["onsite"])
    H = _oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R, M, seed = w["R"], w["M"], w["seed"]
    mu_o, per_o = O.moments_doubling(H, a, b, I.rademacher_block(seed, H.n, R), M)
    with colres_env(None):
        with K.kpm_create_stencil(**kw) as h:
            l0 = K.kpm_kernel_launches()
            mu, per = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp64", per_vec=True)
            launches = K.kpm_kernel_launches() - l0
            assert K.kpm_testing_last_step_form(h) == FORM
            again = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp64")   # graph replay
            third = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp64")
    with colres_env("0"):
        with K.kpm_create_stencil(**kw) as h:
            chain = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp64")
            assert K.kpm_testing_last_step_form(h) == "fused step"
    # prescale + one solve launch + the realisation counter + finalisation (2)
    assert launches <= 6
    assert np.abs(per - per_o).max() <= TOL["fp64"]
    assert np.abs(mu - mu_o).max() <= TOL["fp64"]
    assert np.all(per[:, 0] == 1.0)              # mu_0 = 1 exactly for Rademacher vectors
    assert np.array_equal(again, mu) and np.array_equal(third, mu)
    assert np.abs(chain - mu).max() <= 1e-13     # the same recursion, sums in another order


# (C, cpc): one-CTA clusters, several columns per cluster, the non-portable
# 16-CTA cluster, 32 columns per cluster (no lane shuffles), and shapes that
# need more than one wave of clusters
SHAPES = [(1, 1), (2, 4), (4, 2), (8, 1), (16, 1), (16, 4), (4, 32), (2, 16)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("C,cpc", SHAPES)
def test_every_cluster_shape_matches_oracle(K, C, cpc, prec):
    kw, cplx = _ragged()
    H = _oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R, M, seed = 13, 66, 21                      # 13 columns: the last group is part padding
    mu_o, per_o = O.moments_doubling(H, a, b, I.random_block(seed, H.n, R, cplx), M)
    with colres_env(f"{C},{cpc}"):
        with K.kpm_create_stencil(complex_=cplx, **kw) as h:
            mu, per = K.kpm_moments(h, M, R, a, b, seed=seed, precision=prec, per_vec=True)
            assert K.kpm_testing_last_step_form(h) == FORM
    assert np.abs(per - per_o).max() <= TOL[prec]
    assert np.abs(mu - mu_o).max() <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("complex_", [False, True])
def test_open_chain_with_idle_ctas(K, complex_, prec):
    # 5 sites over 16 CTAs: one row per CTA, eleven CTAs hold no row but take
    # part in every cluster barrier
    hop = None
    if complex_:
        hop = np.exp(1j * np.array([0.3, -1.1, 2.0, 0.7, 0.0])).reshape(5, 1)
    kw = dict(dims=1, L=(5,), periodic=(False,), t=0.9, onsite=I.onsite_disorder(3, 5, 1.0))
    if hop is not None:
        kw["hop"] = hop
    H = _oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R, M = 3, 40
    mu_o, _ = O.moments_doubling(H, a, b, I.random_block(2, H.n, R, complex_), M)
    with colres_env("16,1"):
        with K.kpm_create_stencil(complex_=complex_, **kw) as h:
            mu = K.kpm_moments(h, M, R, a, b, seed=2, precision=prec)
            assert K.kpm_testing_last_step_form(h) == FORM
    assert np.abs(mu - mu_o).max() <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_realisations_and_first_realisation_index(K, prec):
    kw, cplx = _ragged()
    H = _oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R, M, seed = 6, 48, 9
    union = np.concatenate([I.random_block(seed, H.n, R, cplx, s=s) for s in range(3)], axis=1)
    mu_o, per_o = O.moments_doubling(H, a, b, union, M)
    with colres_env(None):
        with K.kpm_create_stencil(complex_=cplx, **kw) as h:
            mu, per = K.kpm_moments(h, M, R, a, b, seed=seed, S=3, precision=prec, per_vec=True)
            assert K.kpm_testing_last_step_form(h) == FORM
            _, per2 = K.kpm_moments(h, M, R, a, b, seed=seed, S=1, s0=2, precision=prec,
                                    per_vec=True)
    assert np.abs(per - per_o).max() <= TOL[prec]
    assert np.abs(mu - mu_o).max() <= TOL[prec]
    assert np.array_equal(per2, per[2 * R:3 * R])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_continued_solve_equals_one_call(K, prec):
    # kpm_moments_extend continues from v_{n-1}, v_n in global memory with the
    # same per-product arithmetic and sum order: bit for bit one call
    kw, cplx = _ragged()
    H = _oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R, chain = 7, (40, 42, 300)
    with colres_env(None):
        with K.kpm_create_stencil(complex_=cplx, **kw) as h:
            direct, pv_direct = K.kpm_moments(h, chain[-1], R, a, b, seed=4, precision=prec,
                                              per_vec=True)
            assert K.kpm_testing_last_step_form(h) == FORM
            K.kpm_moments(h, chain[0], R, a, b, seed=4, precision=prec)
            for m in chain[1:]:
                mu, pv = K.kpm_moments_extend(h, m, R=R, per_vec=True)
    assert np.array_equal(mu, direct)
    assert np.array_equal(pv, pv_direct)
    mu_o, _ = O.moments_doubling(H, a, b, I.random_block(4, H.n, R, cplx), chain[-1])
    assert np.abs(mu - mu_o).max() <= TOL[prec]


def test_device_start_block_local_moments(K):
    # unit-vector start columns written on the device, loaded by the solve
    kw, cplx = _ragged()
    H = _oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    sites = [0, 52, 104, 52]
    with colres_env(None):
        with K.kpm_create_stencil(complex_=cplx, **kw) as h:
            got = K.kpm_ldos_moments(h, sites, 80, a, b, precision="fp64")
            assert K.kpm_testing_last_step_form(h) == FORM
    assert np.abs(got - O.ldos_exact(H, a, b, sites, 80)).max() <= TOL["fp64"]


def _csr_handle(K, kw, cplx):
    rp, col, val = K.kpm_stencil_to_csr(complex_=cplx, **kw)
    return K.kpm_create_csr(rp.size - 1, rp, col, val, complex_=cplx)


def test_csr_small_solve_matches_oracle_and_chain(K):
    # the 2D L=32 FP64 workload as a CSR matrix (5 entries per row: a padded
    # ELL of width 6)
    w = I.workload("square_L32_fp64")
    kw = dict(dims=2, L=w["L"], onsite=w["onsite"])
    H = _oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R, M, seed = w["R"], w["M"], w["seed"]
    mu_o, per_o = O.moments_doubling(H, a, b, I.rademacher_block(seed, H.n, R), M)
    with colres_env(None):
        with _csr_handle(K, kw, False) as h:
            mu, per = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp64", per_vec=True)
            assert K.kpm_testing_last_step_form(h) == FORM
            again = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp64")
    with colres_env("0"):
        with _csr_handle(K, kw, False) as h:
            chain = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp64")
            assert K.kpm_testing_last_step_form(h) == "fused step"
    assert np.abs(per - per_o).max() <= TOL["fp64"]
    assert np.abs(mu - mu_o).max() <= TOL["fp64"]
    assert np.array_equal(again, mu)
    assert np.abs(chain - mu).max() <= 1e-13


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("C,cpc", [(1, 1), (4, 2), (16, 1), (16, 4), (4, 32)])
def test_csr_every_cluster_shape_matches_oracle(K, C, cpc, prec):
    # complex spin hoppings, open edge, dilution, disorder: rows of up to 7
    # entries in a padded ELL of width 8
    kw, cplx = _ragged()
    H = _oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R, M, seed = 13, 66, 21
    mu_o, per_o = O.moments_doubling(H, a, b, I.random_block(seed, H.n, R, cplx), M)
    with colres_env(f"{C},{cpc}"):
        with _csr_handle(K, kw, cplx) as h:
            mu, per = K.kpm_moments(h, M, R, a, b, seed=seed, precision=prec, per_vec=True)
            assert K.kpm_testing_last_step_form(h) == FORM
    assert np.abs(per - per_o).max() <= TOL[prec]
    assert np.abs(mu - mu_o).max() <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_csr_continued_solve_equals_one_call(K, prec):
    kw = dict(dims=1, L=(37,), periodic=(False,), t=0.7)      # padded ELL of width 2
    H = _oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R, chain = 5, (40, 42, 300)
    with colres_env(None):
        with _csr_handle(K, kw, False) as h:
            direct = K.kpm_moments(h, chain[-1], R, a, b, seed=4, precision=prec)
            assert K.kpm_testing_last_step_form(h) == FORM
            K.kpm_moments(h, chain[0], R, a, b, seed=4, precision=prec)
            for m in chain[1:]:
                mu = K.kpm_moments_extend(h, m)
    assert np.array_equal(mu, direct)
    mu_o, _ = O.moments_doubling(H, a, b, I.rademacher_block(4, H.n, R), chain[-1])
    assert np.abs(mu - mu_o).max() <= TOL[prec]


@pytest.mark.parametrize("case,form", [
    # 2D L=64 real FP64, R=8: 256 elements per CTA with the bulk dot sums
    # (measured 1.84 us per product against 2.91-3.09 for the step chain)
    (("square", 64, False, 8, "fp64"), FORM),
    # 2D L=80 real FP64, R=8: 400 elements per CTA, bulk sums in 160 KB
    # batches (measured 3.01 us per product against 3.87 for the step chain)
    (("square", 80, False, 8, "fp64"), FORM),
    # complex FP64 3D L=16, R=16 (measured 7.81 against 7.27)
    (("cube", 16, True, 16, "fp64"), "fused step"),
    # FP32 2D L=96, R=16: 576 elements per CTA (4.58 against 3.31)
    (("square", 96, False, 16, "fp32"), "fused step"),
    # FP32 2D L=128, R=32: more elements per CTA than one per thread at one wave
    (("square", 128, False, 32, "fp32"), "fused step")])
def test_planner_takes_the_faster_form(K, case, form):
    kind, L, cplx, R, prec = case
    if kind == "square":
        kw = dict(dims=2, L=(L, L), onsite=I.onsite_disorder(1, L * L, 1.0))
    else:
        kw = dict(dims=3, L=(L, L, L), hop=I.spin_hoppings((L, L, L), *I.spins(2, L ** 3)))
    with colres_env(None):
        with K.kpm_create_stencil(complex_=cplx, **kw) as h:
            K.kpm_moments(h, 8, R, 12.0, 0.0, seed=1, precision=prec)
            assert K.kpm_testing_last_step_form(h) == form
