"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Tolerances: |d mu_n| <= 1e-10 on
the FP64 path, <= 1e-5 on the FP32-vector / FP64-moment path."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def make_case(name):
    """(oracle CSR, kwargs of the library's stencil handle, complex?)"""
    if name == "square_L32":          # the 2D L=32 FP64 workload (disorder W=1, t=1)
        w = I.workload("square_L32_fp64")
        kw = dict(dims=2, L=w["L"], onsite=w["onsite"])
        return kw, False
    if name == "cube_spin_L8":        # 3D spin hoppings, scaled-down cubic workload
        L = (8, 8, 8)
        kw = dict(dims=3, L=L, hop=I.spin_hoppings(L, *I.spins(2, 512)))
        return kw, True
    if name == "ragged_open_mask":    # odd sizes, one open dimension, dilution and disorder
        L = (5, 3, 7)
        N = 105
        kw = dict(dims=3, L=L, periodic=(True, False, True), onsite=I.onsite_disorder(4, N, 2.0),
                  hop=I.spin_hoppings(L, *I.spins(4, N)), bond_mask=I.dilution_mask(4, N, 3))
        return kw, True
    if name == "degenerate_dims":     # L=2 and L=1 wraps
        L = (2, 1, 9)
        kw = dict(dims=3, L=L, onsite=I.onsite_disorder(5, 18, 1.0))
        return kw, False
    if name == "chain_open":
        kw = dict(dims=1, L=(37,), periodic=(False,), t=0.7)
        return kw, False
    raise KeyError(name)


def oracle_H(kw):
    return O.lattice_hamiltonian(kw["L"], periodic=kw.get("periodic"), onsite=kw.get("onsite"),
                                 hop=kw.get("hop"), t=kw.get("t", 1.0), mask=kw.get("bond_mask"))


def handle(K, kw, cplx, csr=False):
    if not csr:
        return K.kpm_create_stencil(complex_=cplx, **kw)
    rp, col, val = K.kpm_stencil_to_csr(complex_=cplx, **kw)
    return K.kpm_create_csr(rp.size - 1, rp, col, val, complex_=cplx)


@pytest.fixture(scope="module")
def K(gpu_lib):
    from paper_1105_5481_gb300 import kpm

    return kpm


CASES = ["square_L32", "cube_spin_L8", "ragged_open_mask", "degenerate_dims", "chain_open"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("csr", [False, True], ids=["stencil", "csr"])
@pytest.mark.parametrize("name", CASES)
def test_moments_match_oracle(K, name, csr, prec):
    kw, cplx = make_case(name)
    H = oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R = {"square_L32": 8, "cube_spin_L8": 64}.get(name, 5)
    M = 256 if name in ("square_L32", "cube_spin_L8") else 66
    seed = 11
    v0 = I.random_block(seed, H.n, R, cplx)
    mu_o, per_o = O.moments_doubling(H, a, b, v0, M)
    with handle(K, kw, cplx, csr) as h:
        assert K.kpm_info(h)["nnz"] == H.nnz      # stored entries of H (closed form or count)
        mu, per = K.kpm_moments(h, M, R, a, b, seed=seed, precision=prec, per_vec=True)
    tol = TOL[prec]
    assert np.abs(per - per_o).max() <= tol
    assert np.abs(mu - mu_o).max() <= tol
    if prec == "fp64" and not cplx:
        assert np.all(per[:, 0] == 1.0)     # mu_0 = 1 exactly for Rademacher vectors


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_user_v0_full_basis_gives_exact_trace(K, prec):
    kw, cplx = make_case("ragged_open_mask")
    H = oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    M = 128
    ex = O.exact_moments(H, a, b, M)
    v0 = math.sqrt(H.n) * np.eye(H.n)
    with handle(K, kw, cplx) as h:
        mu = K.kpm_moments(h, M, H.n, a, b, precision=prec, user_v0=v0.astype(np.complex128))
    assert np.abs(mu - ex).max() <= TOL[prec]


def test_paper_cube_full_basis_matches_golden(K):
    from test_golden import load_cubic10

    a, b, gold = load_cubic10()
    with K.kpm_create_stencil(3, (10, 10, 10), onsite=np.zeros(1000)) as h:
        mu = K.kpm_moments(h, 512, 1000, a, b, user_v0=math.sqrt(1000) * np.eye(1000))
    assert np.abs(mu - gold).max() <= 1e-10


def test_realisations_equal_wider_block(K):
    kw, cplx = make_case("cube_spin_L8")
    with handle(K, kw, cplx) as h:
        m3, p3 = K.kpm_moments(h, 64, 4, 6.1, 0.0, seed=5, S=3, per_vec=True)
        m1, p1 = K.kpm_moments(h, 64, 12, 6.1, 0.0, seed=5, S=1, per_vec=True)
    assert np.abs(p3 - p1).max() < 1e-13 and np.abs(m3 - m1).max() < 1e-13


def test_repeat_call_is_bitwise_identical(K):
    kw, cplx = make_case("cube_spin_L8")
    with handle(K, kw, cplx) as h:
        for prec in ("fp64", "fp32"):
            m1 = K.kpm_moments(h, 128, 64, 6.1, 0.1, seed=9, precision=prec)
            m2 = K.kpm_moments(h, 128, 64, 6.1, 0.1, seed=9, precision=prec)
            assert np.array_equal(m1, m2)


@pytest.mark.parametrize("M,R,L", [(2, 1, (1,)), (2, 3, (4,)), (4, 1, (3, 3))])
def test_tiny_edge_cases(K, M, R, L):
    kw = dict(dims=len(L), L=L, onsite=I.onsite_disorder(2, int(np.prod(L)), 1.0))
    H = oracle_H(kw)
    gmin, gmax = O.gershgorin(H)
    a, b = max(gmax - gmin, 1.0), 0.5 * (gmax + gmin)   # a 1-site lattice has gmin == gmax
    mu_o, _ = O.moments_doubling(H, a, b, I.rademacher_block(3, H.n, R), M)
    with K.kpm_create_stencil(**kw) as h:
        mu = K.kpm_moments(h, M, R, a, b, seed=3)
    assert np.abs(mu - mu_o).max() <= 1e-12


def test_bounds_that_miss_the_spectrum_report_divergence(K):
    kw, cplx = make_case("square_L32")
    with handle(K, kw, cplx) as h:
        with pytest.raises(K.KPMError) as e:
            K.kpm_moments(h, 256, 8, 1.0, 0.0, seed=1)
        assert e.value.status == K.KPM_EDIVERGE
        with pytest.raises(K.KPMError) as e:
            K.kpm_moments(h, 7, 8, 5.0, 0.0)
        assert e.value.status == K.KPM_EINVAL


@pytest.mark.parametrize("name", ["square_L32", "cube_spin_L8", "ragged_open_mask", "degenerate_dims"])
@pytest.mark.parametrize("csr", [False, True], ids=["stencil", "csr"])
def test_bounds_match_oracle(K, name, csr):
    kw, cplx = make_case(name)
    H = oracle_H(kw)
    gmin, gmax = O.gershgorin(H)
    with handle(K, kw, cplx, csr) as h:
        e0 = K.kpm_bounds(h, 0, 0.0)
        assert abs(e0[0] - gmin) <= 1e-13 * (gmax - gmin) and abs(e0[1] - gmax) <= 1e-13 * (gmax - gmin)
        assert e0[2] == pytest.approx((gmax - gmin) / 2, rel=1e-15)
        k = min(30, H.n)
        emin, emax, a, b = K.kpm_bounds(h, k, 0.01, seed=6)
    omin, omax, _ = O.lanczos_bounds(H, k, I.lanczos_start(6, H.n))
    span = gmax - gmin
    assert abs(emin - omin) <= 1e-8 * span and abs(emax - omax) <= 1e-8 * span
    lam = np.linalg.eigvalsh(O.dense(H))
    assert emin <= lam[0] + 1e-9 * span and emax >= lam[-1] - 1e-9 * span
    oa, ob = O.rescale(omin, omax, 0.01)
    assert abs(a - oa) <= 1e-8 * span and abs(b - ob) <= 1e-8 * span


# node counts from 5 to 25000: the DCT gives each node 32, 16, 8, 4, 2 or 1
# lanes (the fewer the more nodes), each case against the oracle's sum
@pytest.mark.parametrize("kernel", ["jackson", "none"])
@pytest.mark.parametrize("M,K_", [(256, 1024), (37, 64), (1, 5), (1000, 999), (300, 1500),
                                  (2048, 4096), (700, 6000), (128, 12000), (64, 25000)])
def test_dos_matches_oracle(K, kernel, M, K_):
    rng = np.random.default_rng(M)
    mu = rng.uniform(-1, 1, M) * np.exp(-np.arange(M) / 50.0)
    mu[0] = 1.0
    a, b = 3.7, -0.2
    E_o, rho_o = O.dos(mu, a, b, K_, kernel)
    E, rho = K.kpm_dos(mu, a, b, K_, kernel)
    np.testing.assert_allclose(E, E_o, rtol=0, atol=1e-14 * a)
    # the oracle's sqrt(1 - x_k^2) carries a relative rounding error ~ eps / (1 - x_k^2)
    x = (E_o - b) / a
    tol = 1e-12 * np.abs(rho_o).max() + 1e-15 * np.abs(rho_o) / (1.0 - x * x)
    assert np.all(np.abs(rho - rho_o) <= tol)


def test_dos_device_buffers(K):
    import torch

    mu = torch.zeros(64, dtype=torch.float64, device="cuda")
    mu[0] = 1.0
    E = torch.empty(128, dtype=torch.float64, device="cuda")
    rho = torch.empty(128, dtype=torch.float64, device="cuda")
    K.kpm_dos(mu, 2.0, 0.0, 128, "jackson", E=E, rho=rho)
    torch.cuda.synchronize()
    E_o, rho_o = O.dos(mu.cpu().numpy(), 2.0, 0.0, 128)
    assert np.abs(rho.cpu().numpy() - rho_o).max() <= 1e-12 * np.abs(rho_o).max()


def random_hermitian_csr(n, seed, max_row=20):
    """Sparse Hermitian matrix with rows of very different lengths (generic CSR path)."""
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        k = int(rng.integers(0, max_row // 2))
        js = rng.choice(n, size=k, replace=False)
        A[i, js] += rng.normal(size=k) + 1j * rng.normal(size=k)
    A = A + A.conj().T + np.diag(rng.normal(size=n))
    rows, cols = np.nonzero(A)
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int32), A[rows, cols]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_generic_csr_long_rows_match_oracle(K, prec):
    n, R, M = 300, 6, 96
    rp, col, val = random_hermitian_csr(n, 3)
    assert np.diff(rp).max() > 8            # too long for the padded-ELL layout
    H = O.CSR(n, rp, col, val)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    mu_o, per_o = O.moments_doubling(H, a, b, I.random_block(5, n, R, True), M)
    with K.kpm_create_csr(n, rp, col, val, complex_=True) as h:
        mu, per = K.kpm_moments(h, M, R, a, b, seed=5, precision=prec, per_vec=True)
    assert np.abs(per - per_o).max() <= TOL[prec]


# the widest vector blocks one fused step takes (1024 chunks per row: four
# column blocks of 256 chunks in the grid's y dimension), and one beyond
@pytest.mark.parametrize("prec,cplx,R", [("fp64", True, 1024), ("fp32", False, 8192),
                                         ("fp32", True, 4096)])
def test_widest_vector_block_matches_oracle(K, prec, cplx, R):
    L = (6, 5, 7)
    N = 210
    kw = dict(dims=3, L=L, onsite=I.onsite_disorder(8, N, 1.0))
    if cplx:
        kw["hop"] = I.spin_hoppings(L, *I.spins(8, N))
    H = oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    M, seed = 24, 13
    mu_o, per_o = O.moments_doubling(H, a, b, I.random_block(seed, N, R, cplx), M)
    with handle(K, kw, cplx) as h:
        mu, per = K.kpm_moments(h, M, R, a, b, seed=seed, precision=prec, per_vec=True)
        with pytest.raises(K.KPMError) as e:
            K.kpm_moments(h, M, R + 1, a, b, seed=seed, precision=prec)
        assert e.value.status == K.KPM_EINVAL
    assert np.abs(per - per_o).max() <= TOL[prec]
    assert np.abs(mu - mu_o).max() <= TOL[prec]


# ---------------------------------------------------------------- checkpoint / resume
# kpm_moments_extend continues the last single-realisation call on a handle;
# the moments equal those of one uninterrupted call bit for bit, because the
# same launches run in the same order from the kept v_{n-1}, v_n and sums.


@pytest.mark.parametrize("name,prec,csr,chain",
                         [("square_L32", "fp64", False, (256, 512)),
                          ("cube_spin_L8", "fp32", False, (128, 256, 1024)),
                          ("ragged_open_mask", "fp64", True, (40, 42, 300))])
def test_extend_equals_one_call(K, name, prec, csr, chain):
    kw, cplx = make_case(name)
    H = oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R, M = 8, chain[-1]
    with handle(K, kw, cplx, csr) as h:
        direct, pv_direct = K.kpm_moments(h, M, R, a, b, seed=7, precision=prec, per_vec=True)
        K.kpm_moments(h, chain[0], R, a, b, seed=7, precision=prec)
        for m in chain[1:]:
            mu, pv = K.kpm_moments_extend(h, m, R=R, per_vec=True)
        again = K.kpm_moments(h, M, R, a, b, seed=7, precision=prec)  # the handle rebuilds cleanly
    assert np.array_equal(mu, direct)
    assert np.array_equal(pv, pv_direct)
    assert np.array_equal(again, direct)
    v0 = (I.phase_block if cplx else I.rademacher_block)(7, H.n, R)
    mu_o, _ = O.moments_doubling(H, a, b, v0, M)
    assert np.abs(mu - mu_o).max() <= TOL[prec]


def test_extend_refusals(K):
    kw, cplx = make_case("chain_open")
    H = oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    with handle(K, kw, cplx) as h:
        with pytest.raises(K.KPMError) as e:
            K.kpm_moments_extend(h, 64)                     # no call to resume yet
        assert e.value.status == K.KPM_ENOTREADY
        K.kpm_moments(h, 64, 4, a, b, seed=1, S=2)           # two realisations: not resumable
        with pytest.raises(K.KPMError) as e:
            K.kpm_moments_extend(h, 128)
        assert e.value.status == K.KPM_ENOTREADY
        K.kpm_moments(h, 64, 4, a, b, seed=1)
        for bad in (64, 62, 97):                             # not larger, or odd
            with pytest.raises(K.KPMError) as e:
                K.kpm_moments_extend(h, bad)
            assert e.value.status == K.KPM_EINVAL
        mu = K.kpm_moments_extend(h, 256)                    # grows the per-step sums
    mu_o, _ = O.moments_doubling(H, a, b, I.rademacher_block(1, H.n, 4), 256)
    assert np.abs(mu - mu_o).max() <= 1e-10


@pytest.mark.parametrize("fail_after", [0, 1])
def test_extend_failing_part_way_leaves_nothing_to_resume(K, fail_after):
    # An extend that runs out of device memory after it has started replacing
    # buffers (fail_after = 1: the per-step sums grow, then the per-vector
    # moments cannot) must leave no state behind: a second extend has nothing
    # to resume, and the next kpm_moments rebuilds its plan instead of
    # replaying a graph that points at freed memory.
    kw, cplx = make_case("square_L32")
    H = oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R = 8
    with handle(K, kw, cplx) as h:
        first = K.kpm_moments(h, 64, R, a, b, seed=3)
        K.kpm_moments(h, 64, R, a, b, seed=3)               # second call: captured graph
        K.kpm_testing_fail_allocations(fail_after)
        try:
            with pytest.raises(K.KPMError) as e:
                K.kpm_moments_extend(h, 128)
            assert e.value.status == K.KPM_ENOMEM
        finally:
            K.kpm_testing_fail_allocations(-1)
        with pytest.raises(K.KPMError) as e:
            K.kpm_moments_extend(h, 128)
        assert e.value.status == K.KPM_ENOTREADY
        again = K.kpm_moments(h, 64, R, a, b, seed=3)
        longer = K.kpm_moments(h, 128, R, a, b, seed=3)
        resumed = K.kpm_moments_extend(h, 256)             # resumable again after a full call
    assert np.array_equal(again, first)
    mu_o, _ = O.moments_doubling(H, a, b, I.rademacher_block(3, H.n, R), 256)
    assert np.abs(longer - mu_o[:128]).max() <= TOL["fp64"]
    assert np.abs(resumed - mu_o).max() <= TOL["fp64"]
