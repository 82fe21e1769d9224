"""GPU parity of the paper's dense formulation (every element of H takes part in
every product, FP64): moments against the FP64 oracle (|d mu_n| <= 1e-10),
the paper's 10x10x10 cube stored dense against its golden exact moments, the
bounds against the oracle's Gershgorin and Lanczos, the matrix sizes the
paper sweeps at full size (sampled columns), and the refusals."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def K(gpu_lib):
    from paper_1105_5481_gb300 import kpm

    return kpm


# n not a multiple of the 16/64-row tiles or of the 16-wide k slices; complex;
# a 1 x 1 matrix; more vectors than one block of the sparse path (odd R)
@pytest.mark.parametrize("n,complex_,R", [(200, False, 16), (97, False, 5), (150, True, 8),
                                          (1, False, 3), (130, True, 40), (70, False, 2101)])
def test_dense_moments_match_oracle(K, n, complex_, R):
    A = I.dense_hermitian(40 + n, n, complex_)
    H = O.from_dense(A)
    gmin, gmax = O.gershgorin(H)
    a, b = (O.rescale(gmin, gmax, 0.01) if n > 1 else (1.0, float(A[0, 0].real)))
    M, seed = 66, 17
    mu_o, per_o = O.moments_doubling(H, a, b, I.random_block(seed, n, R, complex_), M)
    with K.kpm_create_dense(A) as h:
        info = K.kpm_info(h)
        assert info["nnz"] == n * n and not info["stencil"] and info["complex"] == complex_
        mu, per = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp64", per_vec=True)
    assert np.abs(per - per_o).max() <= TOL
    assert np.abs(mu - mu_o).max() <= TOL


def test_dense_full_basis_gives_exact_trace(K):
    A = I.dense_hermitian(5, 120, True)
    H = O.from_dense(A)
    a, b = O.rescale(*O.gershgorin(H), 0.01)
    M = 128
    ex = O.exact_moments(H, a, b, M)
    with K.kpm_create_dense(A) as h:
        mu = K.kpm_moments(h, M, 120, a, b, user_v0=math.sqrt(120) * np.eye(120, dtype=np.complex128))
    assert np.abs(mu - ex).max() <= TOL


def test_paper_cube_stored_dense_matches_golden(K):
    # the paper's evaluation lattice (Sec. IV-A) in the paper's own dense form:
    # D = 1000, every row with 7 nonzeros among 1000 stored elements
    from test_golden import load_cubic10

    a, b, gold = load_cubic10()
    A = O.dense(O.lattice_hamiltonian((10, 10, 10)))
    with K.kpm_create_dense(A) as h:
        mu = K.kpm_moments(h, 512, 1000, a, b, user_v0=math.sqrt(1000) * np.eye(1000))
    assert np.abs(mu - gold).max() <= TOL


@pytest.mark.parametrize("complex_", [False, True])
def test_dense_bounds_match_oracle(K, complex_):
    n = 180
    A = I.dense_hermitian(12, n, complex_)
    H = O.from_dense(A)
    gmin, gmax = O.gershgorin(H)
    span = gmax - gmin
    with K.kpm_create_dense(A) as h:
        e0 = K.kpm_bounds(h, 0, 0.0)
        assert abs(e0[0] - gmin) <= 1e-13 * span and abs(e0[1] - gmax) <= 1e-13 * span
        emin, emax, a, b = K.kpm_bounds(h, 30, 0.01, seed=6)
    omin, omax, _ = O.lanczos_bounds(H, 30, I.lanczos_start(6, n))
    assert abs(emin - omin) <= 1e-8 * span and abs(emax - omax) <= 1e-8 * span
    lam = np.linalg.eigvalsh(A)
    assert emin <= lam[0] + 1e-9 * span and emax >= lam[-1] - 1e-9 * span


def test_dense_repeat_calls_and_realisations(K):
    A = I.dense_hermitian(6, 160)
    H = O.from_dense(A)
    a, b = O.rescale(*O.gershgorin(H), 0.01)
    R, S, M, seed = 8, 3, 64, 4
    mu_o, _ = O.moments_doubling(H, a, b, I.random_block(seed, 160, R * S, False), M)
    with K.kpm_create_dense(A) as h:
        runs = [K.kpm_moments(h, M, R, a, b, seed=seed, S=S) for _ in range(3)]
    assert np.abs(runs[0] - mu_o).max() <= TOL
    assert np.array_equal(runs[0], runs[1]) and np.array_equal(runs[1], runs[2])


def test_dense_refusals(K):
    A = I.dense_hermitian(7, 40)
    with pytest.raises(K.KPMError) as e:
        K.kpm_create_dense(A + np.triu(np.full((40, 40), 1e-3), 1))
    assert e.value.status == K.KPM_EINVAL
    with K.kpm_create_dense(A) as h:
        with pytest.raises(K.KPMError) as e:
            K.kpm_moments(h, 64, 8, 2.0, 0.0, precision="fp32")
        assert e.value.status == K.KPM_EINVAL
        with pytest.raises(K.KPMError) as e:
            K.kpm_moments(h, 64, 8, 0.5, 0.0, seed=1)      # bounds miss the spectrum
        assert e.value.status == K.KPM_EDIVERGE


@pytest.mark.parametrize("D", [512, 4096])
def test_dense_paper_sizes_sampled_columns(K, D):
    # the paper's matrix-size sweep (Sec. IV-C: H_SIZE up to 4096, N = 128
    # moments, R x S = 1792 vectors) as the benchmark runs it: one block of
    # 1792 real vectors; the oracle recomputes two sampled columns
    w = I.workload(f"dense_wigner_D{D}")
    A, R, M = w["H"], w["R"], w["M"]
    H = O.from_dense(A)
    omin, omax, _ = O.lanczos_bounds(H, 30, I.lanczos_start(6, D))
    a, b = O.rescale(omin, omax, 0.01)
    cols = [0, R - 1]
    seed = 21
    v0 = I.random_columns(seed, D, R, cols, False)
    _, per_o = O.moments_doubling(H, a, b, v0, M)
    with K.kpm_create_dense(A) as h:
        mu, per = K.kpm_moments(h, M, R, a, b, seed=seed, per_vec=True)
    assert np.abs(per[cols] - per_o).max() <= TOL
    assert np.abs(per[:, 0] - 1.0).max() <= 1e-14
    # Wigner's semicircle of radius 2/sqrt(3): mu_2 = r^2/2 - 1 with r = radius / a,
    # up to finite-size and stochastic deviations
    r = 2.0 / math.sqrt(3.0) / a
    assert abs(mu[2] - (r * r / 2.0 - 1.0)) < 0.02
