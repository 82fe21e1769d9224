"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks re-uses an oracle formula: they compare it with closed
forms (plane-wave spectra, low-order traces), with library routines
(numpy.linalg.eigvalsh, numpy.polynomial.chebyshev) and with brute force.
"""
import math

import numpy as np
import numpy.polynomial.chebyshev as C
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def plane_wave_spectrum(L, t=1.0):
    """Clean periodic hypercubic lattice: E(m) = -2 t sum_d cos(2 pi m_d / L_d)."""
    grids = np.meshgrid(*[np.cos(2 * np.pi * np.arange(l) / l) for l in L], indexing="ij")
    return np.sort((-2.0 * t * sum(grids)).ravel())


def full_basis(N):
    # unit vectors scaled to the random vectors' norm (|r|^2 = N, Sec. II-A-3)
    return math.sqrt(N) * np.eye(N)


def cheb_T(n, x):
    return C.chebval(x, np.eye(n + 1)[n])


# ---------------------------------------------------------------- lattice (a1)

def test_paper_cube_has_seven_entries_per_row():
    # Sec. IV-A: 10x10x10 lattice, symmetric, every row seven entries, zero diagonal, -1 elsewhere
    H = O.lattice_hamiltonian((10, 10, 10), onsite=np.zeros(1000))
    A = O.dense(H)
    assert H.n == 1000
    assert np.all(np.diff(H.rowptr) == 7)
    assert np.all(np.diag(A) == 0.0)
    off = A[~np.eye(1000, dtype=bool)]
    assert np.count_nonzero(off) == 6000 and set(np.unique(off[off != 0])) == {-1.0}
    assert np.array_equal(A, A.T)


@pytest.mark.parametrize("L", [(7,), (2,), (1,), (4, 6), (3, 4, 5), (2, 3, 2)])
def test_clean_lattice_spectrum_is_plane_waves(L):
    H = O.lattice_hamiltonian(L)
    lam = np.linalg.eigvalsh(O.dense(H))
    np.testing.assert_allclose(lam, plane_wave_spectrum(L), atol=1e-12)


def test_open_chain_spectrum():
    L = 9
    H = O.lattice_hamiltonian((L,), periodic=(False,))
    lam = np.linalg.eigvalsh(O.dense(H))
    expect = np.sort(-2.0 * np.cos(np.pi * np.arange(1, L + 1) / (L + 1)))
    np.testing.assert_allclose(lam, expect, atol=1e-12)


def test_parallel_spins_reduce_to_clean_lattice():
    L = (4, 4, 4)
    N = 64
    hop = I.spin_hoppings(L, np.full(N, 0.7), np.full(N, 1.3))
    np.testing.assert_allclose(hop, 1.0 + 0j, atol=1e-15)
    H = O.lattice_hamiltonian(L, hop=hop)
    np.testing.assert_allclose(np.linalg.eigvalsh(O.dense(H)), plane_wave_spectrum(L), atol=1e-12)


def test_spin_hamiltonian_is_hermitian_with_bounded_hoppings():
    w = I.workload("cubic_spin_L4")
    H = O.lattice_hamiltonian(w["L"], hop=w["hop"], mask=I.dilution_mask(4, 64, 3))
    A = O.dense(H)
    assert np.abs(A - A.conj().T).max() == 0.0
    assert np.abs(w["hop"]).max() <= 1.0 + 1e-15


# ---------------------------------------------------------------- bounds (a2)

def _test_matrices():
    w = I.workload("cubic_spin_L4")
    yield O.lattice_hamiltonian(w["L"], hop=w["hop"])
    yield O.lattice_hamiltonian((6, 5), onsite=I.onsite_disorder(3, 30, 4.0))
    yield O.lattice_hamiltonian((5, 4, 3), periodic=(True, False, True), hop=I.spin_hoppings(
        (5, 4, 3), *I.spins(9, 60)), mask=I.dilution_mask(9, 60, 3), onsite=I.onsite_disorder(9, 60, 1.0))


def test_gershgorin_clean_chain_is_pm2():
    assert O.gershgorin(O.lattice_hamiltonian((11,))) == (-2.0, 2.0)


@pytest.mark.parametrize("H", list(_test_matrices()), ids=["spin3d", "dis2d", "mixed3d"])
def test_bounds_enclose_spectrum(H):
    lam = np.linalg.eigvalsh(O.dense(H))
    gmin, gmax = O.gershgorin(H)
    assert gmin <= lam[0] + 1e-12 and lam[-1] <= gmax + 1e-12   # Gershgorin circle theorem
    start = I.lanczos_start(6, H.n)
    emin, emax, info = O.lanczos_bounds(H, 30, start)
    # Cauchy interlacing: Ritz values lie inside the spectrum
    assert lam[0] - 1e-10 <= info["theta_min"] and info["theta_max"] <= lam[-1] + 1e-10
    assert gmin <= emin <= lam[0] + 1e-9 and lam[-1] - 1e-9 <= emax <= gmax
    # full Krylov space: Lanczos is exact
    emin, emax, info = O.lanczos_bounds(H, H.n, start)
    assert abs(info["theta_min"] - lam[0]) < 1e-10 and abs(info["theta_max"] - lam[-1]) < 1e-10


def test_rescale_maps_bounds_inside_unit_interval():
    a, b = O.rescale(-3.0, 5.0, eps=0.0)
    assert (a, b) == (4.0, 1.0)
    a, b = O.rescale(-3.0, 5.0, eps=0.01)
    assert abs((5.0 - b) / a - (1.0 - 0.005)) < 1e-15 and abs((-3.0 - b) / a + (1.0 - 0.005)) < 1e-15


# ---------------------------------------------------------------- moments (a3-a6)

def test_exact_moments_match_library_chebyshev():
    H = O.lattice_hamiltonian((6, 5), onsite=I.onsite_disorder(3, 30, 2.0))
    a, b = O.rescale(*O.gershgorin(H))
    lam = np.linalg.eigvalsh(O.dense(H))
    x = (lam - b) / a
    mu = O.exact_moments(H, a, b, 40)
    expect = np.array([cheb_T(n, x).mean() for n in range(40)])
    np.testing.assert_allclose(mu, expect, atol=1e-12)


def test_low_order_moments_closed_form():
    eps = I.onsite_disorder(5, 24, 3.0)
    hop = I.spin_hoppings((2, 3, 4), *I.spins(5, 24))
    H = O.lattice_hamiltonian((2, 3, 4), periodic=(False, True, True), onsite=eps, hop=hop)
    a, b = 7.5, 0.3
    A = (O.dense(H) - b * np.eye(24)) / a
    mu1 = (eps.mean() - b) / a                                 # Tr H~ / N
    mu2 = 2.0 * np.linalg.norm(A, "fro") ** 2 / 24 - 1.0       # T_2 = 2x^2 - 1
    ex = O.exact_moments(H, a, b, 3)
    dbl, _ = O.moments_doubling(H, a, b, full_basis(24), 4)
    for mu in (ex, dbl):
        assert abs(mu[0] - 1.0) < 1e-14 and abs(mu[1] - mu1) < 1e-14 and abs(mu[2] - mu2) < 1e-13


@pytest.mark.parametrize("H", list(_test_matrices()), ids=["spin3d", "dis2d", "mixed3d"])
def test_full_basis_gives_exact_trace(H):
    # the estimator with the full basis is Tr T_n(H~)/N exactly
    gmin, gmax = O.gershgorin(H)
    a, b = O.rescale(gmin, gmax)
    M = 96
    ex = O.exact_moments(H, a, b, M)
    v0 = full_basis(H.n)
    d, _ = O.moments_direct(H, a, b, v0, M)
    m, _ = O.moments_doubling(H, a, b, v0, M)
    np.testing.assert_allclose(d, ex, atol=1e-12)
    np.testing.assert_allclose(m, ex, atol=1e-12)


@pytest.mark.parametrize("complex_", [False, True])
def test_diagonal_hamiltonian_estimator_is_exact(complex_):
    N, R, M = 50, 3, 64
    eps = I.onsite_disorder(11, N, 3.0)
    H = O.lattice_hamiltonian((N,), onsite=eps, t=0.0)
    a, b = O.rescale(eps.min(), eps.max())
    v0 = I.random_block(11, N, R, complex_)
    mu, per = O.moments_doubling(H, a, b, v0, M)
    x = (eps - b) / a
    expect = np.array([cheb_T(n, x).mean() for n in range(M)])
    np.testing.assert_allclose(mu, expect, atol=1e-13)
    np.testing.assert_allclose(per, np.tile(expect, (R, 1)), atol=1e-13)


def test_doubling_equals_direct_recursion():
    H = O.lattice_hamiltonian((8, 8), onsite=I.onsite_disorder(1, 64, 1.0))
    a, b = O.rescale(*O.gershgorin(H))
    v0 = I.rademacher_block(1, 64, 4)
    d, dp = O.moments_direct(H, a, b, v0, 1024)
    m, mp = O.moments_doubling(H, a, b, v0, 1024)
    assert np.abs(d - m).max() < 1e-11 and np.abs(dp - mp).max() < 1e-11


def test_stochastic_error_bound_and_invariants():
    L = (6, 6, 6)
    N, R, M = 216, 16, 128
    H = O.lattice_hamiltonian(L, hop=I.spin_hoppings(L, *I.spins(2, N)))
    a, b = O.rescale(*O.gershgorin(H))
    ex = O.exact_moments(H, a, b, M)
    for complex_ in (False, True):
        v0 = I.random_block(7, N, R, complex_)
        mu, per = O.moments_doubling(H, a, b, v0, M)
        assert np.abs(mu - ex).max() <= 5.0 * math.sqrt(2.0 / (R * N))
        assert np.abs(per[:, 0] - 1.0).max() < 1e-14            # mu_0 = 1: |xi| = 1
        assert np.abs(per).max() <= 1.0 + 1e-12                   # |T_n| <= 1 on [-1, 1]


def test_bipartite_lattice_has_zero_odd_moments():
    L = (4, 6)
    H = O.lattice_hamiltonian(L, hop=I.spin_hoppings(L, *I.spins(3, 24)))
    a, b = O.rescale(*O.gershgorin(H), eps=0.05)
    b = 0.0
    ex = O.exact_moments(H, a, b, 64)
    assert np.abs(ex[1::2]).max() < 1e-13


# ---------------------------------------------------------------- kernel + DOS (a7-a8)

@pytest.mark.parametrize("M", [2, 17, 256, 1000])
def test_jackson_kernel_is_sine_window_autocorrelation(M):
    # review Eqs. 70-71: g_n = sum_nu a_nu a_{nu+n}, a_nu ~ sin(pi (nu+1)/(M+1)), sum a_nu^2 = 1
    g = O.jackson_kernel(M)
    av = np.sin(np.pi * (np.arange(M) + 1) / (M + 1))
    av /= np.linalg.norm(av)
    expect = np.array([np.dot(av[: M - n], av[n:]) for n in range(M)])
    np.testing.assert_allclose(g, expect, atol=1e-14)
    assert g[0] == pytest.approx(1.0, abs=1e-15)
    assert np.all(g > 0) and np.all(np.diff(g) < 0)


def test_clean_chain_dos_is_arcsine():
    # clean chain, t=1, M <= L: mu = (1,0,0,...), DOS = 1/(pi sqrt(4 t^2 - E^2))
    L, M, K = 300, 256, 512
    H = O.lattice_hamiltonian((L,))
    a, b = O.rescale(*O.gershgorin(H), eps=0.0)
    mu, _ = O.moments_doubling(H, a, b, full_basis(L), M)
    np.testing.assert_allclose(mu, np.eye(M)[0], atol=1e-12)
    E, rho = O.dos(mu, a, b, K)
    np.testing.assert_allclose(rho, 1.0 / (np.pi * np.sqrt(4.0 - E * E)), rtol=1e-12)


def test_dos_matches_library_chebyshev_series():
    rng = np.random.default_rng(0)
    M, K, a, b = 37, 64, 2.5, -0.4
    mu = rng.uniform(-1, 1, M)
    mu[0] = 1.0
    for kernel in ("jackson", "none"):
        g = O.jackson_kernel(M) if kernel == "jackson" else np.ones(M)
        E, rho = O.dos(mu, a, b, K, kernel)
        x = np.cos(np.pi * (np.arange(K) + 0.5) / K)
        c = 2.0 * g * mu
        c[0] = g[0] * mu[0]
        expect = C.chebval(x, c) / (np.pi * np.sqrt(1 - x * x)) / a
        np.testing.assert_allclose(E, a * x + b, atol=1e-15)
        np.testing.assert_allclose(rho, expect, rtol=1e-12, atol=1e-12)


def test_dos_integrates_to_one_and_is_nonnegative():
    H = O.lattice_hamiltonian((6, 5), onsite=I.onsite_disorder(3, 30, 2.0))
    a, b = O.rescale(*O.gershgorin(H))
    M, K = 128, 256
    mu = O.exact_moments(H, a, b, M)
    E, rho = O.dos(mu, a, b, K)
    x = (E - b) / a
    # Gauss-Chebyshev quadrature is exact for polynomials of degree < 2K
    integral = np.sum(np.pi / K * np.sqrt(1 - x * x) * rho * a)
    assert abs(integral - 1.0) < 1e-13
    assert rho.min() > -1e-12                                   # Jackson kernel keeps rho >= 0


# ---------------------------------------------------------------- dense formulation

@pytest.mark.parametrize("complex_", [False, True])
def test_dense_formulation_stores_every_element(complex_):
    A = I.dense_hermitian(4, 37, complex_)
    A[3, 5] = A[5, 3] = 0.0                         # a zero stays a stored element
    H = O.from_dense(A)
    assert H.nnz == 37 * 37
    np.testing.assert_array_equal(O.dense(H), A)
    X = I.random_block(2, 37, 5, complex_)
    np.testing.assert_allclose(H.matvec(X), A @ X, rtol=1e-13, atol=1e-14)
    offdiag = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
    gmin, gmax = O.gershgorin(H)
    assert abs(gmin - np.min(np.diag(A).real - offdiag)) < 1e-13
    assert abs(gmax - np.max(np.diag(A).real + offdiag)) < 1e-13


def test_dense_wigner_moments_follow_the_semicircle():
    # Wigner's semicircle law: entries of variance s^2 = 1/(3n) give a spectrum
    # on [-2/sqrt(3), 2/sqrt(3)] with density (2/pi) sqrt(1 - x^2) in units of
    # the radius, whose Chebyshev moments are 1, 0, -1/2, 0, 0, ...; at n = 400
    # the finite-size deviations are O(1/n) in mu_2 and mu_4.
    n = 400
    A = I.dense_hermitian(9, n)
    a = 2.0 / math.sqrt(3.0)
    mu = O.exact_moments(O.from_dense(A), a, 0.0, 8)
    assert abs(mu[0] - 1.0) < 1e-14
    assert abs(mu[2] + 0.5) < 0.02 and abs(mu[4]) < 0.03 and abs(mu[6]) < 0.03
    assert abs(mu[1]) < 0.01 and abs(mu[3]) < 0.01
    # mu_2 exactly: 2 ||H~||_F^2 / n - 1
    assert abs(mu[2] - (2.0 * np.linalg.norm(A / a, "fro") ** 2 / n - 1.0)) < 1e-12


@pytest.mark.parametrize("M", [128, 256, 512])
def test_jackson_broadens_a_level_to_width_pi_over_M(M):
    # the Jackson-damped series of one level at x0 = 0 (mu_n = T_n(0)) is a
    # near-Gaussian of standard deviation pi/M (the KPM review's resolution of
    # the Jackson kernel), so doubling M halves the width (the paper's Fig. 6:
    # more moments, finer DOS); integrated by the K-node Gauss-Chebyshev rule
    mu = np.cos(np.arange(M) * np.pi / 2)
    K = 4 * M
    E, rho = O.dos(mu, 1.0, 0.0, K)
    w = np.pi / K * np.sqrt(1.0 - E * E)
    m0, m2 = np.sum(w * rho), np.sum(w * rho * E * E)
    assert abs(m0 - 1.0) < 1e-12
    sigma = math.sqrt(m2 / m0)
    assert abs(sigma * M / math.pi - 1.0) < 3.0 / M
