"""Pins of the oracle's Lorentz kernel and of its stochastic error bars
(oracle.lorentz_kernel, dos with kernel="lorentz", dos_many, stats,
dos_error_integral) against closed forms and invariants."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I


def lorentz_series_closed(M, lam, phi):
    """sum_{n<M} (2 - delta_n0) sinh(lam (1 - n/M))/sinh(lam) cos(n phi), from the two
    finite geometric sums sinh(lam (1 - n/M)) = (e^lam r^n - e^-lam r^-n)/2, r = e^(-lam/M)."""
    r = math.exp(-lam / M)

    def G(z):
        return (1.0 - z ** M) / (1.0 - z)

    z = np.exp(1j * np.asarray(phi, dtype=np.float64))
    s = (math.exp(lam) * G(r * z) - math.exp(-lam) * G(z / r)) / (2.0 * math.sinh(lam))
    return 2.0 * s.real - 1.0


@pytest.mark.parametrize("M,lam", [(16, 0.5), (300, 4.0), (1024, 3.0)])
def test_lorentz_kernel_geometric_closed_form(M, lam):
    g = O.lorentz_kernel(M, lam)
    assert g[0] == pytest.approx(1.0, abs=1e-15)
    phi = np.linspace(0.05, 3.1, 37)
    n = np.arange(M)
    direct = ((2.0 - (n == 0)) * g)[None, :] * np.cos(n[None, :] * phi[:, None])
    np.testing.assert_allclose(direct.sum(axis=1), lorentz_series_closed(M, lam, phi),
                               rtol=0, atol=1e-9 * M)


@pytest.mark.parametrize("x0", [0.3, -0.71])
def test_lorentz_dos_of_one_level(x0):
    # H = [x0], a = 1, b = 0: mu_n = T_n(x0); the damped series is the closed form
    # evaluated at theta_k -+ theta_0 (product to sum of the two cosines)
    M, K, lam = 200, 64, 4.0
    mu = np.cos(np.arange(M) * math.acos(x0))
    E, rho = O.dos(mu, 1.0, 0.0, K, "lorentz", lam)
    th = math.pi * (np.arange(K) + 0.5) / K
    t0 = math.acos(x0)
    S = 0.5 * (lorentz_series_closed(M, lam, th - t0) + lorentz_series_closed(M, lam, th + t0))
    np.testing.assert_allclose(rho, S / (math.pi * np.sin(th)), rtol=0, atol=1e-10)
    np.testing.assert_allclose(E, np.cos(th), rtol=0, atol=1e-15)


def test_dos_many_rows_equal_dos():
    rng = np.random.default_rng(3)
    P = rng.uniform(-1, 1, (4, 40)) * np.exp(-np.arange(40) / 10.0)
    for kernel in ("jackson", "none", "lorentz"):
        E, R = O.dos_many(P, 2.5, 0.3, 33, kernel, 4.0)
        for r in range(4):
            E1, rho1 = O.dos(P[r], 2.5, 0.3, 33, kernel, 4.0)
            np.testing.assert_allclose(R[r], rho1, rtol=0, atol=1e-12)
            np.testing.assert_allclose(E, E1, rtol=0, atol=1e-15)


def test_stats_of_diagonal_hamiltonian_have_no_spread():
    # diagonal H: <r|f(H)|r> = Tr f(H) for every Rademacher vector, so every vector
    # gives the same moments and the error bars vanish
    n = 24
    diag = np.linspace(-1.5, 2.0, n)
    H = O.CSR(n, np.arange(n + 1), np.arange(n), diag)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    _, P = O.moments_doubling(H, a, b, I.rademacher_block(5, n, 9), 32)
    mu_m, mu_e, E, rho_m, rho_e = O.stats(P, a, b, 50)
    assert np.abs(mu_e).max() <= 1e-15 and np.abs(rho_e).max() <= 1e-13
    np.testing.assert_allclose(mu_m, O.exact_moments(H, a, b, 32), rtol=0, atol=1e-13)


def test_stats_match_hutchinson_variance():
    # per-vector doubling moments are <r|T_m(H~)|r>/N; for Rademacher r their variance is
    # 2 (||T_m||_F^2 - sum_i T_m,ii^2) / N^2 (T_m from the eigendecomposition)
    L = (4, 4)
    H = O.lattice_hamiltonian(L, onsite=np.random.default_rng(1).uniform(-1, 1, 16))
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    M, R = 8, 4000
    _, P = O.moments_doubling(H, a, b, I.rademacher_block(21, H.n, R), M)
    _, mu_e, _, _, _ = O.stats(P, a, b, 16)
    lam, U = np.linalg.eigh(O.dense(H))
    x = np.clip((lam - b) / a, -1, 1)
    N = H.n
    for m in range(1, M):
        Tm = (U * np.cos(m * np.arccos(x))[None, :]) @ U.T
        var = 2.0 * (np.sum(Tm * Tm) - np.sum(np.diag(Tm) ** 2)) / N ** 2
        assert mu_e[m] * math.sqrt(R) == pytest.approx(math.sqrt(var), rel=0.08), m
    assert mu_e[0] == 0.0


@pytest.mark.parametrize("kernel", ["jackson", "none", "lorentz"])
def test_mean_dos_is_dos_of_mean_moments(kernel):
    rng = np.random.default_rng(9)
    P = rng.uniform(-1, 1, (7, 50)) * np.exp(-np.arange(50) / 12.0)
    mu_m, _, E, rho_m, _ = O.stats(P, 1.7, -0.2, 41, kernel, 3.0)
    E2, rho2 = O.dos(P.mean(axis=0), 1.7, -0.2, 41, kernel, 3.0)
    np.testing.assert_allclose(rho_m, rho2, rtol=0, atol=1e-12)


def test_dos_error_integral_of_a_constant():
    K, a, c = 257, 2.3, 0.01
    expect = c * a * math.pi / (K * math.sin(math.pi / (2 * K)))  # closed form of the node sum
    assert O.dos_error_integral(np.full(K, c), a) == pytest.approx(expect, rel=1e-13)


def test_ldos_exact_sums_to_the_dos_and_is_local_for_diagonal_h():
    # sum over all sites of <i|T_n|i> = Tr T_n = N mu_n (exact moments); for a
    # diagonal H the local moments of site i are T_n(E~_i)
    H = O.lattice_hamiltonian((5, 4), onsite=np.random.default_rng(2).uniform(-1, 1, 20))
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    loc = O.ldos_exact(H, a, b, np.arange(H.n), 30)
    np.testing.assert_allclose(loc.sum(axis=0), H.n * O.exact_moments(H, a, b, 30), rtol=0,
                               atol=1e-11)
    d = np.array([0.3, -0.7, 1.1])
    Hd = O.CSR(3, np.arange(4), np.arange(3), d)
    loc = O.ldos_exact(Hd, 2.0, 0.1, [2, 0], 12)
    x = (d - 0.1) / 2.0
    np.testing.assert_allclose(loc, [np.cos(np.arange(12) * np.arccos(x[2])),
                                     np.cos(np.arange(12) * np.arccos(x[0]))], atol=1e-13)


def lorentz_sine_closed(M, lam, phi):
    """sum_{n<M} (2 - delta_n0) sinh(lam (1 - n/M))/sinh(lam) sin(n phi) (two finite
    geometric sums, as lorentz_series_closed)."""
    r = math.exp(-lam / M)

    def G(z):
        return (1.0 - z ** M) / (1.0 - z)

    z = np.exp(1j * np.asarray(phi, dtype=np.float64))
    s = (math.exp(lam) * G(r * z) - math.exp(-lam) * G(z / r)) / (2.0 * math.sinh(lam))
    return 2.0 * s.imag


@pytest.mark.parametrize("x0", [0.2, -0.55])
def test_green_of_one_level_closed_form(x0):
    # H = [x0], a = 1, b = 0: mu_n = T_n(x0); 2 cos(n t0) e^{-i n t} splits into the
    # damped cosine and sine series at t -+ t0
    M, K, lam = 256, 48, 4.0
    mu = np.cos(np.arange(M) * math.acos(x0))
    E, G = O.green(mu, 1.0, 0.0, K, "lorentz", lam)
    th = math.pi * (np.arange(K) + 0.5) / K
    t0 = math.acos(x0)
    C = 0.5 * (lorentz_series_closed(M, lam, th - t0) + lorentz_series_closed(M, lam, th + t0))
    S = 0.5 * (lorentz_sine_closed(M, lam, th + t0) + lorentz_sine_closed(M, lam, th - t0))
    np.testing.assert_allclose(G.real, -S / np.sin(th), rtol=0, atol=1e-9)
    np.testing.assert_allclose(G.imag, -C / np.sin(th), rtol=0, atol=1e-9)


def test_green_imaginary_part_is_minus_pi_rho():
    rng = np.random.default_rng(4)
    mu = rng.uniform(-1, 1, 60) * np.exp(-np.arange(60) / 15.0)
    for kernel in ("jackson", "lorentz", "none"):
        E, G = O.green(mu, 2.2, 0.4, 37, kernel, 3.0)
        E2, rho = O.dos(mu, 2.2, 0.4, 37, kernel, 3.0)
        np.testing.assert_allclose(G.imag, -math.pi * rho, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(E, E2, rtol=0, atol=1e-15)


def test_thermo_closed_forms():
    # clean chain with the band [-2, 2] exactly (a = 2): the DOS is the arcsine law,
    # whose only nonzero moment is mu_0; at T = 0 and mu_c = 0, n = 1/2 and
    # u = -2/pi; at beta = 0 every state is half filled: n = 1/2, s = ln 2, c = 0
    mu = np.zeros(64)
    mu[0] = 1.0
    K = 4096
    t0 = O.thermo(mu, 2.0, 0.0, K, [np.inf], 0.0, "none")[0]
    assert t0[0] == pytest.approx(0.5, abs=1.0 / K) and t0[1] == pytest.approx(-2 / math.pi, abs=2.0 / K)
    assert t0[2] == 0.0 and t0[3] == 0.0
    hot = O.thermo(mu, 2.0, 0.0, K, [0.0], 0.3, "none")[0]
    assert hot[0] == pytest.approx(0.5, abs=1e-12) and hot[2] == pytest.approx(math.log(2), abs=1e-12)
    assert hot[3] == 0.0


def test_thermo_identities():
    # c = -beta^2 d(u - mu_c n)/dbeta and ds/dbeta = -c/beta (at fixed mu_c), by
    # central differences on a disordered lattice's moments
    H = O.lattice_hamiltonian((10, 10), onsite=np.random.default_rng(6).uniform(-1, 1, 100))
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    mu = O.exact_moments(H, a, b, 128)
    mu_c, beta, h = 0.3, 2.5, 1e-4
    r = O.thermo(mu, a, b, 2048, [beta - h, beta, beta + h], mu_c)
    g = r[:, 1] - mu_c * r[:, 0]
    assert -beta ** 2 * (g[2] - g[0]) / (2 * h) == pytest.approx(r[1, 3], rel=1e-6)
    assert (r[2, 2] - r[0, 2]) / (2 * h) == pytest.approx(-r[1, 3] / beta, rel=1e-6)
