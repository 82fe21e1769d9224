"""Stochastic error bars (kpm_stats), the Lorentz kernel (kpm_dos_kernel) and the
adaptive number of vectors (kpm_moments_adaptive) against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K(gpu_lib):
    from paper_1105_5481_gb300 import kpm

    return kpm


def _pv(seed, nvec, M):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, (nvec, M)) * np.exp(-np.arange(M) / max(M / 6.0, 1.0))[None, :]


@pytest.mark.parametrize("nvec,M,Kn", [(1, 2, 1), (3, 64, 7), (17, 257, 512), (100, 1000, 129)])
@pytest.mark.parametrize("kernel", ["jackson", "none", "lorentz"])
def test_stats_match_oracle(K, nvec, M, Kn, kernel):
    P = _pv(nvec * 31 + M, nvec, M)
    a, b = 3.1, -0.4
    got = K.kpm_stats(P, a, b, Kn, kernel, lam=4.0)
    ref = O.stats(P, a, b, Kn, kernel, 4.0)
    names = ["mu_mean", "mu_err", "E", "rho_mean", "rho_err"]
    for name, g, r in zip(names, got, ref):
        scale = max(1.0, np.abs(r).max())
        np.testing.assert_allclose(g, r, rtol=0, atol=1e-12 * scale * max(1, M / 64), err_msg=name)


def test_stats_from_device_per_vector_moments(K):
    import torch

    w = I.workload("square_L32_fp64")
    h = K.kpm_create_stencil(2, w["L"], onsite=w["onsite"])
    _, _, a, b = K.kpm_bounds(h, 0, 0.01)
    pv = torch.empty((w["R"], w["M"]), dtype=torch.float64, device="cuda")
    K.kpm_moments(h, w["M"], w["R"], a, b, seed=w["seed"], out_per_vec=pv)
    torch.cuda.synchronize()
    got = K.kpm_stats(pv, a, b, 256)
    ref = O.stats(pv.cpu().numpy(), a, b, 256)
    for g, r in zip(got, ref):
        np.testing.assert_allclose(g, r, rtol=0, atol=1e-12 * max(1.0, np.abs(r).max()))
    h.close()


@pytest.mark.parametrize("lam", [0.5, 4.0])
def test_lorentz_dos_matches_oracle(K, lam):
    mu = _pv(7, 1, 300)[0]
    mu[0] = 1.0
    E, rho = K.kpm_dos(mu, 2.0, 0.1, 200, "lorentz", lam=lam)
    E_o, rho_o = O.dos(mu, 2.0, 0.1, 200, "lorentz", lam)
    np.testing.assert_allclose(E, E_o, rtol=0, atol=1e-14)
    # an FP64 series of M terms: rounding grows with M and with the largest value
    # (weak damping leaves large values next to the band edges)
    tol = 1e-12 * max(1.0, np.abs(rho_o).max()) * max(1, mu.size / 64)
    np.testing.assert_allclose(rho, rho_o, rtol=0, atol=tol)


def test_lorentz_needs_positive_lambda(K):
    with pytest.raises(K.KPMError):
        K.kpm_dos(np.ones(8), 1.0, 0.0, 8, "lorentz", lam=0.0)
    with pytest.raises(K.KPMError):
        K.kpm_dos(np.ones(8), 1.0, 0.0, 8, "lorentz")


def test_adaptive_rounds_and_error(K):
    L = (24, 24)
    onsite = I.onsite_disorder(4, 576, 2.0)
    h = K.kpm_create_stencil(2, L, onsite=onsite)
    _, _, a, b = K.kpm_bounds(h, 0, 0.01)
    M, R, Kn = 128, 4, 128
    # unreachable target: all rounds run; the result is the mean over the rounds'
    # vectors, which are those of kpm_moments with seeds 50, 51, 52
    res = K.kpm_moments_adaptive(h, M, R, a, b, Kn, 0.0, 3, seed=50, precision="fp64")
    assert res["rounds"] == 3
    P = np.vstack([K.kpm_moments(h, M, R, a, b, seed=50 + i, precision="fp64", per_vec=True)[1]
                   for i in range(3)])
    ref = O.stats(P, a, b, Kn)
    np.testing.assert_allclose(res["mu"], ref[0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(res["mu_err"], ref[1], rtol=0, atol=1e-13)
    np.testing.assert_allclose(res["rho"], ref[3], rtol=0, atol=1e-11)
    np.testing.assert_allclose(res["rho_err"], ref[4], rtol=0, atol=1e-11)
    assert res["error"] == pytest.approx(O.dos_error_integral(ref[4], a), rel=1e-9)
    # a reachable target stops early, with the error at or below it
    loose = 2.0 * res["error"]
    res2 = K.kpm_moments_adaptive(h, M, R, a, b, Kn, loose, 10, seed=50, precision="fp64")
    assert 1 <= res2["rounds"] <= 3 and res2["error"] <= loose
    h.close()


@pytest.mark.parametrize("complex_", [False, True], ids=["real", "complex"])
def test_ldos_moments_match_exact(K, complex_):
    L = (6, 5, 4)
    n = 120
    kw = {}
    if complex_:
        kw["hop"] = I.spin_hoppings(L, *I.spins(3, n))
    onsite = I.onsite_disorder(8, n, 1.0)
    H = O.lattice_hamiltonian(L, onsite=onsite, **kw)
    h = K.kpm_create_stencil(3, L, onsite=onsite, complex_=complex_, **kw)
    _, _, a, b = K.kpm_bounds(h, 0, 0.01)
    sites = [0, 17, 119]
    got = K.kpm_ldos_moments(h, sites, 64, a, b)
    np.testing.assert_allclose(got, O.ldos_exact(H, a, b, sites, 64), rtol=0, atol=1e-10)
    h.close()


@pytest.mark.parametrize("kernel", ["lorentz", "jackson"])
def test_green_matches_oracle(K, kernel):
    mu = _pv(13, 1, 400)[0]
    mu[0] = 1.0
    E, G = K.kpm_green(mu, 1.8, -0.3, 160, kernel, lam=4.0)
    E_o, G_o = O.green(mu, 1.8, -0.3, 160, kernel, 4.0)
    tol = 1e-12 * max(1.0, np.abs(G_o).max()) * (mu.size / 64)
    np.testing.assert_allclose(E, E_o, rtol=0, atol=1e-14)
    np.testing.assert_allclose(G.real, G_o.real, rtol=0, atol=tol)
    np.testing.assert_allclose(G.imag, G_o.imag, rtol=0, atol=tol)


def test_thermo_matches_oracle(K):
    rng = np.random.default_rng(21)
    mu = rng.uniform(-1, 1, 200) * np.exp(-np.arange(200) / 40.0)
    mu[0] = 1.0
    betas = np.array([0.0, 0.5, 3.0, 40.0, np.inf])
    got = K.kpm_thermo(mu, 2.4, 0.2, 300, betas, mu_c=0.35)
    ref = O.thermo(mu, 2.4, 0.2, 300, betas, 0.35)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-12)
