"""Local and momentum-resolved moments through the C ABI (kpm_ldos_moments,
kpm_spectral_moments): start blocks of unit vectors or plane waves written on
the device, the recursion of Eq. (rn), against the oracle's eigendecomposition
(ldos_exact, spectral_exact) and closed forms.  Tolerances as every parity
test: |d mu| <= 1e-10 (FP64 path), <= 1e-5 (FP32-vector path)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module")
def K(gpu_lib):
    from paper_1105_5481_gb300 import kpm

    return kpm


def _disordered(complex_):
    L = (6, 5, 4)
    n = 120
    kw = dict(onsite=I.onsite_disorder(8, n, 1.0))
    if complex_:
        kw["hop"] = I.spin_hoppings(L, *I.spins(3, n))
    return L, kw


def _handle(K, L, kw, complex_, csr):
    if not csr:
        return K.kpm_create_stencil(len(L), L, complex_=complex_, **kw)
    rp, col, val = K.kpm_stencil_to_csr(len(L), L, complex_=complex_, **kw)
    return K.kpm_create_csr(rp.size - 1, rp, col, val, complex_=complex_)


@pytest.mark.parametrize("complex_,prec,csr", [(False, "fp64", False), (True, "fp64", False),
                                               (True, "fp32", False), (False, "fp32", True),
                                               (True, "fp64", True)])
def test_ldos_matches_exact_local_moments(K, complex_, prec, csr):
    import torch

    L, kw = _disordered(complex_)
    H = O.lattice_hamiltonian(L, **kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    sites = [0, 17, 119, 17, 64]                 # a repeated site is allowed
    M = 96
    with _handle(K, L, kw, complex_, csr) as h:
        got = K.kpm_ldos_moments(h, sites, M, a, b, precision=prec)
        out = torch.empty(len(sites) * M, dtype=torch.float64, device="cuda")
        K.kpm_ldos_moments(h, sites, M, a, b, precision=prec, out=out)
        torch.cuda.synchronize()
        dev = out.cpu().numpy().reshape(len(sites), M)
        mu = K.kpm_moments(h, M, 4, a, b, seed=5, precision=prec)   # random vectors again after
    exact = O.ldos_exact(H, a, b, sites, M)
    assert np.abs(got - exact).max() <= TOL[prec]
    assert np.array_equal(dev, got)
    mu_o, _ = O.moments_doubling(H, a, b, I.random_block(5, H.n, 4, complex_), M)
    assert np.abs(mu - mu_o).max() <= TOL[prec]


def test_ldos_summed_over_all_sites_is_the_trace(K):
    L = (9, 7)
    onsite = I.onsite_disorder(4, 63, 2.0)
    H = O.lattice_hamiltonian(L, onsite=onsite)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    with K.kpm_create_stencil(2, L, onsite=onsite) as h:
        loc = K.kpm_ldos_moments(h, np.arange(63), 128, a, b)
    np.testing.assert_allclose(loc.sum(axis=0), 63 * O.exact_moments(H, a, b, 128), rtol=0,
                               atol=63 * 1e-10)


def test_ldos_large_lattice_fp32(K):
    # 2D L=128 disordered lattice (N=16384): the oracle runs the same recursion
    # from the unit start vectors sqrt(N) e_i (its per-vector moments)
    L = (128, 128)
    N = 16384
    onsite = I.onsite_disorder(12, N, 3.0)
    H = O.lattice_hamiltonian(L, onsite=onsite)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    sites = np.array([0, 1, 127, 128, 8191, 9000, 16256, 16383])
    V = np.zeros((N, sites.size))
    V[sites, np.arange(sites.size)] = math.sqrt(N)
    _, per_o = O.moments_doubling(H, a, b, V, 512)
    with K.kpm_create_stencil(2, L, onsite=onsite) as h:
        for prec in ("fp32", "fp64"):
            got = K.kpm_ldos_moments(h, sites, 512, a, b, precision=prec)
            assert np.abs(got - per_o).max() <= TOL[prec], prec


def test_ldos_refusals(K):
    with K.kpm_create_stencil(2, (4, 4)) as h:
        for bad in ([-1], [16], []):
            with pytest.raises(K.KPMError) as e:
                K.kpm_ldos_moments(h, bad, 16, 4.1, 0.0)
            assert e.value.status == K.KPM_EINVAL


def _grid_k(L, ms):
    return 2 * math.pi * np.asarray(ms, dtype=np.float64) / np.asarray(L, dtype=np.float64)


# FP32 vectors on a single eigenstate: the scaled operator's coefficients are
# rounded to FP32 (relative error u = 2^-24), which moves the state's rescaled
# energy x = cos(theta) by up to about 2u; mu_n = cos(n theta) then moves by up
# to n |d theta| = 2 n u / sin(theta).  Many states (the DOS moments of random
# vectors) average this out, one sharp state does not, so the FP32 path is held
# to 4 n u / sin(theta) + 1e-6 per moment here and the FP64 path to 1e-10.
@pytest.mark.parametrize("complex_,prec", [(False, "fp64"), (True, "fp64"), (False, "fp32"),
                                           (True, "fp32")])
def test_spectral_clean_lattice_closed_form(K, complex_, prec):
    # clean periodic lattice: the plane wave e^{i k.x} with k on the reciprocal
    # grid is an eigenvector, E(k) = -2 |t| sum_d cos(k_d + arg t) (H_ij = -t on
    # forward bonds), so mu_n = cos(n arccos E~(k)); a complex t makes E(k)
    # differ from E(-k), which pins the sign of the phase
    L, M = (8, 6, 5), 200
    t = complex(math.cos(0.4), math.sin(0.4)) if complex_ else 1.0
    H = O.lattice_hamiltonian(L, t=t)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    k = _grid_k(L, [[0, 0, 0], [1, 0, 0], [7, 0, 0], [3, 2, 1], [5, 4, 4], [4, 3, 0]])
    arg = math.atan2(t.imag, t.real) if complex_ else 0.0
    E = -2 * abs(t) * np.cos(k + arg).sum(axis=1)
    theta = np.arccos((E - b) / a)
    expect = np.cos(np.arange(M)[None, :] * theta[:, None])
    with K.kpm_create_stencil(3, L, t=t, complex_=complex_) as h:
        got = K.kpm_spectral_moments(h, k, M, a, b, precision=prec)
    if prec == "fp64":
        tol = TOL["fp64"]
    else:
        tol = 4 * np.arange(M)[None, :] * 2.0**-24 / np.sin(theta)[:, None] + 1e-6
    assert np.all(np.abs(got - expect) <= tol)


@pytest.mark.parametrize("complex_,prec", [(False, "fp64"), (True, "fp64"), (True, "fp32")])
def test_spectral_disordered_matches_oracle(K, complex_, prec):
    import torch

    L, kw = _disordered(complex_)
    H = O.lattice_hamiltonian(L, **kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    k = np.array([[0.3, -1.2, 2.5], [math.pi, 0.0, 0.0], [0.0, 0.0, 0.0], [1.0, 1.0, 1.0]])
    M = 128
    with K.kpm_create_stencil(3, L, complex_=complex_, **kw) as h:
        got = K.kpm_spectral_moments(h, k, M, a, b, precision=prec)
        out = torch.empty(k.shape[0] * M, dtype=torch.float64, device="cuda")
        K.kpm_spectral_moments(h, k, M, a, b, precision=prec, out=out)
        torch.cuda.synchronize()
    assert np.abs(got - O.spectral_exact(H, a, b, L, k, M)).max() <= TOL[prec]
    assert np.array_equal(out.cpu().numpy().reshape(k.shape[0], M), got)


def test_spectral_needs_a_lattice(K):
    rp, col, val = K.kpm_stencil_to_csr(2, (4, 4))
    with K.kpm_create_csr(16, rp, col, val) as h:
        with pytest.raises(K.KPMError) as e:
            K.kpm_spectral_moments(h, [[0.0, 0.0]], 16, 4.1, 0.0)
        assert e.value.status == K.KPM_EINVAL
