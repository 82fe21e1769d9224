"""The paper's evaluation lattice run in the paper's own parameters on the GPU
path, FP64 as in the paper: the DOS comparison of Fig. 6 (Sec. IV-A: the
10x10x10 cube, R = 14 vectors, S = 128 realisations, N = 256 against N = 512
moments), with the same random vectors for both: both DOS integrate to one,
and the larger moment count resolves the spectrum more finely."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K(gpu_lib):
    from paper_1105_5481_gb300 import kpm

    return kpm


def test_fig6_more_moments_resolve_the_dos_more_finely(K):
    H = O.lattice_hamiltonian((10, 10, 10))
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    lam = np.sort(np.linalg.eigvalsh(O.dense(H)))       # the exact (discrete) spectrum
    Kn = 2048
    E_ref, rho_ref = O.dos(O.exact_moments(H, a, b, 4096), a, b, Kn)
    dens, cdf = {}, {}
    with K.kpm_create_stencil(3, (10, 10, 10)) as h:
        for M in (256, 512):
            mu = K.kpm_moments(h, M, 14, a, b, seed=3, S=128, precision="fp64")
            E, rho = K.kpm_dos(mu, a, b, Kn)
            np.testing.assert_allclose(E, E_ref, rtol=0, atol=1e-13)
            order = np.argsort(E)
            E, rho, r_ref = E[order], rho[order], rho_ref[order]
            w = a * np.pi / Kn * np.sqrt(1.0 - ((E - b) / a) ** 2)  # Gauss-Chebyshev in E
            assert abs(np.sum(w * rho) - 1.0) < 1e-12
            # distance to the exact spectrum broadened at M = 4096, and between the
            # integrated DOS and the exact staircase: both shrink as M grows
            dens[M] = float(np.sum(w * np.abs(rho - r_ref)))
            stair = np.searchsorted(lam, E, side="right") / lam.size
            gap = np.abs(np.cumsum(w * rho) - stair)
            cdf[M] = float(np.sum(0.5 * (gap[1:] + gap[:-1]) * np.diff(E)))  # trapezoid rule
    assert dens[512] < 0.95 * dens[256], dens
    assert cdf[512] < 0.7 * cdf[256], cdf
