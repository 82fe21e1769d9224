"""Failure detection on the GPU without a fault: every wait inside the
TMA-fed step is bounded, and a wait that runs out is reported to the host as
KPM_ETIMEOUT with the context left usable.  The failure is made on the host
(kpm_testing_stall_step_pipeline: the step's producer issues no copy, so the
consumers wait for data that never comes, about a second, and give up); no
kernel is made to fault, trap or hang."""
import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K(gpu_lib):
    from paper_1105_5481_gb300 import kpm

    return kpm


def _csr(K):
    L = (35, 34, 33)          # large enough for the TMA-fed step (full 256-thread CTAs)
    N = 35 * 34 * 33
    kw = dict(dims=3, L=L, hop=I.spin_hoppings(L, *I.spins(5, N)), bond_mask=I.dilution_mask(5, N, 3))
    H = O.lattice_hamiltonian(L, hop=kw["hop"], mask=kw["bond_mask"])
    rp, col, val = K.kpm_stencil_to_csr(complex_=True, **kw)
    return H, rp, col, val


def test_step_wait_runs_out_and_reports_a_timeout(K):
    H, rp, col, val = _csr(K)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    K.kpm_testing_stall_step_pipeline(True)
    try:
        with K.kpm_create_csr(rp.size - 1, rp, col, val, complex_=True) as h:
            with pytest.raises(K.KPMError) as e:
                K.kpm_moments(h, 4, 32, a, b, seed=1, precision="fp32")   # one regular step
            assert e.value.status == K.KPM_ETIMEOUT
            assert K.kpm_testing_last_step_form(h) == "TMA-fed ELL step"
    finally:
        K.kpm_testing_stall_step_pipeline(False)
    # the context is still usable: a handle planned afterwards gives the oracle's moments
    with K.kpm_create_csr(rp.size - 1, rp, col, val, complex_=True) as h:
        mu = K.kpm_moments(h, 64, 32, a, b, seed=1, precision="fp32")
        assert K.kpm_testing_last_step_form(h) == "TMA-fed ELL step"
    mu_o, _ = O.moments_doubling(H, a, b, I.random_block(1, H.n, 32, True), 64)
    assert np.abs(mu - mu_o).max() <= 1e-5
