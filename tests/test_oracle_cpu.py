"""The C/OpenMP restatement of the oracle's doubling form (oracle/kpm_cpu.c),
used as the multi-core CPU baseline, against the NumPy oracle it restates."""
import numpy as np
import pytest

import oracle as O
from oracle import kpm_cpu as OC
from paper_1105_5481_gb300 import inputs as I


def _cases():
    rng = np.random.default_rng(5)
    L2 = (12, 10)
    H2 = O.lattice_hamiltonian(L2, onsite=rng.uniform(-1, 1, 120))
    yield "2d_real_onsite", H2, I.rademacher_block(3, H2.n, 6)
    L3 = (6, 5, 4)
    n3 = 6 * 5 * 4
    hop = I.spin_hoppings(L3, *I.spins(7, n3))
    H3 = O.lattice_hamiltonian(L3, hop=hop)
    yield "3d_complex_spin", H3, I.random_block(11, H3.n, 5, True)
    mask = I.dilution_mask(13, n3, 3)
    H4 = O.lattice_hamiltonian(L3, hop=hop, mask=mask, periodic=(True, False, True))
    yield "3d_diluted_open", H4, I.random_block(17, H4.n, 3, True)


@pytest.mark.parametrize("threads", [1, 2, 0])
def test_c_oracle_matches_numpy_oracle(threads):
    for name, H, v0 in _cases():
        a, b = O.rescale(*O.gershgorin(H), eps=0.01)
        mu_o, per_o = O.moments_doubling(H, a, b, v0, 64)
        mu_c, per_c = OC.moments_doubling(H, a, b, v0, 64, threads=threads)
        assert np.abs(per_c - per_o).max() <= 1e-12, name
        assert np.abs(mu_c - mu_o).max() <= 1e-12, name


def test_c_oracle_rejects_odd_moment_count():
    H = O.lattice_hamiltonian((4, 4))
    with pytest.raises(ValueError):
        OC.moments_doubling(H, 4.1, 0.0, I.rademacher_block(1, H.n, 2), 7)
