"""GPU parity of the FP32 path on mid-size lattices walked in line blocks
(2D and 3D stencils, chunks of one and two passes): moments against the FP64
oracle, |d mu_n| <= 1e-5, on periodic lattices, a ragged one with an open
last dimension, disorder and dilution, moment counts on either side of a
multiple of the cross-CTA reduction block (M/2 = 65, 66 steps), several
realisations, and the direct / captured / replayed forms of one call."""
import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def K(gpu_lib):
    from paper_1105_5481_gb300 import kpm

    return kpm


def case(name):
    if name == "cube_spin_L16":          # periodic 3D, complex spin hoppings
        L = (16, 16, 16)
        N = 4096
        return dict(dims=3, L=L, hop=I.spin_hoppings(L, *I.spins(21, N))), True
    if name == "box_open_z":             # ragged 3D, open last dimension, disorder + dilution
        L = (20, 12, 18)
        N = 20 * 12 * 18
        return dict(dims=3, L=L, periodic=(True, True, False), onsite=I.onsite_disorder(22, N, 2.0),
                    hop=I.spin_hoppings(L, *I.spins(23, N)),
                    bond_mask=I.dilution_mask(24, N, 3)), True
    if name == "plane_64x1024":          # periodic 2D, disorder, real
        L = (64, 1024)
        return dict(dims=2, L=L, onsite=I.onsite_disorder(25, 64 * 1024, 1.5)), False
    raise KeyError(name)


def oracle_H(kw):
    return O.lattice_hamiltonian(kw["L"], periodic=kw.get("periodic"), onsite=kw.get("onsite"),
                                 hop=kw.get("hop"), t=kw.get("t", 1.0), mask=kw.get("bond_mask"))


@pytest.mark.parametrize("M", [130, 132])
@pytest.mark.parametrize("name", ["cube_spin_L16", "box_open_z", "plane_64x1024"])
def test_line_traversal_moments_match_oracle(K, name, M):
    kw, cplx = case(name)
    H = oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R = 64 if cplx else 32
    seed = 31
    mu_o, per_o = O.moments_doubling(H, a, b, I.random_block(seed, H.n, R, cplx), M)
    with K.kpm_create_stencil(complex_=cplx, **kw) as h:
        mu, per = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp32", per_vec=True)
    assert np.abs(per - per_o).max() <= TOL
    assert np.abs(mu - mu_o).max() <= TOL


def test_line_traversal_realisations_and_replay(K):
    kw, cplx = case("cube_spin_L16")
    H = oracle_H(kw)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    R, S, M, seed = 64, 3, 200, 7
    # realisation s draws the columns s R .. (s+1) R - 1 of one R S block
    mu_o, _ = O.moments_doubling(H, a, b, I.random_block(seed, H.n, R * S, cplx), M)
    with K.kpm_create_stencil(complex_=cplx, **kw) as h:
        runs = [K.kpm_moments(h, M, R, a, b, seed=seed, S=S, precision="fp32") for _ in range(3)]
    assert np.abs(runs[0] - mu_o).max() <= TOL
    # direct launch, graph capture and graph replay give the same bits
    assert np.array_equal(runs[0], runs[1]) and np.array_equal(runs[1], runs[2])
