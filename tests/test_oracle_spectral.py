"""Pins of the oracle's momentum-resolved moments (plane_waves, spectral_exact)
against closed forms and identities that do not reuse their formulas:

- on a clean periodic lattice a plane wave with k on the reciprocal grid is an
  eigenvector of H with E(k) = -2 t sum_d cos k_d (H_ij = -t on the bonds), so
  <k|T_n(H~)|k> = cos(n arccos E~(k)) exactly;
- the plane waves of the reciprocal grid are an orthogonal basis, so the
  average over the grid of <k|T_n|k> is the exact trace moment (any disorder,
  any Hermitian hopping);
- the recursion of Eq. (rn) from a plane-wave start vector (the doubling form)
  gives the same moments as the eigendecomposition."""
import math

import numpy as np

import oracle as O
from paper_1105_5481_gb300 import inputs as I


def _grid(L):
    ms = np.stack(np.meshgrid(*[np.arange(n) for n in L], indexing="ij"), axis=-1).reshape(-1, len(L))
    return 2 * math.pi * ms / np.asarray(L, dtype=np.float64)


def test_clean_lattice_plane_waves_are_eigenvectors():
    L, t = (6, 5, 4), 0.8
    H = O.lattice_hamiltonian(L, t=t)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    k = _grid(L)[[0, 1, 7, 33, 60, 119]]
    got = O.spectral_exact(H, a, b, L, k, 40)
    E = -2 * t * np.cos(k).sum(axis=1)
    x = (E - b) / a
    expect = np.cos(np.arange(40)[None, :] * np.arccos(x)[:, None])
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-12)
    # the same plane wave through the recursion
    _, per = O.moments_doubling(H, a, b, O.plane_waves(L, k), 40)
    np.testing.assert_allclose(per, expect, rtol=0, atol=1e-12)


def test_plane_waves_of_the_grid_are_orthogonal_and_sum_to_the_trace():
    L = (5, 4, 3)
    N = 60
    hop = I.spin_hoppings(L, *I.spins(5, N))
    H = O.lattice_hamiltonian(L, onsite=I.onsite_disorder(6, N, 2.0), hop=hop)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    k = _grid(L)
    P = O.plane_waves(L, k)
    np.testing.assert_allclose(P.conj().T @ P, N * np.eye(N), rtol=0, atol=1e-9)
    spec = O.spectral_exact(H, a, b, L, k, 32)
    np.testing.assert_allclose(spec.mean(axis=0), O.exact_moments(H, a, b, 32), rtol=0, atol=1e-12)


def test_recursion_from_plane_waves_matches_the_eigendecomposition():
    L = (7, 6)
    N = 42
    H = O.lattice_hamiltonian(L, periodic=(True, False), onsite=I.onsite_disorder(7, N, 1.5))
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    k = np.array([[0.3, 1.1], [2.0, -0.4], [math.pi, 0.0]])
    _, per = O.moments_doubling(H, a, b, O.plane_waves(L, k), 64)
    np.testing.assert_allclose(per, O.spectral_exact(H, a, b, L, k, 64), rtol=0, atol=1e-11)
