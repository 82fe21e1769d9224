"""The stored exact moments of the paper's 10x10x10 lattice (Sec. IV-A) against
the plane-wave closed form and against the oracle's stochastic estimator with
the full basis."""
import math
import os

import numpy as np

import oracle as O

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_cubic10():
    a = b = None
    mu = []
    with open(os.path.join(HERE, "cubic10_exact_moments.txt")) as f:
        for line in f:
            if line.startswith("# a ="):
                parts = line.split()
                a, b = float(parts[3]), float(parts[6])
            elif not line.startswith("#"):
                mu.append(float(line.split()[1]))
    return a, b, np.array(mu)


def test_golden_matches_plane_wave_closed_form():
    a, b, mu = load_cubic10()
    assert a == 12.0 / 1.99 and b == 0.0 and mu.size == 512
    c = np.cos(2 * np.pi * np.arange(10) / 10)
    lam = -2.0 * (c[:, None, None] + c[None, :, None] + c[None, None, :]).ravel()
    x = (lam - b) / a
    expect = np.cos(np.arange(512)[:, None] * np.arccos(x)[None, :]).mean(axis=1)
    np.testing.assert_allclose(mu, expect, atol=1e-12)
    assert np.abs(mu[1::2]).max() < 1e-13      # bipartite, no on-site term


def test_golden_matches_full_basis_estimator():
    a, b, mu = load_cubic10()
    H = O.lattice_hamiltonian((10, 10, 10), onsite=np.zeros(1000))
    est, _ = O.moments_doubling(H, a, b, math.sqrt(1000) * np.eye(1000), 256)
    np.testing.assert_allclose(est, mu[:256], atol=1e-12)
