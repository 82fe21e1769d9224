"""The dense formulation's products on the bf16 tensor cores (the Ozaki
splitting scheme: beta-bit integer slices of S and of each vector block,
exact FP32 slice products, FP64 recombination), against the FP64 oracle
(|d mu| <= 1e-10) and against the FP64-pipe kernel on the same inputs
(|d mu| <= 1e-12: both are FP64-accurate, they differ only in rounding).
KPM_DENSE_TENSOR selects the form: 1 forces the tensor cores at any size, 0
the FP64 kernel."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K(gpu_lib):
    from paper_1105_5481_gb300 import kpm

    return kpm


def _moments(K, A, M, R, a, b, seed, tensor, user_v0=None):
    old = os.environ.get("KPM_DENSE_TENSOR")
    os.environ["KPM_DENSE_TENSOR"] = tensor
    try:
        with K.kpm_create_dense(A) as h:
            out = [K.kpm_moments(h, M, R, a, b, seed=seed, per_vec=True, user_v0=user_v0)
                   for _ in range(2)]   # a direct call, then the captured graph
            form = K.kpm_testing_last_step_form(h)
    finally:
        if old is None:
            del os.environ["KPM_DENSE_TENSOR"]
        else:
            os.environ["KPM_DENSE_TENSOR"] = old
    assert np.array_equal(out[0][1], out[1][1])
    assert form == ("dense tensor cores" if tensor == "1" else "dense FP64 pipe")
    return out[0]


@pytest.mark.parametrize("n,R", [(1, 3), (97, 5), (200, 16), (70, 2101), (513, 24)])
def test_tensor_core_products_match_oracle_and_fp64(K, n, R):
    A = I.dense_hermitian(40 + n, n, False)
    H = O.from_dense(A)
    a, b = O.rescale(*O.gershgorin(H), 0.01) if n > 1 else (1.0, float(A[0, 0]))
    M, seed = 66, 17
    mu_o, per_o = O.moments_doubling(H, a, b, I.random_block(seed, n, R, False), M)
    mu_t, per_t = _moments(K, A, M, R, a, b, seed, "1")
    mu_f, per_f = _moments(K, A, M, R, a, b, seed, "0")
    assert np.abs(per_t - per_o).max() <= 1e-10
    assert np.abs(mu_t - mu_o).max() <= 1e-10
    assert np.abs(per_t - per_f).max() <= 1e-12


def test_slice_products_at_the_exactness_bound(K):
    # D = 4096 (beta = 6): S = 0.99 everywhere and constant start columns make
    # the first slice product 4096 * 63 * 63 = 16,257,024, just below 2^24, the
    # largest the FP32 accumulation must still hold exactly
    n, R, M = 4096, 8, 24
    A = np.full((n, n), 0.99)
    a, b = 0.99 * n / 1.98, 0.99 * n / 2      # spectrum {0, 0.99 n} inside [b - a, b + a]
    v0 = np.ones((n, R)) * np.where(np.arange(R) % 2, -1.0, 1.0)
    mu_t, per_t = _moments(K, A, M, R, a, b, 0, "1", user_v0=v0)
    mu_f, per_f = _moments(K, A, M, R, a, b, 0, "0", user_v0=v0)
    # one coherent state: the two FP64-accurate forms' own rounding grows to
    # about 1e-11 here; a slice product that lost its exactness would be off
    # by 2^-24 relative, about 1e-8
    assert np.abs(per_t - per_f).max() <= 1e-10
    # the exact moments: v0 / sqrt(N) is the eigenvector of 0.99 n; x = (0.99 n - b) / a
    x = (0.99 * n - b) / a
    assert np.abs(mu_t - np.cos(np.arange(M) * np.arccos(x))).max() <= 1e-10
