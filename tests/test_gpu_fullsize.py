"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: the oracle recomputes sampled vector columns (each column's recursion
is independent of the others), and every column must satisfy the invariants
mu_0 = 1 and |mu_n| <= 1 that hold at any size."""
import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K(gpu_lib):
    from paper_1105_5481_gb300 import kpm

    return kpm


def test_cubic_L64_full_size_sampled_columns(K):
    # 3D L=64 spin lattice (N=262144), R=64 random phases, M=1024: eight columns
    # spread over the block, every moment, both precisions, against the oracle's
    # C form (pinned to the NumPy oracle by test_oracle_cpu.py)
    from oracle import kpm_cpu as OC

    w = I.workload("cubic_spin_L64")
    H = O.lattice_hamiltonian(w["L"], hop=w["hop"])
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    cols = [0, 7, 8, 21, 33, 41, 56, 63]
    seed = 1000
    v0 = I.random_columns(seed, H.n, w["R"], cols, True)
    _, per_o = OC.moments_doubling(H, a, b, v0, w["M"], threads=OC.max_threads())
    with K.kpm_create_stencil(3, w["L"], hop=w["hop"], complex_=True) as h:
        for prec, tol, tol0 in (("fp32", 1e-5, 1e-6), ("fp64", 1e-10, 1e-14)):
            mu, per = K.kpm_moments(h, w["M"], w["R"], a, b, seed=seed, precision=prec, per_vec=True)
            assert np.abs(per[cols] - per_o).max() <= tol, prec
            assert np.abs(per[:, 0] - 1.0).max() <= tol0
            assert np.abs(per).max() <= 1.0 + tol
            np.testing.assert_allclose(mu, per.mean(axis=0), rtol=0, atol=1e-14)


def test_csr_L160_full_size_all_moments(K):
    # 3D L=160 spin lattice with 10% bond dilution as CSR (N=4.1M, nnz=22.1M),
    # R=32, M=4096, FP32 vectors, in the launch configuration the benchmark
    # times: two sampled columns over all 4096 moments against the oracle's C
    # form (the FP32 rounding grows with n, so the deepest moments are the
    # ones that matter), the invariants on every column and moment
    from oracle import kpm_cpu as OC

    w = I.workload("csr_spin_dilute_L160")
    rp, col, val = K.kpm_stencil_to_csr(3, w["L"], hop=w["hop"], bond_mask=w["mask"], complex_=True)
    H = O.lattice_hamiltonian(w["L"], hop=w["hop"], mask=w["mask"])
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    seed, c = 77, [0, 19]
    with K.kpm_create_csr(rp.size - 1, rp, col, val, complex_=True) as h:
        mu, per = K.kpm_moments(h, w["M"], w["R"], a, b, seed=seed, precision="fp32", per_vec=True)
    assert np.abs(per[:, 0] - 1.0).max() <= 1e-6
    assert np.abs(per).max() <= 1.0 + 1e-5
    v0 = I.random_columns(seed, H.n, w["R"], c, True)
    _, per_o = OC.moments_doubling(H, a, b, v0, w["M"], threads=OC.max_threads())
    assert np.abs(per[c] - per_o).max() <= 1e-5


def test_batch_256_full_size_sampled_instances(K):
    # the full batch workload (256 2D disorder realisations, L 16..128, M 128..2048,
    # R = 16 FP32) in one persistent launch; the oracle recomputes one vector column
    # of four sampled instances at full M, and every instance obeys the invariants
    insts = I.batch_workload(3, 256)
    R = 16
    hs = [K.kpm_create_stencil(2, x["L"], onsite=x["onsite"]) for x in insts]
    ab = [K.kpm_bounds(h, 0, 0.01)[2:] for h in hs]
    Ms = [x["M"] for x in insts]
    with K.kpm_batch_create(hs, Ms, R, [p[0] for p in ab], [p[1] for p in ab],
                            [x["seed"] for x in insts], "fp32") as bt:
        parts = bt.split(K.kpm_batch_run(bt))
    sizes = [x["L"][0] for x in insts]
    picks = {int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 200}
    for k, mu in enumerate(parts):
        assert abs(mu[0] - 1.0) <= 1e-6 and np.abs(mu).max() <= 1.0 + 1e-5
    for k in sorted(picks):
        x = insts[k]
        H = O.lattice_hamiltonian(x["L"], onsite=x["onsite"])
        a, b = ab[k]
        v0 = I.random_block(x["seed"], H.n, R, False)
        mu_o, _ = O.moments_doubling(H, a, b, v0, x["M"])
        assert np.abs(parts[k] - mu_o).max() <= 1e-5, k
    for h in hs:
        h.close()
