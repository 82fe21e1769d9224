"""The batched persistent launch: every instance against the oracle, the same
instance alone and in a mix (bitwise, for a fixed cluster size), all cluster
sizes, R-tiling (an instance's columns split into independent tasks), the
resident form (vector rows kept in the clusters' shared memory), and the
autotuner with its on-disk cache."""
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


def instances(n=10, seed=21):
    """2D disorder realisations of uneven size (a scaled-down batch workload)."""
    rng = np.random.default_rng(seed)
    Ls = [5, 8, 13, 16, 24, 32, 7, 40, 11, 20, 3, 48][:n]
    out = []
    for k, L in enumerate(Ls):
        W = float(rng.uniform(0, 4))
        on = I.onsite_disorder(seed * 1000 + k, L * L, W)
        M = int(2 * rng.integers(8, 80))
        H = O.lattice_hamiltonian((L, L), onsite=on)
        a, b = O.rescale(*O.gershgorin(H), eps=0.01)
        out.append(dict(L=(L, L), onsite=on, M=M, H=H, a=a, b=b, seed=seed * 100 + k))
    return out


def make_batch(K, insts, prec, R=16):
    hs = [K.kpm_create_stencil(2, x["L"], onsite=x["onsite"]) for x in insts]
    bt = K.kpm_batch_create(hs, [x["M"] for x in insts], R, [x["a"] for x in insts],
                            [x["b"] for x in insts], [x["seed"] for x in insts], precision=prec)
    return bt


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_instances_match_oracle(K, prec):
    insts = instances()
    R = 16
    with make_batch(K, insts, prec, R) as bt:
        K.kpm_batch_set_config(bt, 4, 4, 100)
        parts = bt.split(K.kpm_batch_run(bt))
    for x, mu in zip(insts, parts):
        mu_o, _ = O.moments_doubling(x["H"], x["a"], x["b"], I.rademacher_block(x["seed"], x["H"].n, R),
                                     x["M"])
        assert np.abs(mu - mu_o).max() <= TOL[prec]


def test_batch_equals_single_instance_call(K):
    insts = instances(6)
    with make_batch(K, insts, "fp64") as bt:
        parts = bt.split(K.kpm_batch_run(bt))
    for x, mu in zip(insts, parts):
        with K.kpm_create_stencil(2, x["L"], onsite=x["onsite"]) as h:
            ref = K.kpm_moments(h, x["M"], 16, x["a"], x["b"], seed=x["seed"])
        assert np.abs(mu - ref).max() <= 1e-12


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_instance_alone_and_in_the_mix_is_bitwise_identical(K, prec):
    insts = instances()
    for C in (1, 4):
        with make_batch(K, insts, prec) as bt:
            K.kpm_batch_set_config(bt, C, 4, 100)
            mix = bt.split(K.kpm_batch_run(bt))
        for k in (0, 5, 7):
            with make_batch(K, [insts[k]], prec) as b1:
                K.kpm_batch_set_config(b1, C, 4, 100)
                alone = K.kpm_batch_run(b1)
            assert np.array_equal(alone, mix[k])


@pytest.mark.parametrize("C", [1, 2, 4, 8, 16])
def test_every_cluster_size(K, C):
    insts = instances(8)
    with make_batch(K, insts, "fp64") as bt:
        K.kpm_batch_set_config(bt, C, 2, 50)
        parts = bt.split(K.kpm_batch_run(bt))
        info = K.kpm_batch_info(bt)
    assert info["cluster"] == C and info["clusters"] >= 1
    for x, mu in zip(insts, parts):
        mu_o, _ = O.moments_doubling(x["H"], x["a"], x["b"], I.rademacher_block(x["seed"], x["H"].n, 16),
                                     x["M"])
        assert np.abs(mu - mu_o).max() <= 1e-10


# R = 16 real FP32 is 2 chunks per row; R = 32 real FP32, R = 16 complex FP32
# and R = 8 real FP64 are 4 (the most tiles); R = 13 leaves padded columns
@pytest.mark.parametrize("prec,R,tiles", [("fp32", 16, 2), ("fp32", 32, 4), ("fp64", 8, 4),
                                          ("fp32", 13, 2), ("fp64", 8, 2)])
def test_rtiles_match_oracle(K, prec, R, tiles):
    insts = instances(8)
    with make_batch(K, insts, prec, R) as bt:
        assert K.kpm_batch_get_rtiles(bt) == (1, 0, min(4, -(-R // {"fp32": 8, "fp64": 2}[prec])))
        K.kpm_batch_set_config(bt, 2, 4, 100)
        K.kpm_batch_set_rtiles(bt, tiles)
        assert K.kpm_batch_get_rtiles(bt)[:2] == (tiles, len(insts))
        parts = bt.split(K.kpm_batch_run(bt))
        again = bt.split(K.kpm_batch_run(bt))      # the tile counters restart on each replay
    for x, mu, mu2 in zip(insts, parts, again):
        mu_o, _ = O.moments_doubling(x["H"], x["a"], x["b"], I.rademacher_block(x["seed"], x["H"].n, R),
                                     x["M"])
        assert np.abs(mu - mu_o).max() <= TOL[prec]
        assert np.array_equal(mu, mu2)


@pytest.mark.parametrize("top", [1, 3])
def test_rtiles_of_the_largest_instances_only(K, top):
    # only the `top` instances of largest N*M are tiled; the others run whole
    insts = instances(10)
    with make_batch(K, insts, "fp32", 32) as bt:
        K.kpm_batch_set_config(bt, 4, 4, 100)
        K.kpm_batch_set_rtiles(bt, 4, top)
        assert K.kpm_batch_get_rtiles(bt)[:2] == (4, top)
        parts = bt.split(K.kpm_batch_run(bt))
    for x, mu in zip(insts, parts):
        mu_o, _ = O.moments_doubling(x["H"], x["a"], x["b"], I.rademacher_block(x["seed"], x["H"].n, 32),
                                     x["M"])
        assert np.abs(mu - mu_o).max() <= 1e-5


def test_rtiles_complex_and_refusals(K):
    L = (12, 10)
    N = 120
    hop = I.spin_hoppings(L, *I.spins(3, N))
    H = O.lattice_hamiltonian(L, hop=hop)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    with K.kpm_create_stencil(2, L, hop=hop, complex_=True) as h:
        bt = K.kpm_batch_create([h, h], [40, 62], 16, [a, a], [b, b], [5, 6], precision="fp32")
        with bt:
            for bad in (3, 8):
                with pytest.raises(K.KPMError) as e:
                    K.kpm_batch_set_rtiles(bt, bad)
                assert e.value.status == K.KPM_EINVAL
            K.kpm_batch_set_rtiles(bt, 4)
            parts = bt.split(K.kpm_batch_run(bt))
    for M, seed, mu in zip((40, 62), (5, 6), parts):
        mu_o, _ = O.moments_doubling(H, a, b, I.phase_block(seed, N, 16), M)
        assert np.abs(mu - mu_o).max() <= 1e-5


def test_autotuner_writes_and_reuses_its_cache(K, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("KPM_TUNE_CACHE", str(cache))
    insts = instances(6)
    with make_batch(K, insts, "fp32") as bt:
        info = K.kpm_batch_tune(bt, reps=1)
        mu = K.kpm_batch_run(bt)
        tiles, tiled, _ = K.kpm_batch_get_rtiles(bt)
        resident = K.kpm_batch_get_resident(bt)[0]
        chunk_bytes = K.kpm_batch_get_chunk_bytes(bt)[0]
    assert not (resident and tiles > 1)
    text = cache.read_text()
    assert "batch|" in text and f"= {info['cluster']} {info['chunk']}" in text
    fields = text.strip().splitlines()[-1].split(" = ")[1].split()
    assert int(fields[3]) == tiles and (tiles == 1 or int(fields[4]) in (0, tiled))
    assert int(fields[5]) == int(resident)
    assert int(fields[6]) == {32: 1, 16: 2}[chunk_bytes]
    with make_batch(K, insts, "fp32") as bt2:
        info2 = K.kpm_batch_info(bt2)
        mu2 = K.kpm_batch_run(bt2)
        assert K.kpm_batch_get_rtiles(bt2)[:2] == (tiles, tiled)
        assert K.kpm_batch_get_resident(bt2)[0] == resident
        assert K.kpm_batch_get_chunk_bytes(bt2)[0] == chunk_bytes
    assert (info2["cluster"], info2["chunk"]) == (info["cluster"], info["chunk"])
    assert np.array_equal(mu, mu2)


# ---------------------------------------------------------------- resident form
# Each cluster keeps its instance's two vector blocks in shared memory (CTA k
# owns rows [kP, kP + P), P = ceil(N / C)) and reads the other CTAs' rows
# through distributed shared memory.


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_resident_instances_match_oracle(K, prec):
    insts = instances()
    with make_batch(K, insts, prec) as bt:
        K.kpm_batch_set_resident(bt, True)
        on, cmin = K.kpm_batch_get_resident(bt)
        # largest instance 48 x 48, R = 16: 2 x 295 KB of FP64 rows fit 4 CTAs
        assert on and 1 <= cmin <= 4
        K.kpm_batch_set_config(bt, 4, 4, 100)
        parts = bt.split(K.kpm_batch_run(bt))
        again = bt.split(K.kpm_batch_run(bt))
    for x, mu, mu2 in zip(insts, parts, again):
        mu_o, _ = O.moments_doubling(x["H"], x["a"], x["b"], I.rademacher_block(x["seed"], x["H"].n, 16),
                                     x["M"])
        assert np.abs(mu - mu_o).max() <= TOL[prec]
        assert np.array_equal(mu, mu2)


@pytest.mark.parametrize("C", [1, 2, 4, 8, 16])
def test_resident_every_cluster_size_alone_and_in_the_mix(K, C):
    # C = 16 leaves the last CTAs of the 5 x 5 instance without rows
    insts = instances(8)
    with make_batch(K, insts, "fp32") as bt:
        K.kpm_batch_set_resident(bt, True)
        assert K.kpm_batch_get_resident(bt)[1] == 1  # 40 x 40, R = 16 FP32: 2 x 100 KB
        K.kpm_batch_set_config(bt, C, 4, 50)
        parts = bt.split(K.kpm_batch_run(bt))
        assert K.kpm_batch_info(bt)["cluster"] == C
    for x, mu in zip(insts, parts):
        mu_o, _ = O.moments_doubling(x["H"], x["a"], x["b"], I.rademacher_block(x["seed"], x["H"].n, 16),
                                     x["M"])
        assert np.abs(mu - mu_o).max() <= 1e-5
    for k in (0, 5):
        with make_batch(K, [insts[k]], "fp32") as b1:
            K.kpm_batch_set_resident(b1, True)
            K.kpm_batch_set_config(b1, C, 4, 100)
            assert np.array_equal(K.kpm_batch_run(b1), parts[k])


@pytest.mark.parametrize("prec,R,tol", [("fp32", 16, 1e-5), ("fp64", 8, 1e-10)])
def test_resident_complex_hoppings_open_edge_3d(K, prec, R, tol):
    # spin-derived complex hoppings, on-site disorder, one open direction;
    # random-phase vectors (R = 16 complex FP32: 4 chunks per row)
    L, periodic = (6, 5, 4), (True, False, True)
    N = 120
    hop = I.spin_hoppings(L, *I.spins(7, N))
    on = I.onsite_disorder(8, N, 1.0)
    H = O.lattice_hamiltonian(L, periodic=periodic, onsite=on, hop=hop)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    with K.kpm_create_stencil(3, L, periodic=periodic, onsite=on, hop=hop, complex_=True) as h:
        with K.kpm_batch_create([h, h], [40, 62], R, [a, a], [b, b], [5, 6], precision=prec) as bt:
            K.kpm_batch_set_resident(bt, True)
            K.kpm_batch_set_config(bt, 4, 4, 100)
            parts = bt.split(K.kpm_batch_run(bt))
    for M, seed, mu in zip((40, 62), (5, 6), parts):
        mu_o, _ = O.moments_doubling(H, a, b, I.phase_block(seed, N, R), M)
        assert np.abs(mu - mu_o).max() <= tol


@pytest.mark.parametrize("periodic", [True, False])
def test_resident_chain_across_ctas(K, periodic):
    # a 1D chain of 50 sites on 2 CTAs: the bonds 24-25 (and 49-0 when
    # periodic) join rows held by different CTAs
    N = 50
    on = I.onsite_disorder(9, N, 2.0)
    H = O.lattice_hamiltonian((N,), periodic=(periodic,), onsite=on)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    with K.kpm_create_stencil(1, (N,), periodic=(periodic,), onsite=on) as h:
        with K.kpm_batch_create([h], [64], 8, [a], [b], [11], precision="fp64") as bt:
            K.kpm_batch_set_resident(bt, True)
            K.kpm_batch_set_config(bt, 2, 4, 100)
            mu = K.kpm_batch_run(bt)
    mu_o, _ = O.moments_doubling(H, a, b, I.rademacher_block(11, N, 8), 64)
    assert np.abs(mu - mu_o).max() <= 1e-10


def test_resident_refusals(K):
    # too large for any cluster: 128 x 128, R = 16 FP64 is 2 x 2 MB of rows
    L = (128, 128)
    with K.kpm_create_stencil(2, L) as h:
        with K.kpm_batch_create([h], [8], 16, [4.1], [0.0], [1], precision="fp64") as bt:
            K.kpm_batch_set_resident(bt, True)
            assert K.kpm_batch_get_resident(bt) == (True, 0)
            with pytest.raises(K.KPMError) as e:
                K.kpm_batch_run(bt)
            assert e.value.status == K.KPM_EINVAL
            with pytest.raises(K.KPMError) as e:
                K.kpm_batch_set_rtiles(bt, 2)
            assert e.value.status == K.KPM_EINVAL
            K.kpm_batch_set_resident(bt, False)
            assert np.abs(K.kpm_batch_run(bt)[0] - 1.0) <= 1e-12
    # CSR operators have no resident form
    Hs = O.lattice_hamiltonian((6, 6))
    with K.kpm_create_csr(Hs.n, Hs.rowptr, Hs.col, Hs.val) as h:
        with K.kpm_batch_create([h], [8], 8, [4.1], [0.0], [1], precision="fp64") as bt:
            with pytest.raises(K.KPMError) as e:
                K.kpm_batch_set_resident(bt, True)
            assert e.value.status == K.KPM_EINVAL
            assert K.kpm_batch_get_resident(bt) == (False, 0)


# ---------------------------------------------------------------- threads per row
# 16-byte chunks: each thread moves 4 real FP32 columns of a row, so a row
# takes twice the threads of the default 32-byte chunk (same row layout).


@pytest.mark.parametrize("R", [16, 13, 32])
@pytest.mark.parametrize("C", [1, 4])
def test_half_chunks_match_oracle(K, R, C):
    insts = instances(8)
    Rp = {16: 16, 13: 16, 32: 32}[R]   # padded to a power of two of 8-column chunks
    with make_batch(K, insts, "fp32", R) as bt:
        assert K.kpm_batch_get_chunk_bytes(bt) == (32, Rp // 8)
        K.kpm_batch_set_chunk_bytes(bt, 16)
        assert K.kpm_batch_get_chunk_bytes(bt) == (16, Rp // 4)
        K.kpm_batch_set_config(bt, C, 4, 100)
        parts = bt.split(K.kpm_batch_run(bt))
        again = bt.split(K.kpm_batch_run(bt))
    for x, mu, mu2 in zip(insts, parts, again):
        mu_o, _ = O.moments_doubling(x["H"], x["a"], x["b"], I.rademacher_block(x["seed"], x["H"].n, R),
                                     x["M"])
        assert np.abs(mu - mu_o).max() <= 1e-5
        assert np.array_equal(mu, mu2)


def test_half_chunks_with_rtiles_and_other_lattices(K):
    # R = 16: four 16-byte chunks per row, so four column tiles fit
    insts = instances(6)
    with make_batch(K, insts, "fp32") as bt:
        K.kpm_batch_set_chunk_bytes(bt, 16)
        assert K.kpm_batch_get_rtiles(bt)[2] == 4
        K.kpm_batch_set_rtiles(bt, 4)
        K.kpm_batch_set_config(bt, 2, 2, 100)
        parts = bt.split(K.kpm_batch_run(bt))
        with pytest.raises(K.KPMError) as e:
            K.kpm_batch_set_chunk_bytes(bt, 32)  # 4 tiles do not divide 2 chunks per row
        assert e.value.status == K.KPM_EINVAL
    for x, mu in zip(insts, parts):
        mu_o, _ = O.moments_doubling(x["H"], x["a"], x["b"], I.rademacher_block(x["seed"], x["H"].n, 16),
                                     x["M"])
        assert np.abs(mu - mu_o).max() <= 1e-5
    # a 3D box with an open direction and a 1D chain
    for dims, L, periodic in ((3, (7, 6, 5), (True, True, False)), (1, (61,), (True,))):
        N = int(np.prod(L))
        on = I.onsite_disorder(12 + dims, N, 1.5)
        H = O.lattice_hamiltonian(L, periodic=periodic, onsite=on)
        a, b = O.rescale(*O.gershgorin(H), eps=0.01)
        with K.kpm_create_stencil(dims, L, periodic=periodic, onsite=on) as h:
            with K.kpm_batch_create([h, h], [30, 52], 16, [a, a], [b, b], [3, 4], precision="fp32") as bt:
                K.kpm_batch_set_chunk_bytes(bt, 16)
                K.kpm_batch_set_config(bt, 4, 4, 100)
                got = bt.split(K.kpm_batch_run(bt))
        for M, seed, mu in zip((30, 52), (3, 4), got):
            mu_o, _ = O.moments_doubling(H, a, b, I.rademacher_block(seed, N, 16), M)
            assert np.abs(mu - mu_o).max() <= 1e-5


def test_half_chunks_refusals(K):
    insts = instances(3)
    with make_batch(K, insts, "fp64", 8) as bt:      # FP64 rows always move 16-byte chunks
        assert K.kpm_batch_get_chunk_bytes(bt) == (16, 4)
        with pytest.raises(K.KPMError):
            K.kpm_batch_set_chunk_bytes(bt, 16)
    with make_batch(K, insts, "fp32") as bt:
        for bad in (8, 64):
            with pytest.raises(K.KPMError):
                K.kpm_batch_set_chunk_bytes(bt, bad)
        K.kpm_batch_set_resident(bt, True)
        with pytest.raises(K.KPMError):
            K.kpm_batch_set_chunk_bytes(bt, 16)
        K.kpm_batch_set_resident(bt, False)
        K.kpm_batch_set_chunk_bytes(bt, 16)
        with pytest.raises(K.KPMError):
            K.kpm_batch_set_resident(bt, True)
    L = (12, 10)
    hop = I.spin_hoppings(L, *I.spins(3, 120))
    with K.kpm_create_stencil(2, L, hop=hop, complex_=True) as h:   # complex rows: 32-byte chunks
        with K.kpm_batch_create([h], [8], 16, [9.0], [0.0], [1], precision="fp32") as bt:
            with pytest.raises(K.KPMError):
                K.kpm_batch_set_chunk_bytes(bt, 16)
