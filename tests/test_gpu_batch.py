"""The batched persistent launch: every instance against the oracle, the same
instance alone and in a mix (bitwise, for a fixed cluster size), all cluster
sizes, and the autotuner with its on-disk cache."""
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


def test_autotuner_writes_and_reuses_its_cache(K, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("KPM_TUNE_CACHE", str(cache))
    insts = instances(6)
    with make_batch(K, insts, "fp32") as bt:
        info = K.kpm_batch_tune(bt, reps=1)
        mu = K.kpm_batch_run(bt)
    text = cache.read_text()
    assert "batch|" in text and f"= {info['cluster']} {info['chunk']}" in text
    with make_batch(K, insts, "fp32") as bt2:
        info2 = K.kpm_batch_info(bt2)
        mu2 = K.kpm_batch_run(bt2)
    assert (info2["cluster"], info2["chunk"]) == (info["cluster"], info["chunk"])
    assert np.array_equal(mu, mu2)
