"""The serving loop: a stream of mixed requests submitted while others run
(continuous batching), each result bitwise identical to the same request
served alone and within tolerance of the oracle; admission under an HBM
budget; cancellation leaving the others unchanged."""
import threading

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


def request_mix():
    """(kind, L, M, R, precision, seed): 2D/3D, real/complex spin hoppings, several R,
    and one request large enough for the full-GPU path (3D L = 52: 140,608 sites)."""
    return [
        ("real", (24, 24), 128, 8, "fp32", 1), ("cplx", (16, 16), 96, 16, "fp32", 2),
        ("real", (6, 7, 5), 64, 8, "fp64", 3), ("cplx", (8, 8, 8), 200, 32, "fp32", 4),
        ("real", (40, 40), 256, 16, "fp32", 5), ("cplx", (10, 9, 8), 64, 8, "fp64", 6),
        ("real", (52, 52, 52), 48, 8, "fp32", 7), ("cplx", (31, 17), 150, 8, "fp32", 8),
        ("real", (12, 12), 512, 64, "fp32", 9), ("cplx", (5, 5, 5), 40, 16, "fp64", 10),
    ]


def build(K, kind, L, seed):
    N = int(np.prod(L))
    th, ph = I.spins(seed, N)
    if kind == "real":
        ph = np.zeros(N)
    hop = I.spin_hoppings(L, th, ph)
    cplx = kind == "cplx"
    h = K.kpm_create_stencil(len(L), L, hop=hop if cplx else hop.real, complex_=cplx)
    H = O.lattice_hamiltonian(L, hop=hop if cplx else hop.real)
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    return h, H, a, b


def serve(K, items, budget=2 << 30, threads=2, cancel=None):
    srv = K.kpm_server_create(budget, steps_per_tick=16, cluster=4)
    ids = [None] * len(items)

    def submit(rng):
        for k in rng:
            h, M, R, a, b, prec, seed, Kn = items[k]
            ids[k] = K.kpm_server_submit(srv, h, M, R, a, b, seed=seed, precision=prec, K=Kn)

    ts = [threading.Thread(target=submit, args=(range(j, len(items), threads),)) for j in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if cancel is not None:
        K.kpm_server_cancel(srv, ids[cancel])
    out = []
    for k, rid in enumerate(ids):
        K.kpm_server_wait(srv, rid, 120.0)
        if k == cancel:
            with pytest.raises(K.KPMError):
                K.kpm_server_poll(srv, rid)
            out.append(None)
        else:
            out.append(K.kpm_server_poll(srv, rid))
    stats = K.kpm_server_stats(srv)
    srv.close()
    return out, stats


def test_mixed_stream_same_alone_and_in_mix_and_matches_oracle(K):
    mix = request_mix()
    built = [build(K, kind, L, seed) for kind, L, M, R, prec, seed in mix]
    items = [(b_[0], m[2], m[3], b_[2], b_[3], m[4], m[5], 64) for b_, m in zip(built, mix)]
    res, stats = serve(K, items)
    assert stats["completed"] == len(items) and stats["failed"] == 0
    assert stats["p99_s"] >= stats["p50_s"] > 0
    for k, (item, m) in enumerate(zip(items, mix)):
        alone, _ = serve(K, [item], threads=1)
        assert np.array_equal(alone[0][0], res[k][0]), f"request {k} differs alone and in the mix"
        assert np.array_equal(alone[0][2], res[k][2])
        # every request against the oracle, the full-GPU L = 52^3 one included
        H, a, b = built[k][1], built[k][2], built[k][3]
        v0 = I.random_block(m[5], H.n, m[3], m[0] == "cplx")
        mu_o, _ = O.moments_doubling(H, a, b, v0, m[2])
        assert np.abs(res[k][0] - mu_o).max() <= TOL[m[4]], k
        E_ref, rho_ref = K.kpm_dos(res[k][0], item[3], item[4], 64)
        assert np.abs(res[k][2] - rho_ref).max() <= 1e-12 * np.abs(rho_ref).max()
    for b_ in built:
        b_[0].close()


def test_admission_under_a_small_budget_and_cancel(K):
    mix = [m for m in request_mix() if m[1] != (52, 52, 52)]
    built = [build(K, kind, L, seed) for kind, L, M, R, prec, seed in mix]
    items = [(b_[0], m[2], m[3], b_[2], b_[3], m[4], m[5], 0) for b_, m in zip(built, mix)]
    full, _ = serve(K, items)
    small = 1 << 20                       # a few requests at a time
    res, stats = serve(K, items, budget=small, cancel=3)
    assert stats["peak_bytes"] <= stats["budget_bytes"] == small
    assert stats["peak_resident"] < len(items)
    assert stats["cancelled"] == 1 and stats["completed"] == len(items) - 1
    for k in range(len(items)):
        if k != 3:
            assert np.array_equal(res[k][0], full[k][0])
    with pytest.raises(K.KPMError) as e:
        srv = K.kpm_server_create(1 << 20, 16, 4)
        K.kpm_server_submit(srv, built[4][0], 4096, 64, built[4][2], built[4][3])
    assert e.value.status == K.KPM_ENOMEM
    srv.close()
    for b_ in built:
        b_[0].close()


def test_cancel_a_large_request_in_flight_returns_its_memory(K):
    import time

    # 3D L = 52 with R = 64: a full-GPU request (its products run on the large
    # requests' streams, chunk after chunk, while the scheduler only polls)
    h, H, a, b = build(K, "real", (52, 52, 52), 7)
    M, R = 65536, 64
    srv = K.kpm_server_create(2 << 30, 16, 4)
    rid = K.kpm_server_submit(srv, h, M, R, a, b, seed=1)
    K.kpm_server_wait(srv, rid, 300.0)
    ref = K.kpm_server_poll(srv, rid)[0]
    one = K.kpm_server_stats(srv)["peak_bytes"]
    srv.close()
    # a budget for one such request at a time
    srv = K.kpm_server_create(int(one * 1.5), 16, 4)
    big = K.kpm_server_submit(srv, h, M, R, a, b, seed=2)
    time.sleep(0.15)  # a fraction of its 32768 products
    K.kpm_server_cancel(srv, big)
    K.kpm_server_wait(srv, big, 300.0)
    with pytest.raises(K.KPMError):
        K.kpm_server_poll(srv, big)
    # its memory has come back: the same footprint is admitted and completes,
    # with the moments of the same request served alone
    again = K.kpm_server_submit(srv, h, M, R, a, b, seed=1)
    K.kpm_server_wait(srv, again, 300.0)
    mu = K.kpm_server_poll(srv, again)[0]
    assert np.array_equal(mu, ref)
    st = K.kpm_server_stats(srv)
    assert st["cancelled"] == 1 and st["completed"] == 1 and st["peak_bytes"] <= int(one * 1.5)
    srv.close()
    h.close()
