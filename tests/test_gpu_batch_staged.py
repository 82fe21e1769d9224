"""The staged form of the batched persistent launch (vector tiles brought into
shared memory by bulk asynchronous copies): every instance against the FP64
oracle at the parity tolerances, at every cluster size and tile size; the
same instance bitwise alone and in a mix for a fixed configuration; lattices
whose neighbour rows fall outside the halo the rings hold (read from global
memory), complex hoppings, open edges, 1D chains and instances smaller than
one tile or than the cluster's CTAs; and the refusals."""
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


def square_instances(n=10, seed=31):
    """2D disorder realisations of uneven size, a few of them smaller than
    one tile of rows (the batch workload scaled down)."""
    rng = np.random.default_rng(seed)
    Ls = [5, 8, 13, 16, 24, 33, 7, 40, 11, 20, 3, 48][:n]
    out = []
    for k, L in enumerate(Ls):
        on = I.onsite_disorder(seed * 1000 + k, L * L, float(rng.uniform(0, 4)))
        M = int(2 * rng.integers(8, 70))
        H = O.lattice_hamiltonian((L, L), onsite=on)
        a, b = O.rescale(*O.gershgorin(H), eps=0.01)
        out.append(dict(dims=2, L=(L, L), kw=dict(onsite=on), M=M, H=H, a=a, b=b,
                        seed=seed * 100 + k))
    return out


def run_staged(K, insts, prec, R, C, chunk=2, complex_=False):
    hs = [K.kpm_create_stencil(x["dims"], x["L"], complex_=complex_, **x["kw"]) for x in insts]
    with K.kpm_batch_create(hs, [x["M"] for x in insts], R, [x["a"] for x in insts],
                            [x["b"] for x in insts], [x["seed"] for x in insts], precision=prec) as bt:
        K.kpm_batch_set_config(bt, C, chunk, 100)
        K.kpm_batch_set_staged(bt, True)
        assert K.kpm_batch_get_staged(bt)[0]
        parts = bt.split(K.kpm_batch_run(bt))
    for h in hs:
        h.close()
    return parts


def oracle_mu(x, R, complex_=False):
    v0 = (I.phase_block if complex_ else I.rademacher_block)(x["seed"], x["H"].n, R)
    return O.moments_doubling(x["H"], x["a"], x["b"], v0, x["M"])[0]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("C", [1, 2, 4, 8, 16])
def test_staged_instances_match_oracle(K, prec, C):
    insts = square_instances()
    R = 16
    parts = run_staged(K, insts, prec, R, C)
    for x, mu in zip(insts, parts):
        assert np.abs(mu - oracle_mu(x, R)).max() <= TOL[prec], (x["L"], C)


@pytest.mark.parametrize("chunk", [1, 4])
@pytest.mark.parametrize("R", [8, 13, 32])
def test_staged_tile_sizes_and_widths(K, chunk, R):
    # tiles of about 4 and 16 KB; R = 8 (one chunk per row), 13 (padded
    # columns), 32 (four chunks per row)
    insts = square_instances(8, seed=37)
    parts = run_staged(K, insts, "fp32", R, 4, chunk=chunk)
    for x, mu in zip(insts, parts):
        assert np.abs(mu - oracle_mu(x, R)).max() <= TOL["fp32"]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_staged_alone_and_in_the_mix_is_bitwise_identical(K, prec):
    insts = square_instances()
    for C in (1, 4):
        mix = run_staged(K, insts, prec, 16, C)
        for k in (0, 5, 7, 9):
            alone = run_staged(K, [insts[k]], prec, 16, C)[0]
            assert np.array_equal(alone, mix[k]), (k, C)


@pytest.mark.parametrize("prec,R", [("fp32", 16), ("fp64", 8)])
def test_staged_3d_complex_open_edges_beyond_the_halo(K, prec, R):
    # 3D lattices with spin-derived complex hoppings, dilution-free, one open
    # direction; the largest has planes of 900 rows, more than the rings hold
    # on either side of a tile, so its z-neighbours are read from global memory
    out = []
    for k, (L, per) in enumerate([((30, 30, 6), (True, True, False)), ((9, 7, 5), (True, False, True)),
                                  ((4, 4, 4), (True, True, True)), ((17, 3, 11), (False, True, True))]):
        N = int(np.prod(L))
        hop = I.spin_hoppings(L, *I.spins(70 + k, N))
        on = I.onsite_disorder(80 + k, N, 1.5)
        H = O.lattice_hamiltonian(L, periodic=per, onsite=on, hop=hop)
        a, b = O.rescale(*O.gershgorin(H), eps=0.01)
        out.append(dict(dims=3, L=L, kw=dict(periodic=per, onsite=on, hop=hop), M=2 * (20 + 7 * k),
                        H=H, a=a, b=b, seed=500 + k))
    for C in (1, 4):
        parts = run_staged(K, out, prec, R, C, complex_=True)
        for x, mu in zip(out, parts):
            assert np.abs(mu - oracle_mu(x, R, True)).max() <= TOL[prec], (x["L"], C)


@pytest.mark.parametrize("periodic", [True, False])
def test_staged_chains(K, periodic):
    # 1D chains of 1000 and 301 sites: the periodic wrap joins the first and
    # last tiles, read from global memory unless both are in the halo
    out = []
    for k, n in enumerate([1000, 301, 64]):
        on = I.onsite_disorder(90 + k, n, 1.0)
        H = O.lattice_hamiltonian((n,), periodic=(periodic,), onsite=on)
        a, b = O.rescale(*O.gershgorin(H), eps=0.01)
        out.append(dict(dims=1, L=(n,), kw=dict(periodic=(periodic,), onsite=on), M=96, H=H, a=a, b=b,
                        seed=600 + k))
    for C in (1, 2, 8):
        parts = run_staged(K, out, "fp32", 16, C)
        for x, mu in zip(out, parts):
            assert np.abs(mu - oracle_mu(x, 16)).max() <= TOL["fp32"], (x["L"], C)


def test_staged_uniform_operator_without_onsite(K):
    # clean square lattices (no on-site array): the stream ring carries
    # nothing on the first product
    out = []
    for k, L in enumerate([12, 35, 64]):
        H = O.lattice_hamiltonian((L, L))
        a, b = O.rescale(*O.gershgorin(H), eps=0.01)
        out.append(dict(dims=2, L=(L, L), kw={}, M=64, H=H, a=a, b=b, seed=700 + k))
    parts = run_staged(K, out, "fp32", 16, 2)
    for x, mu in zip(out, parts):
        assert np.abs(mu - oracle_mu(x, 16)).max() <= TOL["fp32"]


def test_staged_agrees_with_the_global_memory_form(K):
    insts = square_instances()
    parts = run_staged(K, insts, "fp64", 16, 4)
    hs = [K.kpm_create_stencil(2, x["L"], **x["kw"]) for x in insts]
    with K.kpm_batch_create(hs, [x["M"] for x in insts], 16, [x["a"] for x in insts],
                            [x["b"] for x in insts], [x["seed"] for x in insts], precision="fp64") as bt:
        K.kpm_batch_set_config(bt, 4, 2, 100)
        ref = bt.split(K.kpm_batch_run(bt))
    for h in hs:
        h.close()
    for a_, b_ in zip(parts, ref):
        assert np.abs(a_ - b_).max() <= 1e-12


def test_staged_refusals(K):
    x = square_instances(1)[0]
    h = K.kpm_create_stencil(2, x["L"], **x["kw"])
    with K.kpm_batch_create([h], [x["M"]], 16, [x["a"]], [x["b"]], [1], precision="fp32") as bt:
        K.kpm_batch_set_rtiles(bt, 2)
        K.kpm_batch_set_staged(bt, True)
        assert K.kpm_batch_get_rtiles(bt)[0] == 1        # setting it cleared the R-tiling
        with pytest.raises(K.KPMError):
            K.kpm_batch_set_rtiles(bt, 2)
        K.kpm_batch_set_staged(bt, False)
        assert not K.kpm_batch_get_staged(bt)[0]
        K.kpm_batch_set_chunk_bytes(bt, 16)
        with pytest.raises(K.KPMError):
            K.kpm_batch_set_staged(bt, True)              # 16-byte chunks
    # rows wider than 32 chunks
    with K.kpm_batch_create([h], [x["M"]], 80, [x["a"]], [x["b"]], [1], precision="fp64") as bt:
        with pytest.raises(K.KPMError):
            K.kpm_batch_set_staged(bt, True)
    h.close()
    # CSR operators
    rp, col, val = K.kpm_stencil_to_csr(2, x["L"], **x["kw"])
    with K.kpm_create_csr(rp.size - 1, rp, col, val) as hc:
        with K.kpm_batch_create([hc], [x["M"]], 16, [x["a"]], [x["b"]], [1], precision="fp32") as bt:
            with pytest.raises(K.KPMError):
                K.kpm_batch_set_staged(bt, True)
