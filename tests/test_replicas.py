"""The multi-process (replica) path on CPU with gloo, world size 2: each rank
runs its own realisation of the random vectors (here with the oracle, as a
stand-in for its GPU), and the combined moments equal one run over the union
of the vectors."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import oracle as O
    from paper_1105_5481_gb300 import inputs as I
    from paper_1105_5481_gb300.replicas import combine_moments

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L, R, M, seed = (6, 5), 3 + rank, 64, 17   # uneven vector counts per rank
    H = O.lattice_hamiltonian(L, onsite=I.onsite_disorder(2, 30, 1.5))
    a, b = O.rescale(*O.gershgorin(H))
    # rank k owns vectors k*3 .. k*3 + R - 1 of one generator sequence
    cols = np.arange(3 * rank, 3 * rank + R)
    mu, _ = O.moments_doubling(H, a, b, I.random_columns(seed, H.n, 7, cols, False), M)
    comb = combine_moments(mu, R)
    if rank == 0:
        ref, _ = O.moments_doubling(H, a, b, I.random_columns(seed, H.n, 7, np.arange(7), False), M)
        out.put(float(np.abs(comb - ref).max()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_combine_to_the_union_of_their_vectors():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    err = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert err < 1e-14
