"""The multi-process (replica) form on the GPU: two processes, each with its
own CUDA context on cuda:0, run one realisation each of the same seed through
the C ABI (kpm_params.s0 = rank) and combine their moments with one gloo
all-reduce of M + 1 doubles (the vector-weighted mean of Eq. (munr) over the
union of their vectors).  The result must equal one kpm_moments call with
S = 2 to rounding and the FP64 oracle on the union of the vectors within the
parity tolerances.  The two processes' kernels never wait on one another."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as O
from paper_1105_5481_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::DeprecationWarning")]

L, R, M, SEED = (8, 7, 6), 6, 256, 23
TOL = {"fp64": 1e-10, "fp32": 1e-5}


def _lattice():
    N = int(np.prod(L))
    return dict(dims=3, L=L, hop=I.spin_hoppings(L, *I.spins(9, N)),
                onsite=I.onsite_disorder(9, N, 1.0)), N


def _rank(rank, world, port, prec, a, b, out):
    import torch
    import torch.distributed as dist

    from paper_1105_5481_gb300 import kpm as K
    from paper_1105_5481_gb300.replicas import combine_moments

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    kw, _ = _lattice()
    with K.kpm_create_stencil(complex_=True, **kw) as h:
        mu = K.kpm_moments(h, M, R, a, b, seed=SEED, s0=rank, precision=prec)
    comb = combine_moments(mu, R)
    if rank == 0:
        out.put(comb)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_two_gpu_processes_combine_to_one_two_realisation_run(gpu_lib, prec):
    from paper_1105_5481_gb300 import kpm as K

    kw, N = _lattice()
    H = O.lattice_hamiltonian(kw["L"], onsite=kw["onsite"], hop=kw["hop"])
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, prec, a, b, q)) for r in range(2)]
    for p in procs:
        p.start()
    comb = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    with K.kpm_create_stencil(complex_=True, **kw) as h:
        one = K.kpm_moments(h, M, R, a, b, seed=SEED, S=2, precision=prec)
    assert np.abs(comb - one).max() <= 1e-13
    union = np.concatenate([I.random_block(SEED, N, R, True, s=s) for s in range(2)], axis=1)
    mu_o, _ = O.moments_doubling(H, a, b, union, M)
    assert np.abs(comb - mu_o).max() <= TOL[prec]


def test_first_realisation_index_selects_the_realisation(gpu_lib):
    # realisation s0 alone equals the s0-th realisation of a longer run
    from paper_1105_5481_gb300 import kpm as K

    kw, N = _lattice()
    H = O.lattice_hamiltonian(kw["L"], onsite=kw["onsite"], hop=kw["hop"])
    a, b = O.rescale(*O.gershgorin(H), eps=0.01)
    with K.kpm_create_stencil(complex_=True, **kw) as h:
        _, pv3 = K.kpm_moments(h, 64, R, a, b, seed=SEED, S=3, per_vec=True)
        _, pv2 = K.kpm_moments(h, 64, R, a, b, seed=SEED, S=1, s0=2, per_vec=True)
        with pytest.raises(K.KPMError) as e:
            K.kpm_moments(h, 64, R, a, b, seed=SEED, s0=-1)
        assert e.value.status == K.KPM_EINVAL
    assert np.array_equal(pv2, pv3[2 * R:3 * R])
    mu_o, _ = O.moments_doubling(H, a, b, I.random_block(SEED, N, R, True, s=2), 64)
    assert np.abs(pv2.mean(axis=0) - mu_o).max() <= TOL["fp64"]
