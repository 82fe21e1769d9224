"""Seeded synthetic inputs for the kernel polynomial method (KPM) workloads.

This module is the one piece shared by the CUDA path's tests/bench and the
FP64 oracle.  It draws random numbers and lays out model parameters; it holds
none of the KPM arithmetic (no rescaling, no recursion, no moments, no kernel,
no DOS).  Every draw comes from one counter-based generator so that the CUDA
side can regenerate the same numbers independently:

    splitmix64(z):  z += 0x9E3779B97F4A7C15
                    z  = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
                    z  = (z ^ (z >> 27)) * 0x94D049BB133111EB
                    return z ^ (z >> 31)
    u64(seed, stream, counter) = splitmix64((seed ^ (0x9E3779B97F4A7C15 * (1 + stream))) + counter)

(SplitMix64 as published by Steele, Lea and Flood, OOPSLA 2014.)  Streams:
0 random vectors, 1 on-site energies, 2 spin polar angle, 3 spin azimuth,
4 bond dilution, 5 batch instance shapes, 6 Lanczos start vector, 7 dense
matrix entries.

Random vectors follow the paper's stochastic trace (Sec. II-A-3): entries
xi_{r,i} with zero mean and unit variance.  Real vectors are Rademacher +-1
(top bit of u64); complex vectors are unit random phases exp(i 2 pi u) with
u = (u64 >> 11) * 2^-53.  Vector entry (s, r, i) uses counter (s*R + r)*N + i.

Lattice sites are numbered i = x + Lx*(y + Ly*z); bond direction d joins site
i to its forward neighbour i + e_d (periodic wrap when the dimension is
periodic).  The tight-binding model is H_ii = eps_i, H_{i,i+e_d} = -t_{i,d},
H_{i+e_d,i} = conj(H_{i,i+e_d}); the 10x10x10 cubic lattice of the paper's
evaluation (Sec. IV-A: 7 stored entries per row, zero diagonal, -1
off-diagonals) is t = 1, eps = 0, periodic.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_VECTORS = 0
STREAM_ONSITE = 1
STREAM_THETA = 2
STREAM_PHI = 3
STREAM_DILUTION = 4
STREAM_SHAPES = 5
STREAM_LANCZOS = 6
STREAM_DENSE = 7


def splitmix64(z):
    """SplitMix64 output function applied to uint64 array ``z`` (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def u64(seed: int, stream: int, counter):
    """Counter-based 64-bit draw for (seed, stream, counter)."""
    with np.errstate(over="ignore"):
        key = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (GOLDEN * np.uint64(1 + stream))
        return splitmix64(key + np.asarray(counter, dtype=np.uint64))


def uniform(seed: int, stream: int, counter):
    """Uniform double in [0, 1) from the top 53 bits."""
    return (u64(seed, stream, counter) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _vector_counters(N: int, R: int, s: int):
    r = np.arange(R, dtype=np.uint64)[None, :]
    i = np.arange(N, dtype=np.uint64)[:, None]
    return (np.uint64(s) * np.uint64(R) + r) * np.uint64(N) + i


def rademacher_block(seed: int, N: int, R: int, s: int = 0) -> np.ndarray:
    """N x R block (row-major, R contiguous) of +-1 entries, realisation s."""
    bits = u64(seed, STREAM_VECTORS, _vector_counters(N, R, s)) >> np.uint64(63)
    return np.where(bits == 1, -1.0, 1.0)


def phase_block(seed: int, N: int, R: int, s: int = 0) -> np.ndarray:
    """N x R block of unit random phases exp(i 2 pi u), realisation s."""
    phi = 2.0 * np.pi * uniform(seed, STREAM_VECTORS, _vector_counters(N, R, s))
    return np.cos(phi) + 1j * np.sin(phi)


def random_block(seed: int, N: int, R: int, complex_: bool, s: int = 0) -> np.ndarray:
    return phase_block(seed, N, R, s) if complex_ else rademacher_block(seed, N, R, s)


def random_columns(seed: int, N: int, R: int, cols, complex_: bool, s: int = 0) -> np.ndarray:
    """Columns `cols` of the N x R block of realisation s (same counters as random_block)."""
    cols = np.asarray(cols, dtype=np.uint64)
    i = np.arange(N, dtype=np.uint64)[:, None]
    ctr = (np.uint64(s) * np.uint64(R) + cols[None, :]) * np.uint64(N) + i
    z = u64(seed, STREAM_VECTORS, ctr)
    if complex_:
        phi = 2.0 * np.pi * ((z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53))
        return np.cos(phi) + 1j * np.sin(phi)
    return np.where((z >> np.uint64(63)) == 1, -1.0, 1.0)


def lanczos_start(seed: int, N: int) -> np.ndarray:
    """Real Rademacher start vector for the Lanczos bound estimate (stream 6)."""
    bits = u64(seed, STREAM_LANCZOS, np.arange(N, dtype=np.uint64)) >> np.uint64(63)
    return np.where(bits == 1, -1.0, 1.0)


def onsite_disorder(seed: int, N: int, W: float) -> np.ndarray:
    """On-site energies eps_i uniform in [-W/2, W/2)."""
    return W * (uniform(seed, STREAM_ONSITE, np.arange(N, dtype=np.uint64)) - 0.5)


def dense_hermitian(seed: int, n: int, complex_: bool = False) -> np.ndarray:
    """A dense n x n Hermitian matrix with independent entries on and above the
    diagonal (a Wigner matrix), for the paper's dense formulation: H_ij =
    (2u - 1)/sqrt(n) for i <= j (stream 7, counter i*n + j), plus i (2u' - 1)/sqrt(n)
    with u' at counter n*n + i*n + j off the diagonal when complex;
    H_ji = conj(H_ij)."""
    iu, ju = np.triu_indices(n)
    cnt = (iu.astype(np.uint64) * np.uint64(n) + ju.astype(np.uint64))
    scale = 1.0 / np.sqrt(n)
    re = (2.0 * uniform(seed, STREAM_DENSE, cnt) - 1.0) * scale
    if complex_:
        im = (2.0 * uniform(seed, STREAM_DENSE, cnt + np.uint64(n * n)) - 1.0) * scale
        im[iu == ju] = 0.0
        H = np.zeros((n, n), dtype=np.complex128)
        H[iu, ju] = re + 1j * im
        H[ju, iu] = re - 1j * im
    else:
        H = np.zeros((n, n))
        H[iu, ju] = re
        H[ju, iu] = re
    return H


def lattice_sites(L) -> int:
    n = 1
    for l in L:
        n *= int(l)
    return n


def forward_neighbours(L) -> np.ndarray:
    """[N, dims] index of the forward neighbour i + e_d with periodic wrap."""
    L = [int(l) for l in L]
    dims = len(L)
    N = lattice_sites(L)
    idx = np.arange(N, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for d in range(dims):
        coords.append(rem % L[d])
        rem //= L[d]
    out = np.empty((N, dims), dtype=np.int64)
    for d in range(dims):
        c = [x.copy() for x in coords]
        c[d] = (c[d] + 1) % L[d]
        j = np.zeros(N, dtype=np.int64)
        mul = 1
        for e in range(dims):
            j += c[e] * mul
            mul *= L[e]
        out[:, d] = j
    return out


def boundary_bonds(L, periodic) -> np.ndarray:
    """[N, dims] bool: True where the forward bond crosses an open boundary."""
    L = [int(l) for l in L]
    N = lattice_sites(L)
    idx = np.arange(N, dtype=np.int64)
    out = np.zeros((N, len(L)), dtype=bool)
    rem = idx.copy()
    for d in range(len(L)):
        c = rem % L[d]
        rem //= L[d]
        if not periodic[d]:
            out[:, d] = c == L[d] - 1
    return out


def spins(seed: int, N: int):
    """Unit spins uniform on the sphere: cos(theta) = 1 - 2u, phi = 2 pi u'."""
    i = np.arange(N, dtype=np.uint64)
    cos_t = 1.0 - 2.0 * uniform(seed, STREAM_THETA, i)
    theta = np.arccos(np.clip(cos_t, -1.0, 1.0))
    phi = 2.0 * np.pi * uniform(seed, STREAM_PHI, i)
    return theta, phi


def spin_hoppings(L, theta, phi) -> np.ndarray:
    """Forward-bond hoppings of the double-exchange model on lattice L.

    t_ij = cos(th_i/2) cos(th_j/2) + sin(th_i/2) sin(th_j/2) exp(-i (ph_i - ph_j)),
    j = i + e_d.  Returns complex128 [N, dims].
    """
    nb = forward_neighbours(L)
    ci, si = np.cos(theta / 2.0), np.sin(theta / 2.0)
    out = np.empty(nb.shape, dtype=np.complex128)
    for d in range(nb.shape[1]):
        j = nb[:, d]
        out[:, d] = ci * ci[j] + si * si[j] * np.exp(-1j * (phi - phi[j]))
    return out


def dilution_mask(seed: int, N: int, dims: int, p: float = 0.1) -> np.ndarray:
    """[N, dims] bool, True where the forward bond is kept; one draw per undirected
    bond keyed by counter i*dims + d, removed iff u < p."""
    c = np.arange(N * dims, dtype=np.uint64)
    u = uniform(seed, STREAM_DILUTION, c).reshape(N, dims)
    return u >= p


def batch_shapes(seed: int, count: int, L_lo=16, L_hi=128, W_hi=4.0, M_lo=128, M_hi=2048):
    """Instance shapes of a batch of 2D disorder realisations (stream 5):
    L uniform in {L_lo..L_hi}, W uniform in [0, W_hi), M even uniform in {M_lo..M_hi}."""
    k = np.arange(count, dtype=np.uint64)
    uL = uniform(seed, STREAM_SHAPES, 3 * k)
    uW = uniform(seed, STREAM_SHAPES, 3 * k + np.uint64(1))
    uM = uniform(seed, STREAM_SHAPES, 3 * k + np.uint64(2))
    L = L_lo + np.floor(uL * (L_hi - L_lo + 1)).astype(np.int64)
    W = W_hi * uW
    nM = (M_hi - M_lo) // 2 + 1
    M = M_lo + 2 * np.floor(uM * nM).astype(np.int64)
    return L, W, M


def batch_workload(seed: int = 3, count: int = 256, L_lo=16, L_hi=128, M_lo=128, M_hi=2048):
    """Independent 2D disorder realisations of uneven size: L ~ U{L_lo..L_hi},
    W ~ U[0, 4), M even ~ U{M_lo..M_hi} (stream 5), t = 1, periodic, on-site
    energies from stream 1 with seed (seed * 1000003 + k), R = 16 Rademacher
    vectors with seed (seed * 7919 + k)."""
    Ls, Ws, Ms = batch_shapes(seed, count, L_lo, L_hi, 4.0, M_lo, M_hi)
    out = []
    for k in range(count):
        L = (int(Ls[k]), int(Ls[k]))
        out.append(dict(dims=2, L=L, periodic=(True, True), W=float(Ws[k]), M=int(Ms[k]),
                        onsite=onsite_disorder(seed * 1000003 + k, L[0] * L[1], float(Ws[k])),
                        R=16, seed=seed * 7919 + k))
    return out


def serving_stream(seed: int = 5, count: int = 64, rate_hz: float = 50.0, N_lo=1e3, N_hi=4e6,
                   M_lo=256, M_hi=8192, Rs=(8, 16, 32, 64)):
    """Poisson stream of DOS requests (stream 5, counters 1000000 + 8k + j):
    arrival gaps exponential with the given rate; 2D or 3D cubic lattice with
    N log-uniform in [N_lo, N_hi] (side rounded, at least 4); M even and
    log-uniform in [M_lo, M_hi]; R uniform in Rs; real or complex spin
    hoppings (real: all azimuths 0); spins from seed 1000 + k."""
    out = []
    t = 0.0
    for k in range(count):
        c = 1000000 + 8 * np.arange(7, dtype=np.uint64) + np.uint64(8 * k)
        u = uniform(seed, STREAM_SHAPES, c)
        t += -np.log(1.0 - u[0]) / rate_hz
        dims = 2 if u[1] < 0.5 else 3
        N = float(np.exp(np.log(N_lo) + u[2] * (np.log(N_hi) - np.log(N_lo))))
        side = max(4, int(round(N ** (1.0 / dims))))
        M = int(np.exp(np.log(M_lo) + u[3] * (np.log(M_hi) - np.log(M_lo))))
        M += M % 2
        R = int(Rs[min(int(u[4] * len(Rs)), len(Rs) - 1)])
        cplx = bool(u[5] < 0.5)
        out.append(dict(t=t, dims=dims, L=(side,) * dims, M=M, R=R, complex=cplx, spin_seed=1000 + k,
                        seed=7000 + k))
    return out


def workload(name: str, seed: int | None = None) -> dict:
    """Hamiltonian inputs for the named synthetic workload.

    Returns dict(dims, L, periodic, onsite (or None), hop (or None => uniform t),
    t, complex, mask (or None), R, M, seed).
    """
    if name == "square_L32_fp64":
        # 2D square lattice L=32, t=1, eps ~ U[-0.5, 0.5], M=256, R=8 Rademacher
        seed = 1 if seed is None else seed
        L = (32, 32)
        N = lattice_sites(L)
        return dict(dims=2, L=L, periodic=(True, True), onsite=onsite_disorder(seed, N, 1.0),
                    hop=None, t=1.0, complex=False, mask=None, R=8, M=256, seed=seed, K=1024)
    if name.startswith("csr_spin_dilute_L"):
        # 3D cubic lattice, spin hoppings, 10% bond dilution, handled as CSR:
        # R=32 complex vectors, M=4096
        Lc = int(name[len("csr_spin_dilute_L"):])
        seed = 4 if seed is None else seed
        L = (Lc, Lc, Lc)
        N = lattice_sites(L)
        th, ph = spins(seed, N)
        return dict(dims=3, L=L, periodic=(True, True, True), onsite=None,
                    hop=spin_hoppings(L, th, ph), t=1.0, complex=True,
                    mask=dilution_mask(seed, N, 3, 0.1), R=32, M=4096, seed=seed, K=4096)
    if name.startswith("cubic_spin_L"):
        # 3D cubic lattice with spin-derived complex hoppings, random-phase vectors
        Lc = int(name[len("cubic_spin_L"):].split("_")[0])
        seed = 2 if seed is None else seed
        L = (Lc, Lc, Lc)
        N = lattice_sites(L)
        th, ph = spins(seed, N)
        return dict(dims=3, L=L, periodic=(True, True, True), onsite=None,
                    hop=spin_hoppings(L, th, ph), t=1.0, complex=True, mask=None,
                    R=64, M=1024, seed=seed, K=1024)
    if name.startswith("dense_wigner_D"):
        # the paper's dense formulation at its largest matrix (Sec. IV-C: H_SIZE
        # up to 4096, N = 128 moments, R x S = 14 x 128 = 1792 random vectors):
        # a real Wigner matrix, FP64, all 1792 vectors in one block
        D = int(name[len("dense_wigner_D"):])
        seed = 8 if seed is None else seed
        return dict(D=D, H=dense_hermitian(seed, D), complex=False, R=1792, M=128, seed=seed,
                    K=1024)
    raise KeyError(name)
