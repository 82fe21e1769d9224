"""Plain, slow, FP64 CPU oracle of the kernel polynomial method (KPM).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports or calls this
module; only the tests, the smoke check and the benchmark's CPU-baseline leg
do.  It shares no code with the CUDA path: it builds its own lattice
Hamiltonian, runs its own recursion and reduction, and takes every random
number (the random vectors, the Lanczos start vector) as an input array.

Every function follows the paper (Zhang, Yamagiwa, Okumura, Yunoki,
"Performance Acceleration of Kernel Polynomial Method Applying Graphics
Processing Units", arXiv:1105.5481), Sec. II-A, and, where the paper only
names a piece, the KPM review it cites (Weisse, Wellein, Alvermann, Fehske,
Rev. Mod. Phys. 78, 275 (2006)):

  from_dense             the paper's dense formulation: all n*n elements of H
                         stored (Sec. II-A-4 without CRS)                      [pinned]
  exact_moments          Eq. (DoStr): mu_n = (1/D) Tr T_n(H~), via eigh      [pinned]
  moments_direct         Eqs. (rn), (munr): r_{n+2} = 2 H~ r_{n+1} - r_n,
                         mu_n = <<(1/DR) sum_r <r_0|r_n>>>                     [pinned]
  moments_doubling       same estimator, two moments per product via
                         mu_2n = 2<v_n|v_n> - mu_0, mu_2n+1 = 2<v_n+1|v_n> - mu_1
                         (review Eq. 34)                                        [pinned]
  jackson_kernel         review Eq. 71 (the paper names it in Sec. I)          [pinned]
  dos                    Eq. (fKPM) on the Chebyshev nodes x_k = cos(pi(k+1/2)/K),
                         rho(E) = f(x)/a with E = a x + b                       [pinned]
  gershgorin             Eq. (tilde) bounds from the Gershgorin theorem         [pinned]
  lanczos_bounds         k-step Lanczos with full reorthogonalisation, Ritz
                         value +- residual |beta_k s_k|, clamped to Gershgorin  [pinned]
  rescale                Eq. (tilde): a = (Emax-Emin)/(2-eps), b = (Emax+Emin)/2  [pinned]
  lorentz_kernel         review Eq. 74: g_n = sinh(lambda (1 - n/M)) / sinh(lambda)  [pinned]
  green                  local Green's function by the review's expansion
                         G(x+i0) = -i/sqrt(1-x^2) [g_0 mu_0 + 2 sum g_n mu_n e^{-in arccos x}] [pinned]
  thermo                 Fermi-occupation integrals of the DOS (n, u, s, c per
                         site) by the Gauss-Chebyshev rule on the DOS nodes       [pinned]
  ldos_exact             local moments <i|T_n(H~)|i> = sum_k |U_ik|^2 T_n(E~_k)
                         (the KPM review's local DOS, a unit start vector)      [pinned]
  plane_waves            e^{i k.x} on the lattice sites (site i = x0 + L0 (x1 + L1 x2)),
                         the start vectors of momentum-resolved moments          [pinned]
  spectral_exact         <k|T_n(H~)|k> = sum_m |<k|u_m>|^2 T_n(E~_m) for the
                         normalised plane wave |k> (the review's spectral
                         function A(k, E) expanded in Chebyshev moments)         [pinned]
  dos_many, stats        the DOS of each vector's moments (Eq. (fKPM)), and the
                         mean and standard error over the independent vectors
                         of the moments and of the DOS (the spread behind the
                         average of Eq. (munr))                                 [pinned]

Notation: N = matrix dimension (the paper's D), M = number of moments (the
paper's N), R = random vectors per realisation.  All arithmetic is float64 /
complex128.  Every function listed above is pinned by tests that do not
re-use the oracle's own formulas (closed forms, library routines, brute force).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "CSR", "lattice_hamiltonian", "dense", "from_dense", "gershgorin", "lanczos_bounds", "rescale",
    "moments_direct", "moments_doubling", "exact_moments", "jackson_kernel", "dos",
    "lorentz_kernel", "damping", "dos_many", "stats", "dos_error_integral", "ldos_exact",
    "green", "thermo", "plane_waves", "spectral_exact",
]


class CSR:
    """Compressed row storage of an N x N Hermitian matrix (the paper's CRS, Sec. II-A-4)."""

    def __init__(self, n, rowptr, col, val):
        self.n = int(n)
        self.rowptr = np.asarray(rowptr, dtype=np.int64)
        self.col = np.asarray(col, dtype=np.int64)
        self.val = np.asarray(val)
        self._row = np.repeat(np.arange(self.n), np.diff(self.rowptr))

    @property
    def nnz(self) -> int:
        return int(self.col.size)

    @property
    def is_complex(self) -> bool:
        return np.iscomplexobj(self.val)

    def matvec(self, X: np.ndarray) -> np.ndarray:
        """Y = H X for an N x R block X (row i of Y = sum_j H_ij X_j)."""
        X = np.asarray(X)
        prod = self.val[:, None] * X[self.col]
        dtype = np.result_type(self.val, X)
        Y = np.zeros((self.n, X.shape[1]), dtype=dtype)
        nonempty = np.flatnonzero(np.diff(self.rowptr) > 0)
        if nonempty.size:
            Y[nonempty] = np.add.reduceat(prod, self.rowptr[nonempty], axis=0)
        return Y


def lattice_hamiltonian(L, periodic=None, onsite=None, hop=None, t=1.0, mask=None) -> CSR:
    """Tight-binding Hamiltonian on a hypercubic lattice (paper Sec. IV-A example).

    Sites i = x_0 + L_0 (x_1 + L_1 x_2); for each site and direction d the
    forward bond joins i to the site with x_d -> x_d + 1 (wrapping when
    periodic[d], absent at the open edge otherwise).  H_ii = onsite_i,
    H_{i,j} += -t_{i,d}, H_{j,i} += -conj(t_{i,d}); hop[i, d] overrides the
    uniform t, mask[i, d] == False removes the bond.  Repeated (i, j) pairs
    (L_d = 1 or 2 with wrap) add up.
    """
    L = [int(l) for l in L]
    dims = len(L)
    periodic = [True] * dims if periodic is None else [bool(p) for p in periodic]
    N = 1
    for l in L:
        N *= l
    rows, cols, vals = [], [], []
    if onsite is not None:
        rows.append(np.arange(N))
        cols.append(np.arange(N))
        vals.append(np.asarray(onsite, dtype=np.float64).astype(np.complex128))
    site = np.arange(N)
    coord = []
    rem = site.copy()
    for d in range(dims):
        coord.append(rem % L[d])
        rem = rem // L[d]
    stride = [1] * dims
    for d in range(1, dims):
        stride[d] = stride[d - 1] * L[d - 1]
    for d in range(dims):
        x = coord[d]
        xn = x + 1
        keep = np.ones(N, dtype=bool)
        if periodic[d]:
            xn = xn % L[d]
        else:
            keep &= xn < L[d]
        if mask is not None:
            keep &= np.asarray(mask)[:, d].astype(bool)
        j = site + (xn - x) * stride[d]
        h = np.full(N, complex(t)) if hop is None else np.asarray(hop)[:, d].astype(np.complex128)
        i_k, j_k, h_k = site[keep], j[keep], h[keep]
        rows += [i_k, j_k]
        cols += [j_k, i_k]
        vals += [-h_k, -np.conj(h_k)]
    r = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    v = np.concatenate(vals) if vals else np.zeros(0, np.complex128)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    if r.size:
        first = np.ones(r.size, dtype=bool)
        first[1:] = (r[1:] != r[:-1]) | (c[1:] != c[:-1])
        starts = np.flatnonzero(first)
        v = np.add.reduceat(v, starts)
        r, c = r[starts], c[starts]
    rowptr = np.zeros(N + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    is_cplx = (hop is not None and np.iscomplexobj(hop)) or isinstance(t, complex)
    return CSR(N, rowptr, c, v if is_cplx else v.real.copy())


def dense(H: CSR) -> np.ndarray:
    A = np.zeros((H.n, H.n), dtype=H.val.dtype)
    A[H._row, H.col] += H.val
    return A


def from_dense(A) -> CSR:
    """The paper's dense formulation (Sec. II-A-4, CRS not applied): every one
    of the n*n elements of H, zeros included, is stored and takes part in
    every product."""
    A = np.asarray(A)
    n = A.shape[0]
    rowptr = np.arange(n + 1, dtype=np.int64) * n
    col = np.tile(np.arange(n, dtype=np.int64), n)
    return CSR(n, rowptr, col, A.reshape(-1).copy())


def green(mu, a: float, b: float, K: int, kernel: str = "lorentz", lam: float = 4.0):
    """Local Green's function on the K Chebyshev nodes by the KPM review's expansion
    (Eq. 86 there), by a direct double sum:
      G(x_k + i0) = -i/sqrt(1 - x_k^2) [g_0 mu_0 + 2 sum_{n=1}^{M-1} g_n mu_n e^{-i n theta_k}],
    theta_k = pi (k + 1/2)/K, x_k = cos theta_k, in energy units (divided by a).
    Returns (E[K], G[K] complex)."""
    mu = np.asarray(mu, dtype=np.float64)
    M = mu.size
    g = damping(M, kernel, lam)
    th = math.pi * (np.arange(K) + 0.5) / K
    G = np.empty(K, dtype=np.complex128)
    for k in range(K):
        s = complex(g[0] * mu[0])
        for n in range(1, M):
            s += 2.0 * g[n] * mu[n] * complex(math.cos(n * th[k]), -math.sin(n * th[k]))
        G[k] = -1j * s / math.sin(th[k]) / a
    return a * np.cos(th) + b, G


def thermo(mu, a: float, b: float, K: int, betas, mu_c: float = 0.0, kernel: str = "jackson",
           lam: float = 0.0):
    """For each inverse temperature beta (inf: ground state), with the Fermi
    occupation f = 1/(1 + exp(beta (E - mu_c))), the integrals per site
      n = int rho f,  u = int E rho f,  s = -int rho [f ln f + (1-f) ln(1-f)],
      c = beta^2 int rho (E - mu_c)^2 f (1-f)
    by the Gauss-Chebyshev rule on the K nodes of dos():
    int g rho dE = sum_k g(E_k) rho_k a pi sqrt(1 - x_k^2) / K.  Returns [nT, 4]."""
    E, rho = dos(mu, a, b, K, kernel, lam)
    w = a * math.pi * np.sin(math.pi * (np.arange(K) + 0.5) / K) / K
    out = []
    for beta in np.atleast_1d(betas):
        d = E - mu_c
        if math.isinf(beta):
            f = np.where(d < 0, 1.0, np.where(d > 0, 0.0, 0.5))
            ent = np.zeros(K)
            cv = np.zeros(K)
        else:
            x = beta * d
            f = 1.0 / (1.0 + np.exp(x))
            with np.errstate(divide="ignore", invalid="ignore"):
                ent = -(np.where(f > 0, f * np.log(f), 0.0) +
                        np.where(f < 1, (1 - f) * np.log1p(-f), 0.0))
            cv = x * x * f * (1 - f)
        out.append([np.sum(w * rho * f), np.sum(w * rho * E * f), np.sum(w * rho * ent),
                    np.sum(w * rho * cv)])
    return np.array(out)


def dos_many(P, a: float, b: float, K: int, kernel: str = "jackson", lam: float = 0.0):
    """Eq. (fKPM) for each row of P[nvec, M] (the moments of one vector each):
    the same series as dos(), with the node sums done as one matrix product
    against T[n, k] = cos(n pi (k + 1/2) / K).  Returns (E[K], rho[nvec, K])."""
    P = np.atleast_2d(np.asarray(P, dtype=np.float64))
    M = P.shape[1]
    g = damping(M, kernel, lam) * np.where(np.arange(M) == 0, 1.0, 2.0)
    phase = math.pi * (np.arange(K) + 0.5) / K
    T = np.cos(np.arange(M)[:, None] * phase[None, :])
    f = (P * g[None, :]) @ T / (math.pi * np.sin(phase))[None, :]
    return a * np.cos(phase) + b, f / a


def stats(P, a: float, b: float, K: int, kernel: str = "jackson", lam: float = 0.0):
    """Mean and standard error over the nvec independent vectors (rows of
    P[nvec, M]) of the moments and of the per-vector DOS:
    err = sqrt(sum_r (x_r - mean)^2 / ((nvec - 1) nvec)), 0 for one vector.
    Returns (mu_mean, mu_err, E, rho_mean, rho_err)."""
    P = np.atleast_2d(np.asarray(P, dtype=np.float64))
    nv = P.shape[0]
    E, rho = dos_many(P, a, b, K, kernel, lam)

    def mean_err(X):
        m = X.mean(axis=0)
        if nv < 2:
            return m, np.zeros_like(m)
        return m, np.sqrt(((X - m) ** 2).sum(axis=0) / ((nv - 1) * nv))

    mu_m, mu_e = mean_err(P)
    rho_m, rho_e = mean_err(rho)
    return mu_m, mu_e, E, rho_m, rho_e


def dos_error_integral(rho_err, a: float) -> float:
    """int |sigma_rho(E)| dE by the Gauss-Chebyshev rule on the K nodes:
    sum_k rho_err[k] a pi sqrt(1 - x_k^2) / K."""
    rho_err = np.asarray(rho_err, dtype=np.float64)
    K = rho_err.size
    return float(np.sum(rho_err * a * math.pi * np.sin(math.pi * (np.arange(K) + 0.5) / K)) / K)


def gershgorin(H: CSR):
    """Spectral enclosure [min_i(H_ii - sum_{j!=i}|H_ij|), max_i(H_ii + sum_{j!=i}|H_ij|)]
    (Gershgorin circle theorem; paper Sec. II-A-2 below Eq. (tilde))."""
    diag = np.zeros(H.n)
    rad = np.zeros(H.n)
    on = H._row == H.col
    np.add.at(diag, H._row[on], H.val[on].real)
    np.add.at(rad, H._row[~on], np.abs(H.val[~on]))
    return float(np.min(diag - rad)), float(np.max(diag + rad))


def lanczos_bounds(H: CSR, k: int, start: np.ndarray):
    """k-step Lanczos with full reorthogonalisation (two Gram-Schmidt passes).

    Returns (emin, emax, info) where emax = min(G_max, theta_max + beta_k |s_k|)
    and emin = max(G_min, theta_min - beta_k |s_1k|): the extreme Ritz values
    widened by their residual norms and clamped to the Gershgorin enclosure.
    The start vector is an input (the CUDA path draws it from stream 6).
    """
    gmin, gmax = gershgorin(H)
    if k <= 0:
        return gmin, gmax, dict(steps=0)
    q = np.asarray(start, dtype=np.complex128 if H.is_complex else np.float64).reshape(H.n)
    q = q / np.linalg.norm(q)
    Q = [q]
    alpha, beta = [], []
    for j in range(min(k, H.n)):
        w = H.matvec(Q[j][:, None])[:, 0]
        a_j = float(np.real(np.vdot(Q[j], w)))
        alpha.append(a_j)
        for _ in range(2):
            Qm = np.stack(Q, axis=1)
            w = w - Qm @ (Qm.conj().T @ w)
        b_j = float(np.linalg.norm(w))
        beta.append(b_j)
        if b_j <= 1e-12 * max(1.0, abs(a_j)) or j + 1 == H.n:
            break
        Q.append(w / b_j)
    m = len(alpha)
    T = np.diag(alpha) + np.diag(beta[: m - 1], 1) + np.diag(beta[: m - 1], -1)
    theta, S = np.linalg.eigh(T)
    bk = beta[m - 1]
    emax = theta[-1] + bk * abs(S[m - 1, -1])
    emin = theta[0] - bk * abs(S[m - 1, 0])
    return max(gmin, emin), min(gmax, emax), dict(steps=m, theta_min=theta[0], theta_max=theta[-1],
                                                    beta_k=bk)


def rescale(emin: float, emax: float, eps: float = 0.01):
    """Eq. (tilde): H~ = (H - b)/a with b = alpha_+ = (Emax+Emin)/2 and
    a = alpha_- = (Emax-Emin)/2, widened by the padding eps: a = (Emax-Emin)/(2-eps).
    eps = 0 is the paper's exact Gershgorin scaling."""
    return (emax - emin) / (2.0 - eps), 0.5 * (emax + emin)


def _rescaled_apply(H: CSR, a: float, b: float, X: np.ndarray) -> np.ndarray:
    """H~ X = (H X - b X) / a."""
    return (H.matvec(X) - b * X) / a


def _block(v0) -> np.ndarray:
    v0 = np.asarray(v0)
    return v0[:, None] if v0.ndim == 1 else v0


def moments_direct(H: CSR, a: float, b: float, v0, M: int):
    """Eqs. (rn) and (munr): r_0 = r, r_1 = H~ r_0, r_{n+2} = 2 H~ r_{n+1} - r_n,
    mu_n^r = Re <r_0|r_n> / N.  Returns (mu[M] averaged over the R vectors,
    mu_per_vec[R, M])."""
    V0 = _block(v0)
    N, R = V0.shape
    out = np.zeros((R, M))
    prev = V0.astype(np.result_type(V0, H.val, np.float64))
    out[:, 0] = np.real(np.sum(np.conj(V0) * prev, axis=0)) / N
    if M > 1:
        cur = _rescaled_apply(H, a, b, prev)
        out[:, 1] = np.real(np.sum(np.conj(V0) * cur, axis=0)) / N
        for n in range(2, M):
            nxt = 2.0 * _rescaled_apply(H, a, b, cur) - prev
            out[:, n] = np.real(np.sum(np.conj(V0) * nxt, axis=0)) / N
            prev, cur = cur, nxt
    return out.mean(axis=0), out


def moments_doubling(H: CSR, a: float, b: float, v0, M: int):
    """Stochastic moments with two moments per product (M even, M >= 2):

      v_0 = r, v_1 = H~ v_0, v_{n+1} = 2 H~ v_n - v_{n-1}   (Eq. (rn))
      mu_0^r = <v_0|v_0>/N, mu_1^r = Re<v_1|v_0>/N
      mu_2n^r = 2<v_n|v_n>/N - mu_0^r, mu_2n+1^r = 2 Re<v_n+1|v_n>/N - mu_1^r
      for n = 1 .. M/2 - 1 (uses v_0 .. v_{M/2}).
    Returns (mu[M], mu_per_vec[R, M])."""
    if M < 2 or M % 2:
        raise ValueError("M must be even and >= 2")
    V0 = _block(v0)
    N, R = V0.shape
    out = np.zeros((R, M))
    prev = V0.astype(np.result_type(V0, H.val, np.float64))
    cur = _rescaled_apply(H, a, b, prev)
    mu0 = np.real(np.sum(np.conj(prev) * prev, axis=0)) / N
    mu1 = np.real(np.sum(np.conj(cur) * prev, axis=0)) / N
    out[:, 0], out[:, 1] = mu0, mu1
    for n in range(1, M // 2):
        nxt = 2.0 * _rescaled_apply(H, a, b, cur) - prev
        out[:, 2 * n] = 2.0 * np.real(np.sum(np.conj(cur) * cur, axis=0)) / N - mu0
        out[:, 2 * n + 1] = 2.0 * np.real(np.sum(np.conj(nxt) * cur, axis=0)) / N - mu1
        prev, cur = cur, nxt
    return out.mean(axis=0), out


def exact_moments(H: CSR, a: float, b: float, M: int) -> np.ndarray:
    """Eq. (DoStr): mu_n = (1/N) sum_k T_n(E~_k), T_n(x) = cos(n arccos x), from a
    dense eigendecomposition (small N only).  E~ is clipped to [-1, 1]."""
    lam = np.linalg.eigvalsh(dense(H))
    x = np.clip((lam - b) / a, -1.0, 1.0)
    n = np.arange(M)[:, None]
    return np.cos(n * np.arccos(x)[None, :]).mean(axis=1)


def ldos_exact(H: CSR, a: float, b: float, sites, M: int) -> np.ndarray:
    """Local moments mu_n(i) = <i|T_n(H~)|i> = sum_k |U_ik|^2 cos(n arccos E~_k) for
    each site i in `sites`, from a dense eigendecomposition (small N only).
    Returns [len(sites), M]."""
    lam, U = np.linalg.eigh(dense(H))
    x = np.clip((lam - b) / a, -1.0, 1.0)
    T = np.cos(np.arange(M)[:, None] * np.arccos(x)[None, :])  # [M, N]
    W = np.abs(U[np.asarray(sites, dtype=np.int64), :]) ** 2      # [sites, N]
    return W @ T.T


def plane_waves(L, k) -> np.ndarray:
    """Columns e^{i k_j . x} (not normalised: |column|^2 = N) for the wave vectors
    k[j] (radians per lattice spacing, one component per lattice dimension), x the
    integer coordinates of site i = x0 + L0 (x1 + L1 x2).  Returns [N, nk] complex."""
    L = tuple(int(v) for v in L)
    k = np.atleast_2d(np.asarray(k, dtype=np.float64))[:, :len(L)]
    N = int(np.prod(L))
    i = np.arange(N)
    coords = []
    for Ld in L:                      # x_d = (i // (L0 ... L_{d-1})) mod L_d
        coords.append(i % Ld)
        i = i // Ld
    X = np.stack(coords, axis=1).astype(np.float64)  # [N, dims]
    return np.exp(1j * (X @ k.T))


def spectral_exact(H: CSR, a: float, b: float, L, k, M: int) -> np.ndarray:
    """Momentum-resolved moments <k|T_n(H~)|k> = sum_m |<k|u_m>|^2 cos(n arccos E~_m)
    for the normalised plane waves |k> = N^{-1/2} sum_x e^{i k.x}|x>, from a dense
    eigendecomposition (small N only).  Returns [nk, M]."""
    lam, U = np.linalg.eigh(dense(H))
    x = np.clip((lam - b) / a, -1.0, 1.0)
    T = np.cos(np.arange(M)[:, None] * np.arccos(x)[None, :])  # [M, N]
    P = plane_waves(L, k) / math.sqrt(H.n)                        # [N, nk]
    W = np.abs(U.conj().T @ P) ** 2                                # [N eigen, nk]
    return W.T @ T.T


def jackson_kernel(M: int) -> np.ndarray:
    """Jackson damping factors (review Eq. 71), n = 0 .. M-1:
    g_n = [(M-n+1) cos(pi n/(M+1)) + sin(pi n/(M+1)) cot(pi/(M+1))] / (M+1)."""
    n = np.arange(M, dtype=np.float64)
    q = math.pi / (M + 1)
    return ((M - n + 1) * np.cos(q * n) + np.sin(q * n) / math.tan(q)) / (M + 1)


def lorentz_kernel(M: int, lam: float) -> np.ndarray:
    """Lorentz damping factors (review Eq. 74), n = 0 .. M-1:
    g_n = sinh(lam (1 - n/M)) / sinh(lam), lam > 0."""
    n = np.arange(M, dtype=np.float64)
    return np.sinh(lam * (1.0 - n / M)) / math.sinh(lam)


def damping(M: int, kernel: str = "jackson", lam: float = 0.0) -> np.ndarray:
    if kernel == "jackson":
        return jackson_kernel(M)
    if kernel == "lorentz":
        return lorentz_kernel(M, lam)
    return np.ones(M)


def dos(mu, a: float, b: float, K: int, kernel: str = "jackson", lam: float = 0.0):
    """Eq. (fKPM) evaluated on the K Chebyshev nodes x_k = cos(pi (k + 1/2) / K):

      f(x_k) = [g_0 mu_0 + 2 sum_{n=1}^{M-1} g_n mu_n T_n(x_k)] / (pi sqrt(1 - x_k^2)),
      T_n(x_k) = cos(n pi (k + 1/2) / K)

    by a direct double sum; E_k = a x_k + b, rho(E_k) = f(x_k) / a (so that
    the integral of rho over E is the integral of f over x).  kernel is
    "jackson", "lorentz" (with lam) or "none" (g_n = 1).  Returns (E[K], rho[K]),
    k = 0 .. K-1."""
    mu = np.asarray(mu, dtype=np.float64)
    M = mu.size
    g = damping(M, kernel, lam)
    phase = math.pi * (np.arange(K) + 0.5) / K
    x = np.cos(phase)
    f = np.empty(K)
    for k in range(K):
        s = g[0] * mu[0]
        for n in range(1, M):
            s += 2.0 * g[n] * mu[n] * math.cos(n * phase[k])
        f[k] = s / (math.pi * math.sqrt(1.0 - x[k] * x[k]))
    return a * x + b, f / a
