"""Thin ctypes binding of libkpm.so (include/kpm.h); argument marshalling only.

Every function keeps the C name and returns what the C call writes.  Host
inputs are numpy arrays; outputs are numpy arrays unless the caller passes
preallocated torch CUDA tensors (``out=``), in which case the library writes
device memory directly and the call is asynchronous on ``stream``.  There is
no fallback: if the library is missing or a call fails, an exception is
raised.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libkpm.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "kpm.h")

KPM_OK, KPM_EINVAL, KPM_ENOMEM, KPM_ECUDA, KPM_ETIMEOUT, KPM_EDIVERGE, KPM_EBUSY, KPM_ENOTREADY = range(8)
KPM_REAL, KPM_COMPLEX = 0, 1
KPM_FP64, KPM_FP32_VEC_FP64_MOM = 0, 1
KPM_KERNEL_JACKSON, KPM_KERNEL_NONE, KPM_KERNEL_LORENTZ = 0, 1, 2
KERNELS = {"jackson": KPM_KERNEL_JACKSON, "none": KPM_KERNEL_NONE, "lorentz": KPM_KERNEL_LORENTZ}
PRECISIONS = {"fp64": KPM_FP64, "fp32": KPM_FP32_VEC_FP64_MOM, KPM_FP64: KPM_FP64,
              KPM_FP32_VEC_FP64_MOM: KPM_FP32_VEC_FP64_MOM}
STATUS_NAMES = {0: "KPM_OK", 1: "KPM_EINVAL", 2: "KPM_ENOMEM", 3: "KPM_ECUDA", 4: "KPM_ETIMEOUT",
                5: "KPM_EDIVERGE", 6: "KPM_EBUSY", 7: "KPM_ENOTREADY"}


class KPMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class kpm_stencil_desc(C.Structure):
    _fields_ = [("dims", C.c_int), ("L", C.c_int64 * 3), ("periodic", C.c_int * 3),
                ("onsite", C.c_void_p), ("hop", C.c_void_p), ("t_re", C.c_double),
                ("t_im", C.c_double), ("bond_mask", C.c_void_p)]


class kpm_params(C.Structure):
    _fields_ = [("M", C.c_int), ("R", C.c_int), ("S", C.c_int), ("seed", C.c_uint64),
                ("precision", C.c_int), ("a", C.c_double), ("b", C.c_double),
                ("user_v0", C.c_void_p), ("s0", C.c_int)]


class kpm_server_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("cancelled", C.c_uint64), ("ticks", C.c_uint64), ("p50_s", C.c_double),
                ("p99_s", C.c_double), ("mean_s", C.c_double), ("max_s", C.c_double),
                ("solves_per_s", C.c_double), ("peak_resident", C.c_int),
                ("peak_bytes", C.c_size_t), ("budget_bytes", C.c_size_t)]


_lib = None


def lib() -> C.CDLL:
    """Loads libkpm.so (built in-tree by paper_1105_5481_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1105_5481_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        h = C.c_void_p
        L.kpm_create_stencil.argtypes = [C.POINTER(kpm_stencil_desc), C.c_int, C.POINTER(h)]
        L.kpm_create_csr.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(h)]
        L.kpm_create_dense.argtypes = [C.c_int64, C.c_void_p, C.c_int, C.POINTER(h)]
        L.kpm_stencil_to_csr.argtypes = [C.POINTER(kpm_stencil_desc), C.c_int, C.POINTER(C.c_int64),
                                         C.c_void_p, C.c_void_p, C.c_void_p]
        L.kpm_bounds.argtypes = [h, C.c_int, C.c_double, C.c_uint64] + [C.POINTER(C.c_double)] * 4 + [C.c_void_p]
        L.kpm_moments.argtypes = [h, C.POINTER(kpm_params), C.c_void_p, C.c_void_p, C.c_void_p]
        L.kpm_moments_extend.argtypes = [h, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.kpm_ldos_moments.argtypes = [h, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double,
                                       C.c_int, C.c_void_p, C.c_void_p]
        L.kpm_spectral_moments.argtypes = [h, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double,
                                           C.c_int, C.c_void_p, C.c_void_p]
        L.kpm_dos.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                              C.c_void_p, C.c_void_p, C.c_void_p]
        L.kpm_dos_kernel.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                     C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]
        L.kpm_green.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                C.c_double] + [C.c_void_p] * 4
        L.kpm_thermo.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                 C.c_double, C.c_void_p, C.c_int, C.c_double, C.c_void_p,
                                 C.c_void_p]
        L.kpm_stats.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                C.c_int, C.c_double] + [C.c_void_p] * 6
        L.kpm_moments_adaptive.argtypes = [h, C.POINTER(kpm_params), C.c_int, C.c_int, C.c_double,
                                           C.c_double, C.c_int] + [C.c_void_p] * 5 + [
                                           C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_void_p]
        L.kpm_info.argtypes = [h, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int),
                               C.POINTER(C.c_int)]
        L.kpm_step_timing.argtypes = [h, C.POINTER(C.c_double), C.POINTER(C.c_int)]
        L.kpm_moments_csr_noalloc.argtypes = [C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_double,
                                              C.c_double, C.c_void_p, C.c_void_p]
        L.kpm_batch_create.argtypes = [C.c_int, C.POINTER(C.c_void_p), C.POINTER(kpm_params), C.POINTER(h)]
        L.kpm_batch_run.argtypes = [h, C.c_void_p, C.c_void_p]
        L.kpm_batch_tune.argtypes = [h, C.c_int, C.c_void_p]
        L.kpm_batch_set_config.argtypes = [h, C.c_int, C.c_int, C.c_int]
        L.kpm_batch_info.argtypes = [h, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_double)]
        L.kpm_batch_set_chunk_bytes.argtypes = [h, C.c_int]
        L.kpm_batch_get_chunk_bytes.argtypes = [h, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.kpm_batch_set_resident.argtypes = [h, C.c_int]
        L.kpm_batch_get_resident.argtypes = [h, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.kpm_batch_set_staged.argtypes = [h, C.c_int]
        L.kpm_batch_get_staged.argtypes = [h, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                           C.POINTER(C.c_int)]
        L.kpm_batch_destroy.argtypes = [h]
        L.kpm_batch_destroy.restype = None
        L.kpm_server_create.argtypes = [C.c_size_t, C.c_int, C.c_int, C.POINTER(h)]
        L.kpm_server_submit.argtypes = [h, h, C.POINTER(kpm_params), C.c_int, C.POINTER(C.c_uint64)]
        L.kpm_server_wait.argtypes = [h, C.c_uint64, C.c_double]
        L.kpm_server_poll.argtypes = [h, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.POINTER(C.c_double)]
        L.kpm_server_cancel.argtypes = [h, C.c_uint64]
        L.kpm_server_stats.argtypes = [h, C.POINTER(kpm_server_stats_t)]
        L.kpm_server_destroy.argtypes = [h]
        L.kpm_server_destroy.restype = None
        L.kpm_destroy.argtypes = [h]
        L.kpm_destroy.restype = None
        L.kpm_last_error.restype = C.c_char_p
        L.kpm_kernel_launches.restype = C.c_uint64
        L.kpm_testing_fail_allocations.argtypes = [C.c_int64]
        L.kpm_testing_stall_step_pipeline.argtypes = [C.c_int]
        L.kpm_testing_last_step_form.argtypes = [h, C.POINTER(C.c_int)]
        for name in ("kpm_create_stencil", "kpm_create_csr", "kpm_create_dense", "kpm_stencil_to_csr",
                     "kpm_bounds",
                     "kpm_moments", "kpm_moments_extend", "kpm_ldos_moments", "kpm_spectral_moments",
                     "kpm_dos", "kpm_info", "kpm_step_timing",
                     "kpm_moments_csr_noalloc", "kpm_batch_create", "kpm_batch_run", "kpm_batch_tune",
                     "kpm_batch_set_config", "kpm_batch_info", "kpm_batch_set_rtiles",
                     "kpm_batch_get_rtiles", "kpm_batch_set_resident", "kpm_batch_get_resident",
                     "kpm_batch_set_chunk_bytes", "kpm_batch_get_chunk_bytes",
                     "kpm_server_create",
                     "kpm_server_submit", "kpm_server_wait", "kpm_server_poll", "kpm_server_cancel",
                     "kpm_server_stats", "kpm_testing_fail_allocations",
                     "kpm_testing_stall_step_pipeline", "kpm_testing_last_step_form"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def declared_functions() -> list[str]:
    """Entry points declared in include/kpm.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(kpm_\w+)\s*\(", text, re.M)))


def _check(status: int):
    if status != KPM_OK:
        raise KPMError(status, lib().kpm_last_error().decode())


def _ptr(a):
    """Pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensor must be contiguous"
        return a.data_ptr()
    raise TypeError(type(a))


def _stream(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


def _f64(a, complex_=False):
    if a is None:
        return None
    a = np.asarray(a)
    if complex_:
        a = np.ascontiguousarray(a, dtype=np.complex128)
        return a.view(np.float64)
    return np.ascontiguousarray(a, dtype=np.float64)


class Handle:
    """Owning wrapper of a kpm_handle."""

    def __init__(self, raw: C.c_void_p, complex_: bool, keep=()):
        self.raw = raw
        self.complex = complex_
        self._keep = keep

    def close(self):
        if self.raw:
            lib().kpm_destroy(self.raw)
            self.raw = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _desc(dims, L, periodic, onsite, hop, t, bond_mask, complex_):
    d = kpm_stencil_desc()
    d.dims = int(dims)
    L = list(L) + [1] * (3 - len(L))
    periodic = [True] * dims if periodic is None else list(periodic)
    periodic = list(periodic) + [True] * (3 - len(periodic))
    for k in range(3):
        d.L[k] = int(L[k])
        d.periodic[k] = 1 if periodic[k] else 0
    on = _f64(onsite)
    hp = _f64(hop, complex_)
    mk = None if bond_mask is None else np.ascontiguousarray(np.asarray(bond_mask, dtype=np.uint8))
    d.onsite = _ptr(on)
    d.hop = _ptr(hp)
    t = complex(t)
    d.t_re, d.t_im = t.real, t.imag
    d.bond_mask = _ptr(mk)
    return d, (on, hp, mk)


def kpm_create_stencil(dims, L, periodic=None, onsite=None, hop=None, t=1.0, bond_mask=None,
                       complex_=False) -> Handle:
    d, keep = _desc(dims, L, periodic, onsite, hop, t, bond_mask, complex_)
    raw = C.c_void_p()
    _check(lib().kpm_create_stencil(C.byref(d), KPM_COMPLEX if complex_ else KPM_REAL, C.byref(raw)))
    return Handle(raw, complex_)


def kpm_create_csr(n, rowptr, col, val, complex_=False) -> Handle:
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    vl = _f64(val, complex_)
    raw = C.c_void_p()
    _check(lib().kpm_create_csr(int(n), _ptr(rp), _ptr(cl), _ptr(vl),
                                KPM_COMPLEX if complex_ else KPM_REAL, C.byref(raw)))
    return Handle(raw, complex_)


def kpm_create_dense(H) -> Handle:
    """Dense Hermitian n x n matrix (float64 or complex128 array): the paper's
    dense formulation, FP64 moments only."""
    H = np.asarray(H)
    if H.ndim != 2 or H.shape[0] != H.shape[1]:
        raise ValueError("H must be a square matrix")
    complex_ = bool(np.iscomplexobj(H))
    v = _f64(H, complex_)
    raw = C.c_void_p()
    _check(lib().kpm_create_dense(int(H.shape[0]), _ptr(v), KPM_COMPLEX if complex_ else KPM_REAL,
                                  C.byref(raw)))
    return Handle(raw, complex_)


def kpm_stencil_to_csr(dims, L, periodic=None, onsite=None, hop=None, t=1.0, bond_mask=None,
                       complex_=False):
    d, keep = _desc(dims, L, periodic, onsite, hop, t, bond_mask, complex_)
    f = KPM_COMPLEX if complex_ else KPM_REAL
    nnz = C.c_int64()
    _check(lib().kpm_stencil_to_csr(C.byref(d), f, C.byref(nnz), None, None, None))
    n = int(np.prod([d.L[k] for k in range(dims)]))
    rowptr = np.zeros(n + 1, np.int64)
    col = np.zeros(nnz.value, np.int32)
    val = np.zeros(nnz.value, np.complex128 if complex_ else np.float64)
    _check(lib().kpm_stencil_to_csr(C.byref(d), f, C.byref(nnz), _ptr(rowptr), _ptr(col),
                                    _ptr(val.view(np.float64) if complex_ else val)))
    return rowptr, col, val


def kpm_bounds(h: Handle, lanczos_steps=30, pad_eps=0.01, seed=0, stream=None):
    """Returns (emin, emax, a, b)."""
    out = [C.c_double() for _ in range(4)]
    _check(lib().kpm_bounds(h.raw, int(lanczos_steps), float(pad_eps), int(seed),
                            *[C.byref(o) for o in out], _stream(stream)))
    return tuple(o.value for o in out)


def kpm_moments(h: Handle, M, R, a, b, seed=0, S=1, precision="fp64", user_v0=None, per_vec=False,
                out=None, out_per_vec=None, stream=None, check=True, s0=0):
    """Chebyshev moments.  Returns mu (and mu_per_vec[S*R, M] if per_vec).
    s0: realisation index of this call's first realisation in the seed's sequence.

    ``out``/``out_per_vec`` may be preallocated float64 arrays or CUDA tensors
    (then the call does not synchronise).  With check=False a KPM_EDIVERGE
    status is returned in place of an exception as the last element."""
    p = kpm_params()
    p.M, p.R, p.S, p.seed = int(M), int(R), int(S), int(seed) & 0xFFFFFFFFFFFFFFFF
    p.precision = PRECISIONS[precision]
    p.a, p.b = float(a), float(b)
    p.s0 = int(s0)
    v0 = None
    if user_v0 is not None:
        if hasattr(user_v0, "data_ptr"):
            v0 = user_v0
        else:
            v0 = _f64(user_v0, h.complex)
        p.user_v0 = _ptr(v0)
    mu = out if out is not None else np.zeros(int(M))
    pv = out_per_vec
    if pv is None and per_vec:
        pv = np.zeros((max(int(S), 1) * int(R), int(M)))
    st = lib().kpm_moments(h.raw, C.byref(p), _ptr(mu), _ptr(pv), _stream(stream))
    if st == KPM_EDIVERGE and not check:
        return (mu, pv, st) if per_vec or out_per_vec is not None else (mu, st)
    _check(st)
    return (mu, pv) if per_vec or out_per_vec is not None else mu


def kpm_moments_extend(h: Handle, M, R=None, per_vec=False, out=None, out_per_vec=None, stream=None):
    """Continue the last single-realisation kpm_moments call on ``h`` to M moments.
    Returns mu (and mu_per_vec[R, M] if per_vec; R is that call's R)."""
    mu = out if out is not None else np.zeros(int(M))
    pv = out_per_vec
    if pv is None and per_vec:
        pv = np.zeros((int(R), int(M)))
    _check(lib().kpm_moments_extend(h.raw, int(M), _ptr(mu), _ptr(pv), _stream(stream)))
    return (mu, pv) if per_vec or out_per_vec is not None else mu


def kpm_ldos_moments(h: Handle, sites, M, a, b, precision="fp64", out=None, stream=None):
    """Local Chebyshev moments <i|T_n(H~)|i> of the given sites (start vectors
    built on the device).  Returns [len(sites), M] (numpy unless ``out``, a CUDA
    tensor of len(sites)*M doubles, is given)."""
    sites = np.ascontiguousarray(np.atleast_1d(sites), dtype=np.int64)
    mu = np.zeros((sites.size, int(M))) if out is None else out
    _check(lib().kpm_ldos_moments(h.raw, _ptr(sites), sites.size, int(M), float(a), float(b),
                                  PRECISIONS[precision], _ptr(mu), _stream(stream)))
    return mu


def kpm_spectral_moments(h: Handle, k, M, a, b, precision="fp64", out=None, stream=None):
    """Momentum-resolved moments <k|T_n(H~)|k> of normalised plane waves for the
    wave vectors k ([nk, 3] or [3], radians per lattice spacing).  Returns
    [nk, M] (numpy unless ``out``, a CUDA tensor of nk*M doubles, is given)."""
    k = np.asarray(k, dtype=np.float64)
    k = np.ascontiguousarray(np.pad(k.reshape(-1, k.shape[-1]), ((0, 0), (0, 3 - k.shape[-1]))))
    mu = np.zeros((k.shape[0], int(M))) if out is None else out
    _check(lib().kpm_spectral_moments(h.raw, _ptr(k), k.shape[0], int(M), float(a), float(b),
                                      PRECISIONS[precision], _ptr(mu), _stream(stream)))
    return mu


def kpm_dos(mu, a, b, K, kernel="jackson", E=None, rho=None, stream=None, lam=None):
    """Returns (E[K], rho[K]); host arrays unless device tensors are passed.
    kernel: "jackson", "none" or "lorentz" (with lam > 0)."""
    if not hasattr(mu, "data_ptr"):
        mu = np.ascontiguousarray(mu, dtype=np.float64)
    M = int(mu.shape[0])
    E = np.zeros(int(K)) if E is None else E
    rho = np.zeros(int(K)) if rho is None else rho
    if kernel == "lorentz" or lam is not None:
        _check(lib().kpm_dos_kernel(_ptr(mu), M, float(a), float(b), int(K), KERNELS[kernel],
                                    float(lam or 0.0), _ptr(E), _ptr(rho), _stream(stream)))
    else:
        _check(lib().kpm_dos(_ptr(mu), M, float(a), float(b), int(K), KERNELS[kernel], _ptr(E),
                             _ptr(rho), _stream(stream)))
    return E, rho


def kpm_green(mu, a, b, K, kernel="lorentz", lam=4.0, stream=None):
    """Local Green's function G(E + i0) on the K Chebyshev nodes: returns
    (E[K], G[K] complex) as host arrays (Im G = -pi rho)."""
    if not hasattr(mu, "data_ptr"):
        mu = np.ascontiguousarray(mu, dtype=np.float64)
    M = int(mu.shape[0])
    E, gr, gi = np.zeros(int(K)), np.zeros(int(K)), np.zeros(int(K))
    _check(lib().kpm_green(_ptr(mu), M, float(a), float(b), int(K), KERNELS[kernel],
                           float(lam or 0.0), _ptr(E), _ptr(gr), _ptr(gi), _stream(stream)))
    return E, gr + 1j * gi


def kpm_thermo(mu, a, b, K, betas, mu_c=0.0, kernel="jackson", lam=None, stream=None):
    """Fermi-occupation integrals of the DOS per inverse temperature: returns an
    [nT, 4] array of (n, u, s, c) per site (beta = inf: the ground state)."""
    if not hasattr(mu, "data_ptr"):
        mu = np.ascontiguousarray(mu, dtype=np.float64)
    betas = np.ascontiguousarray(np.atleast_1d(betas), dtype=np.float64)
    out = np.zeros((betas.size, 4))
    _check(lib().kpm_thermo(_ptr(mu), int(mu.shape[0]), float(a), float(b), int(K),
                            KERNELS[kernel], float(lam or 0.0), _ptr(betas), betas.size,
                            float(mu_c), _ptr(out), _stream(stream)))
    return out


def kpm_stats(pv, a, b, K, kernel="jackson", lam=None, stream=None):
    """Mean and standard error over the vectors (rows of pv[nvec, M]) of the
    moments and of the per-vector DOS: returns (mu_mean, mu_err, E, rho_mean,
    rho_err) as host arrays."""
    if not hasattr(pv, "data_ptr"):
        pv = np.ascontiguousarray(pv, dtype=np.float64)
    pv2 = pv if len(pv.shape) == 2 else pv.reshape(1, -1)
    nvec, M = int(pv2.shape[0]), int(pv2.shape[1])
    out = [np.zeros(M), np.zeros(M), np.zeros(int(K)), np.zeros(int(K)), np.zeros(int(K))]
    _check(lib().kpm_stats(_ptr(pv2), nvec, M, float(a), float(b), int(K), KERNELS[kernel],
                           float(lam or 0.0), *[_ptr(o) for o in out], _stream(stream)))
    return tuple(out)


def kpm_moments_adaptive(h: Handle, M, R, a, b, K, target, max_rounds, seed=0, S=1,
                         precision="fp32", kernel="jackson", lam=None, stream=None):
    """Rounds of R (x S) new random vectors (seed + round) until the integrated
    DOS standard error is <= target: returns dict(mu, mu_err, E, rho, rho_err,
    rounds, error)."""
    p = kpm_params()
    p.M, p.R, p.S, p.seed = int(M), int(R), int(S), int(seed) & 0xFFFFFFFFFFFFFFFF
    p.precision = PRECISIONS[precision]
    p.a, p.b = float(a), float(b)
    out = [np.zeros(int(M)), np.zeros(int(M)), np.zeros(int(K)), np.zeros(int(K)), np.zeros(int(K))]
    rounds, err = C.c_int(), C.c_double()
    _check(lib().kpm_moments_adaptive(h.raw, C.byref(p), int(K), KERNELS[kernel], float(lam or 0.0),
                                      float(target), int(max_rounds), *[_ptr(o) for o in out],
                                      C.byref(rounds), C.byref(err), _stream(stream)))
    return dict(mu=out[0], mu_err=out[1], E=out[2], rho=out[3], rho_err=out[4],
                rounds=rounds.value, error=err.value)


def kpm_info(h: Handle):
    n, nnz = C.c_int64(), C.c_int64()
    field, st = C.c_int(), C.c_int()
    _check(lib().kpm_info(h.raw, C.byref(n), C.byref(nnz), C.byref(field), C.byref(st)))
    return dict(n=n.value, nnz=nnz.value, complex=field.value == KPM_COMPLEX, stencil=bool(st.value))


def kpm_step_timing(h: Handle):
    """(ms of the fused-step chain of the last kpm_moments call, fused-step launches)."""
    ms, n = C.c_double(), C.c_int()
    _check(lib().kpm_step_timing(h.raw, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def kpm_moments_csr_noalloc(n, nnz, d_rowptr, d_col, d_val, M, R, a, b, seed=0, complex_=False,
                            out=None, stream=None):
    """FP64 moments of a device-resident CSR matrix using only the library's
    fixed scratch array (no device allocation inside the call).  d_* are
    contiguous CUDA tensors (int64, int32, float64 [or float64 pairs]); ``out``
    a float64 CUDA tensor of M entries (asynchronous) or None (host result)."""
    mu = np.zeros(int(M)) if out is None else out
    _check(lib().kpm_moments_csr_noalloc(int(n), int(nnz), _ptr(d_rowptr), _ptr(d_col), _ptr(d_val),
                                         KPM_COMPLEX if complex_ else KPM_REAL, int(M), int(R),
                                         int(seed) & 0xFFFFFFFFFFFFFFFF, float(a), float(b), _ptr(mu),
                                         _stream(stream)))
    return mu


class Batch:
    """Owning wrapper of a kpm_batch (keeps its handles alive)."""

    def __init__(self, raw, handles, Ms):
        self.raw = raw
        self.handles = list(handles)
        self.Ms = list(Ms)
        self.offsets = np.concatenate([[0], np.cumsum(self.Ms)]).astype(np.int64)

    def close(self):
        if self.raw:
            lib().kpm_batch_destroy(self.raw)
            self.raw = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def split(self, mu):
        return [mu[self.offsets[i]:self.offsets[i + 1]] for i in range(len(self.Ms))]


def kpm_batch_create(handles, Ms, R, a, b, seeds, precision="fp32") -> Batch:
    """Batch of len(handles) instances; Ms, a, b, seeds are per-instance sequences."""
    n = len(handles)
    ps = (kpm_params * n)()
    for i in range(n):
        ps[i].M, ps[i].R, ps[i].S = int(Ms[i]), int(R), 1
        ps[i].seed = int(seeds[i]) & 0xFFFFFFFFFFFFFFFF
        ps[i].precision = PRECISIONS[precision]
        ps[i].a, ps[i].b = float(a[i]), float(b[i])
        ps[i].user_v0 = None
    hs = (C.c_void_p * n)(*[h.raw for h in handles])
    raw = C.c_void_p()
    _check(lib().kpm_batch_create(n, hs, ps, C.byref(raw)))
    return Batch(raw, handles, Ms)


def kpm_batch_run(bt: Batch, out=None, stream=None):
    """Runs the batch; returns the concatenated moments (numpy) unless ``out``
    (a CUDA tensor of sum(M) doubles) is given."""
    mu = np.zeros(int(bt.offsets[-1])) if out is None else out
    _check(lib().kpm_batch_run(bt.raw, _ptr(mu), _stream(stream)))
    return mu


def kpm_batch_tune(bt: Batch, reps=1, stream=None):
    _check(lib().kpm_batch_tune(bt.raw, int(reps), _stream(stream)))
    return kpm_batch_info(bt)


def kpm_batch_set_config(bt: Batch, cluster, chunk=4, percent=100):
    _check(lib().kpm_batch_set_config(bt.raw, int(cluster), int(chunk), int(percent)))


def kpm_batch_set_rtiles(bt: Batch, rtiles, top=0):
    """Split the `top` largest instances (0: all) into `rtiles` column tiles."""
    _check(lib().kpm_batch_set_rtiles(bt.raw, int(rtiles), int(top)))


def kpm_batch_get_rtiles(bt: Batch):
    """(current R-tiles, instances tiled, largest admissible R-tiles)."""
    rt, tp, mx = C.c_int(), C.c_int(), C.c_int()
    _check(lib().kpm_batch_get_rtiles(bt.raw, C.byref(rt), C.byref(tp), C.byref(mx)))
    return rt.value, tp.value, mx.value


def kpm_batch_set_chunk_bytes(bt: Batch, nbytes):
    """Bytes of a row each thread moves per product (32 or 16: twice the threads per row)."""
    _check(lib().kpm_batch_set_chunk_bytes(bt.raw, int(nbytes)))


def kpm_batch_get_chunk_bytes(bt: Batch):
    """(chunk bytes, threads per row)."""
    nb, tpr = C.c_int(), C.c_int()
    _check(lib().kpm_batch_get_chunk_bytes(bt.raw, C.byref(nb), C.byref(tpr)))
    return nb.value, tpr.value


def kpm_batch_set_resident(bt: Batch, resident=True):
    """Keep every instance's vector blocks in its cluster's shared memory."""
    _check(lib().kpm_batch_set_resident(bt.raw, int(bool(resident))))


def kpm_batch_get_resident(bt: Batch):
    """(resident form set, smallest cluster size at which the batch fits; 0: none)."""
    on, cmin = C.c_int(), C.c_int()
    _check(lib().kpm_batch_get_resident(bt.raw, C.byref(on), C.byref(cmin)))
    return bool(on.value), cmin.value


def kpm_batch_set_staged(bt: Batch, staged=True):
    """Bring the vector tiles into shared memory by bulk asynchronous copies."""
    _check(lib().kpm_batch_set_staged(bt.raw, int(bool(staged))))


def kpm_batch_get_staged(bt: Batch):
    """(staged form set, tile rows, v_n ring stages)."""
    on, tr, st = C.c_int(), C.c_int(), C.c_int()
    _check(lib().kpm_batch_get_staged(bt.raw, C.byref(on), C.byref(tr), C.byref(st)))
    return bool(on.value), tr.value, st.value


def kpm_batch_info(bt: Batch):
    cl, ch, nc = C.c_int(), C.c_int(), C.c_int()
    ms = C.c_double()
    _check(lib().kpm_batch_info(bt.raw, C.byref(cl), C.byref(ch), C.byref(nc), C.byref(ms)))
    return dict(cluster=cl.value, chunk=ch.value, clusters=nc.value, last_ms=ms.value)


def kpm_batch_destroy(bt: Batch):
    bt.close()


class Server:
    """Owning wrapper of a kpm_server; remembers (M, K) of each request."""

    def __init__(self, raw):
        self.raw = raw
        self.shapes = {}
        self.handles = {}

    def close(self):
        if self.raw:
            lib().kpm_server_destroy(self.raw)
            self.raw = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def kpm_server_create(hbm_budget_bytes, steps_per_tick=32, cluster=4) -> Server:
    raw = C.c_void_p()
    _check(lib().kpm_server_create(int(hbm_budget_bytes), int(steps_per_tick), int(cluster), C.byref(raw)))
    return Server(raw)


def kpm_server_submit(srv: Server, h: Handle, M, R, a, b, seed=0, precision="fp32", K=0) -> int:
    p = kpm_params()
    p.M, p.R, p.S = int(M), int(R), 1
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.precision = PRECISIONS[precision]
    p.a, p.b = float(a), float(b)
    p.user_v0 = None
    rid = C.c_uint64()
    _check(lib().kpm_server_submit(srv.raw, h.raw, C.byref(p), int(K), C.byref(rid)))
    srv.shapes[rid.value] = (int(M), int(K))
    srv.handles[rid.value] = h
    return rid.value


def kpm_server_wait(srv: Server, rid: int, timeout_s=-1.0):
    _check(lib().kpm_server_wait(srv.raw, int(rid), float(timeout_s)))


def kpm_server_poll(srv: Server, rid: int, check=True):
    """(mu, E, rho, latency_s) of a finished request, or None while it runs."""
    M, K = srv.shapes[rid]
    mu, E, rho = np.zeros(M), np.zeros(max(K, 1)), np.zeros(max(K, 1))
    lat = C.c_double()
    st = lib().kpm_server_poll(srv.raw, int(rid), _ptr(mu), _ptr(E), _ptr(rho), C.byref(lat))
    if st == KPM_ENOTREADY:
        return None
    srv.shapes.pop(rid, None)
    srv.handles.pop(rid, None)
    if check:
        _check(st)
    return mu, E[:K], rho[:K], lat.value


def kpm_server_cancel(srv: Server, rid: int):
    _check(lib().kpm_server_cancel(srv.raw, int(rid)))


def kpm_server_stats(srv: Server) -> dict:
    st = kpm_server_stats_t()
    _check(lib().kpm_server_stats(srv.raw, C.byref(st)))
    return {f: getattr(st, f) for f, _ in st._fields_}


def kpm_server_destroy(srv: Server):
    srv.close()


def kpm_destroy(h: Handle):
    h.close()


def kpm_last_error() -> str:
    return lib().kpm_last_error().decode()


def kpm_kernel_launches() -> int:
    return int(lib().kpm_kernel_launches())


def kpm_testing_fail_allocations(after: int):
    """Testing aid: the next `after` device allocations of the library succeed and
    the one after fails with KPM_ENOMEM (-1 disarms)."""
    _check(lib().kpm_testing_fail_allocations(int(after)))


def kpm_testing_stall_step_pipeline(on: bool):
    """Testing aid: plans made while set give the TMA-fed ELL and stencil steps a
    producer that issues nothing, so their bounded waits run out (KPM_ETIMEOUT)."""
    _check(lib().kpm_testing_stall_step_pipeline(int(bool(on))))


STEP_FORMS = {0: "fused step", 1: "TMA-fed ELL step", 2: "dense FP64 pipe", 3: "dense tensor cores",
              4: "TMA-fed stencil step", 5: "column-resident solve"}


def kpm_testing_last_step_form(h: Handle) -> str:
    """Testing aid: the product form the last plan of kpm_moments on h chose."""
    f = C.c_int()
    _check(lib().kpm_testing_last_step_form(h.raw, C.byref(f)))
    return STEP_FORMS[f.value]
