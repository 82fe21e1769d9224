"""TEST INFRASTRUCTURE ONLY: ctypes wrapper of oracle/kpm_cpu.c, the oracle's
doubling-form moments restated in plain C with OpenMP (a multi-core CPU
baseline).  Only the tests and the benchmark's CPU-baseline leg use it; it
shares no code with the CUDA library.  build() compiles it with gcc."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kpm_cpu.c")
LIB = os.path.join(HERE, "libkpm_cpu.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles libkpm_cpu.so next to the source (portable flags: the same
    source builds on x86-64 and on Arm)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", SRC, "-o", tmp],
                       check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        L.kpm_cpu_moments.restype = C.c_int
        L.kpm_cpu_moments.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                      C.c_double, C.c_double, C.c_void_p, C.c_int, C.c_int,
                                      C.c_void_p, C.c_void_p, C.c_int]
        L.kpm_cpu_max_threads.restype = C.c_int
        _lib = L
    return _lib


def max_threads() -> int:
    return int(lib().kpm_cpu_max_threads())


def moments_doubling(H, a: float, b: float, v0, M: int, threads: int = 0):
    """Same contract as oracle.moments_doubling (H an oracle CSR, v0 an N x R
    block): returns (mu[M], mu_per_vec[R, M])."""
    cplx = bool(np.iscomplexobj(H.val) or np.iscomplexobj(v0))
    V = np.asarray(v0)
    V = V[:, None] if V.ndim == 1 else V
    N, R = V.shape
    dt = np.complex128 if cplx else np.float64
    vals = np.ascontiguousarray(np.asarray(H.val, dtype=dt))
    V = np.ascontiguousarray(V.astype(dt))
    rowptr = np.ascontiguousarray(H.rowptr, dtype=np.int64)
    col = np.ascontiguousarray(H.col, dtype=np.int64)
    mu = np.zeros(M)
    per = np.zeros((R, M))
    rc = lib().kpm_cpu_moments(N, rowptr.ctypes.data, col.ctypes.data, vals.ctypes.data,
                               int(cplx), float(a), float(b), V.ctypes.data, R, M,
                               mu.ctypes.data, per.ctypes.data, int(threads))
    if rc != 0:
        raise ValueError(f"kpm_cpu_moments returned {rc}")
    return mu, per
