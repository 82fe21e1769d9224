"""The C-ABI library without a GPU: it builds, loads, exports every entry
point declared in include/kpm.h, validates arguments before touching the
device, and its host-side lattice-to-CSR builder agrees exactly with the
oracle's independent builder."""
import ctypes as C
import shutil

import numpy as np
import pytest

import oracle as O
from paper_1105_5481_gb300 import inputs as I

nvcc = shutil.which("nvcc") or (shutil.os.path.exists("/usr/local/cuda/bin/nvcc") and "/usr/local/cuda/bin/nvcc")
pytestmark = pytest.mark.skipif(not nvcc, reason="nvcc not available")


@pytest.fixture(scope="module")
def K():
    from paper_1105_5481_gb300 import build, kpm

    build.build()
    return kpm


def test_every_declared_symbol_is_exported(K):
    names = K.declared_functions()
    assert {"kpm_create_stencil", "kpm_create_csr", "kpm_bounds", "kpm_moments", "kpm_dos",
            "kpm_destroy", "kpm_last_error"} <= set(names)
    L = C.CDLL(K.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n


def test_invalid_arguments_are_rejected_before_the_device(K):
    L = K.lib()
    h = C.c_void_p()
    d = K.kpm_stencil_desc()
    d.dims = 4
    assert L.kpm_create_stencil(C.byref(d), 0, C.byref(h)) == K.KPM_EINVAL
    assert "dims" in K.kpm_last_error()
    d.dims, d.L[0] = 1, 0
    assert L.kpm_create_stencil(C.byref(d), 0, C.byref(h)) == K.KPM_EINVAL
    d.L[0], d.t_im = 4, 0.5
    assert L.kpm_create_stencil(C.byref(d), K.KPM_REAL, C.byref(h)) == K.KPM_EINVAL
    rp = np.array([0, 2, 1], np.int64)
    col = np.zeros(2, np.int32)
    val = np.zeros(2)
    assert L.kpm_create_csr(2, rp.ctypes.data, col.ctypes.data, val.ctypes.data, 0, C.byref(h)) == K.KPM_EINVAL
    rp = np.array([0, 1, 2], np.int64)
    col = np.array([0, 5], np.int32)
    assert L.kpm_create_csr(2, rp.ctypes.data, col.ctypes.data, val.ctypes.data, 0, C.byref(h)) == K.KPM_EINVAL
    p = K.kpm_params()
    assert L.kpm_moments(None, C.byref(p), None, None, None) == K.KPM_EINVAL
    mu = np.ones(4)
    assert L.kpm_dos(mu.ctypes.data, 4, -1.0, 0.0, 8, 0, mu.ctypes.data, mu.ctypes.data, None) == K.KPM_EINVAL
    assert L.kpm_bounds(None, 10, 0.01, 0, None, None, None, None, None) == K.KPM_EINVAL
    # dense matrices: size, NULL, non-finite and non-Hermitian input
    A = I.dense_hermitian(3, 6)
    assert L.kpm_create_dense(0, A.ctypes.data, K.KPM_REAL, C.byref(h)) == K.KPM_EINVAL
    assert L.kpm_create_dense(6, None, K.KPM_REAL, C.byref(h)) == K.KPM_EINVAL
    B = A.copy()
    B[1, 4] += 1e-6
    assert L.kpm_create_dense(6, B.ctypes.data, K.KPM_REAL, C.byref(h)) == K.KPM_EINVAL
    assert "Hermitian" in K.kpm_last_error()
    B = A.copy()
    B[2, 2] = np.nan
    assert L.kpm_create_dense(6, B.ctypes.data, K.KPM_REAL, C.byref(h)) == K.KPM_EINVAL
    Z = np.ascontiguousarray(I.dense_hermitian(3, 6, True))
    Zb = Z.copy()
    Zb[0, 0] += 1e-3j                                  # a diagonal entry must be real
    assert L.kpm_create_dense(6, Zb.view(np.float64).ctypes.data, K.KPM_COMPLEX, C.byref(h)) == K.KPM_EINVAL


def test_batch_entry_points_reject_a_null_batch(K):
    # every batch call validates its handle before it touches a device
    L = K.lib()
    i1, i2 = C.c_int(), C.c_int()
    assert L.kpm_batch_set_resident(None, 1) == K.KPM_EINVAL
    assert L.kpm_batch_get_resident(None, C.byref(i1), C.byref(i2)) == K.KPM_EINVAL
    assert L.kpm_batch_set_staged(None, 1) == K.KPM_EINVAL
    assert L.kpm_batch_get_staged(None, C.byref(i1), C.byref(i2), C.byref(i1)) == K.KPM_EINVAL
    assert L.kpm_batch_set_chunk_bytes(None, 16) == K.KPM_EINVAL
    assert L.kpm_batch_get_chunk_bytes(None, C.byref(i1), C.byref(i2)) == K.KPM_EINVAL
    assert L.kpm_batch_set_rtiles(None, 2, 0) == K.KPM_EINVAL
    assert L.kpm_batch_set_config(None, 4, 4, 100) == K.KPM_EINVAL
    assert L.kpm_batch_run(None, None, None) == K.KPM_EINVAL
    assert "NULL" in K.kpm_last_error()
    out = C.c_void_p()
    assert L.kpm_batch_create(0, None, None, C.byref(out)) == K.KPM_EINVAL


def _oracle_csr(L, periodic, onsite, hop, mask, t=1.0):
    H = O.lattice_hamiltonian(L, periodic=periodic, onsite=onsite, hop=hop, mask=mask, t=t)
    return H.rowptr, H.col, H.val


@pytest.mark.parametrize("case", ["chain", "chain2", "chain1", "square_dis", "cube_spin_mask_open",
                                  "cube10"])
def test_library_csr_builder_matches_oracle(K, case):
    if case == "chain":
        L, per, on, hop, mask, cplx = (9,), (True,), None, None, None, False
    elif case == "chain2":
        L, per, on, hop, mask, cplx = (2, 3), (True, True), I.onsite_disorder(1, 6, 1.0), None, None, False
    elif case == "chain1":
        L, per, on, hop, mask, cplx = (1, 4), (True, False), None, None, None, False
    elif case == "square_dis":
        L, per, on, hop, mask, cplx = (6, 5), (True, True), I.onsite_disorder(3, 30, 2.0), None, None, False
    elif case == "cube_spin_mask_open":
        L = (5, 4, 3)
        N = 60
        per, on = (True, False, True), I.onsite_disorder(9, N, 1.0)
        hop, mask, cplx = I.spin_hoppings(L, *I.spins(9, N)), I.dilution_mask(9, N, 3), True
    else:
        L, per, on, hop, mask, cplx = (10, 10, 10), (True, True, True), np.zeros(1000), None, None, False
    rp, col, val = K.kpm_stencil_to_csr(len(L), L, per, on, hop, 1.0, mask, cplx)
    orp, ocol, oval = _oracle_csr(L, per, on, hop, mask)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(col, ocol)
    np.testing.assert_array_equal(val, oval if cplx else np.real(oval))
