"""rd_power_until_periodic_noalloc: the period search on the library's static scratch.

For callers that cannot allocate device memory (their memory belongs to another
allocator, or allocation is forbidden or too slow where they run).  The entry
point is called through the C ABI and its results are compared with those of
rd_power_until_periodic, which uses a caller-owned work buffer, and with the CPU
oracle, on three calls in a row: m = 7 and m = 5 take the multi-kernel dense
step (the larger first, so the second starts from the first one's leftover
scratch contents), and m = 3 the single-CTA search.  This file is collected last
on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib_and_torch():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    from paper_2409_17658_gb300 import build

    build.build()
    import paper_2409_17658_gb300 as rd

    return rd, rd._lib(), torch


def call_noalloc(lib, torch, A, n, kmax):
    gamma = np.zeros(kmax + 1, dtype=np.int64)
    k, p, q = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    st = lib.rd_power_until_periodic_noalloc(ctypes.c_void_p(A.data_ptr()), n, A.stride(0), kmax,
                                             ctypes.c_void_p(gamma.ctypes.data), ctypes.byref(k), ctypes.byref(p),
                                             ctypes.byref(q), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, gamma, (k.value, p.value, q.value)


def call_with_work(lib, torch, rd, A, n, kmax):
    work = rd.power_workspace(n, A.stride(0), kmax, 8)
    gamma = np.zeros(kmax + 1, dtype=np.int64)
    k, p, q = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    st = lib.rd_power_until_periodic(ctypes.c_void_p(A.data_ptr()), n, A.stride(0), kmax,
                                     ctypes.c_void_p(work.data_ptr()), work.numel(),
                                     ctypes.c_void_p(gamma.ctypes.data), ctypes.byref(k), ctypes.byref(p),
                                     ctypes.byref(q), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, gamma, (k.value, p.value, q.value)


def test_noalloc_matches_work_buffer_entry_point(lib_and_torch, orc):
    rd, lib, torch = lib_and_torch
    kmax = 48
    for m in (7, 5, 3):  # calls in a row, the larger problems first
        A, n = rd.transfer_matrix(m)
        st_ref, g_ref, t_ref = call_with_work(lib, torch, rd, A, n, kmax)
        st, g, t = call_noalloc(lib, torch, A, n, kmax)
        assert st_ref == rd.RD_OK
        assert st == st_ref and t == t_ref, (m, st, t, t_ref)
        assert np.array_equal(g, g_ref), m  # integer results: exact
        o = orc.power_until_periodic(m, kmax=kmax)
        assert t == (o["k"], o["p"], o["q"]), (m, t, o)
        assert np.array_equal(g[1:o["j"] + 1], o["gamma"][1:o["j"] + 1]), m


def test_noalloc_rejects_problems_beyond_its_scratch(lib_and_torch):
    rd, lib, torch = lib_and_torch
    A, n = rd.transfer_matrix(8)  # N = 7411: two powers alone need ~220 MB > RD_NOALLOC_SCRATCH_BYTES
    assert rd.power_work_bytes(n, A.stride(0), 30, 2) > 96 * 1024 * 1024
    st, g, _ = call_noalloc(lib, torch, A, n, 30)
    assert st == rd.RD_ERR_NOMEM
