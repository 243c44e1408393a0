"""The C-ABI library builds, loads and exports every entry point include/rd.h declares.

No GPU is needed: only host-side entry points (word counts, padding, argument
validation that rejects a call before any CUDA work) are called here.
"""
import ctypes

import pytest

from conftest import read_golden


@pytest.fixture(scope="module")
def rd():
    from paper_2409_17658_gb300 import build

    build.build()
    import paper_2409_17658_gb300 as rd

    return rd


def test_exports_every_declared_symbol(rd):
    names = rd.declared_symbols()
    assert len(names) >= 10
    lib = ctypes.CDLL(rd.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_state_count_matches_table1(rd):
    for m, cm in read_golden("paper_table1_counts.txt"):
        assert rd.state_count(int(m)) == int(cm)
    assert rd.state_count(1) == 4


def test_state_count_rejects_bad_m(rd):
    for m in (0, -1, rd.RD_MAX_M + 1):
        with pytest.raises(rd.RdError) as e:
            rd.state_count(m)
        assert e.value.status == rd.RD_ERR_ARG


def test_padded_dim(rd):
    assert [rd.padded_dim(n) for n in (0, 1, 7, 8, 9, 33, 21909)] == [0, 8, 8, 8, 16, 40, 21912]


def test_argument_checks_before_any_device_work(rd):
    lib = rd._lib()
    vp = ctypes.c_void_p
    # negative sizes, bad leading dimensions and misaligned pointers are refused up front
    assert lib.rd_minplus_gemm(vp(16), 8, vp(16), 8, vp(16), 8, -1, 1, 1, None, None) == rd.RD_ERR_ARG
    assert lib.rd_minplus_gemm(vp(16), 12, vp(16), 8, vp(16), 8, 4, 4, 4, None, None) == rd.RD_ERR_ARG
    assert lib.rd_minplus_gemm(vp(18), 8, vp(16), 8, vp(16), 8, 4, 4, 4, None, None) == rd.RD_ERR_ARG
    assert lib.rd_minplus_gemm(vp(16), 8, vp(16), 8, vp(16), 4, 4, 8, 4, None, None) == rd.RD_ERR_ARG
    assert lib.rd_build_transfer(3, None, 40, None) == rd.RD_ERR_ARG
    assert lib.rd_build_transfer(3, vp(256), 33, None) == rd.RD_ERR_ARG  # ld not a multiple of 8
    assert lib.rd_build_transfer(0, vp(256), 40, None) == rd.RD_ERR_ARG
    assert lib.rd_enumerate_states(16, vp(256), vp(256), None) == rd.RD_ERR_ARG
    g = (ctypes.c_int64 * 9)()
    k, p, q = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    args = (ctypes.byref(g), ctypes.byref(k), ctypes.byref(p), ctypes.byref(q), None)
    assert lib.rd_power_until_periodic(vp(256), 33, 40, 0, vp(256), 1 << 20, *args) == rd.RD_ERR_ARG
    assert lib.rd_power_until_periodic(vp(256), 33, 40, 8, vp(300), 1 << 20, *args) == rd.RD_ERR_ARG
    assert lib.rd_power_until_periodic(vp(256), 33, 40, 8, vp(256), 64, *args) == rd.RD_ERR_NOMEM
    out = ctypes.c_int64()
    assert lib.rd_gamma_R(3, 2, ctypes.byref(out)) == rd.RD_ERR_ARG  # C_n needs n >= 3
    # row-split step: sizes come from (m, j) alone; bad splits and buffers are refused up front
    sz = ctypes.c_size_t()
    for m, j in ((1, 1), (10, 0), (10, 10), (16, 8), (15, 5), (3, -1)):
        assert lib.rd_split_plan_bytes(m, j, ctypes.byref(sz)) == rd.RD_ERR_ARG, (m, j)
    info = rd.SplitInfo()
    assert lib.rd_split_plan(10, 5, vp(300), 1 << 30, ctypes.byref(info), None) == rd.RD_ERR_ARG
    assert lib.rd_split_plan(10, 5, vp(256), 64, ctypes.byref(info), None) == rd.RD_ERR_NOMEM
    assert lib.rd_split_minplus(ctypes.byref(info), vp(256), vp(256), 8, vp(256), 8, vp(256), 8, None,
                                None) == rd.RD_ERR_ARG  # info of no built plan (m = 0)
    assert lib.rd_gamma_R(0, 5, ctypes.byref(out)) == rd.RD_ERR_ARG


def test_work_layout(rd):
    n, ld, kmax = 33, 40, 16
    b2 = rd.power_work_bytes(n, ld, kmax, 2)
    b5 = rd.power_work_bytes(n, ld, kmax, 5)
    slot = b5 - rd.power_work_bytes(n, ld, kmax, 4)
    assert slot >= n * ld * 2 and slot % 256 == 0 and b5 - b2 == 3 * slot
    offs = [rd.power_slot(n, ld, kmax, b5, k) for k in range(1, 11)]
    assert len(set(offs[:5])) == 5 and offs[5] == offs[0]  # P_k lives in slot k mod 5
    # power 0's slot (where a caller short of memory may build A) is the one P_5 later fills
    assert rd.power_slot(n, ld, kmax, b5, 0) == offs[4]
    with pytest.raises(rd.RdError):
        rd.power_slot(n, ld, kmax, b5, -1)


def test_split_plan_sizes(rd):
    assert [rd.split_default_j(m) for m in (1, 2, 3, 9, 10, 11, 15, 16)] == [0, 1, 1, 4, 5, 6, 8, 0]
    b = {j: rd.split_plan_bytes(10, j) for j in range(2, 9)}
    # the plan is small next to one 64769 x 64776 int16 matrix (8.4 GB), smallest for the balanced split
    assert all(0 < v < 256 << 20 for v in b.values())
    assert min(b, key=b.get) == rd.split_default_j(10) and b[5] < 64 << 20
    assert rd.split_plan_bytes(2, 1) < rd.split_plan_bytes(3, 1) < rd.split_plan_bytes(4, 2)


def test_split_check_flags_absent_in_the_normal_build(rd):
    """The normal build compiles no index checks: rd_split_check_flags answers RD_NOT_FOUND with no CUDA call."""
    assert rd.split_check_flags() is None
    assert rd._lib().rd_split_check_flags(None, 0) == rd.RD_ERR_ARG
